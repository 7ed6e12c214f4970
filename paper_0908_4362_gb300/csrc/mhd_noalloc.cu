// Allocation-free FP64 field sums (declared in include/mhd.h as mhd_sums_noalloc).
//
// Some callers cannot allocate device memory: code that runs inside a process whose device
// memory is owned by another allocator under a fixed budget (a serving loop that has
// handed all of its HBM to resident simulations), or a host thread that must not trigger
// the device-wide synchronisation that cudaMalloc and cudaFree imply while other work is
// in flight.  For them this file keeps the reduction's scratch (one row of 8 partial sums
// per block, plus the 8 results) in a fixed array in device global memory that is part of
// the library image: every GPU that loads the library holds it until the process exits.
//
// The first call on a device looks up the array's device address with
// cudaGetSymbolAddress (with that device current) and remembers it.  Every call shares the
// one array: calls whose work overlaps on the GPU race on it, so the caller serialises them
// (one stream, or synchronise between calls).  Each call writes every scratch slot it later reads, so
// nothing left by an earlier call needs clearing.
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/mhd.h"
#include "mhd_kernels.cuh"

namespace {

constexpr long long kCellsPerBlock = 256LL * 256LL;        // one partial row per 65536 cells
constexpr int kMaxPartials = (int)(MHD_SUMS_NOALLOC_MAX_CELLS / kCellsPerBlock);
static_assert(kMaxPartials * kCellsPerBlock == MHD_SUMS_NOALLOC_MAX_CELLS, "scratch size");

// 4096 rows x 8 partial sums + 8 results = 262,208 bytes
static __device__ __align__(256) double g_sums_scratch[kMaxPartials * 8 + 8];

constexpr int kMaxDevices = 64;
std::mutex g_lock;
double* g_scratch_ptr[kMaxDevices] = {};

// device address of the scratch array on the current device (looked up once per device)
cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_lock);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_sums_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

template <typename T>
cudaError_t launch_sums(const void* const f[8], long long n, int nblocks, double* scratch,
                        cudaStream_t s) {
  mhd::FieldSet<T> fs;
  for (int k = 0; k < 8; ++k) fs.f[k] = (T*)f[k];
  mhd::sums_partial_kernel<T><<<nblocks, 256, 0, s>>>(n, fs, scratch);
  mhd::sums_final_kernel<<<1, 32, 0, s>>>(nblocks, scratch, scratch + (size_t)kMaxPartials * 8);
  return cudaGetLastError();
}

}  // namespace

extern "C" mhd_status mhd_sums_noalloc(const void* const f[8], int dtype, long long n,
                                       double out[8], void* stream) {
  if (!f || !out || (dtype != 0 && dtype != 1) || n < 1) return MHD_ERR_INVALID;
  if (n > MHD_SUMS_NOALLOC_MAX_CELLS) return MHD_ERR_INVALID;
  for (int k = 0; k < 8; ++k)
    if (!f[k]) return MHD_ERR_INVALID;
  double* scratch = nullptr;
  if (scratch_address(&scratch) != cudaSuccess) return MHD_ERR_CUDA;
  const int nblocks = (int)((n + kCellsPerBlock - 1) / kCellsPerBlock);
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = dtype == 0 ? launch_sums<float>(f, n, nblocks, scratch, s)
                             : launch_sums<double>(f, n, nblocks, scratch, s);
  if (e != cudaSuccess) return MHD_ERR_CUDA;
  e = cudaMemcpyAsync(out, scratch + (size_t)kMaxPartials * 8, 8 * sizeof(double),
                      cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return MHD_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return MHD_ERR_CUDA;
  return MHD_OK;
}
