// Device side of the batched persistent form (mhd_batch.cu holds the host side): the work
// items, the tile bodies each item runs, and the persistent kernel, a template over the
// threads per CTA (NT = 128 or 256), instantiated in mhd_batch_nt128.cu and
// mhd_batch_nt256.cu.
//
// The operations are those of one method step (Sect. 4.2, Eq. "eq:L_sequence"): dt from
// the previous step's c_max, then the forward and reverse sweeps of the instance's phase.
// Every tile runs the same device bodies as the standalone kernels (FP32), so each grid's
// result is bit-identical to advancing it alone with mhd_step, whatever the tile shape.
// Loads of the z segments inside the persistent launch use coherent paths (no read-only
// cache), because the buffers are rewritten by other CTAs during the launch.
#pragma once

#include <cuda_runtime.h>

#include "mhd_flat.cuh"
#include "mhd_march.cuh"
#include "mhd_segz.cuh"

namespace mhd {

constexpr long long kSpinCycles = 4000000000LL;   // ~2 s of SM clock per wait
constexpr long long kAutoTiles = 1024;            // target items per z sweep when not set
constexpr int kFlatPerThread = 16;                // cells per thread of a per-cell item
// OP_NOP: a fluid sweep along a flat axis (identity, no items); OP_CMAX: c_max of the state
// (the last fluid sweep of a step along a flat axis); OP_CTFLAT: CT along a flat axis
enum : int { OP_DT = 0, OP_FLUID = 1, OP_CT = 2, OP_NOP = 3, OP_CMAX = 4, OP_CTFLAT = 5 };

struct BatchOp {
  FieldSet<float> in, out;
  GridDesc g;
  int kind, axis, last;
  int rows;            // CT x/y in the shared-row form (ct_rows_xy_tile)
  int s;               // x/y: cells per marching tile along the sweep (128, 192, 256)
  int segk;            // z segments: cells per lane (2 or 3)
  int gx;              // march: tiles across the transverse plane (tile = by * gx + bx)
  int wpt;             // z segments: warp segments per tile
  long long nwarps;    // z segments: warp segments of the sweep
  int tiles;
};
struct BatchItem {
  int inst, op, tile, need;
};
struct BatchInst {
  DevScalars* ds;
  float gamma;
  double h, cfl_h;
};
struct BatchArgs {
  const BatchItem* items;
  long long nitems;
  const BatchOp* ops;
  const BatchInst* inst;
  unsigned long long* queue;
  int* done;
  int* abort;
  int* status;
  long long spin_limit;
};

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_relaxed(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

template <int A, int S, int NT>
__device__ __forceinline__ void batch_fluid_xy_s(const BatchOp& op, const BatchInst& in,
                                                 unsigned tile, unsigned char* smem) {
  const unsigned bx = tile % op.gx, by = tile / op.gx;
  if (op.last)
    fluid_march_xy_tile<float, A, true, PM_FP32, S, NT>(op.g, op.in, op.out, in.gamma, in.h,
                                                        in.ds, bx, by, smem);
  else
    fluid_march_xy_tile<float, A, false, PM_FP32, S, NT>(op.g, op.in, op.out, in.gamma, in.h,
                                                         in.ds, bx, by, smem);
}

template <int A, int S, int NT>
__device__ __forceinline__ void batch_ct_xy_s(const BatchOp& op, const BatchInst& in,
                                              unsigned tile, unsigned char* smem) {
  const unsigned bx = tile % op.gx, by = tile / op.gx;
  if (op.rows)
    ct_rows_xy_tile<float, A, S, NT / 32>(op.g, op.in, op.out, in.h, in.ds, bx, by, smem);
  else
    ct_march_xy_tile<float, A, S, NT>(op.g, op.in, op.out, in.h, in.ds, bx, by, smem);
}

// the marching tile lengths a batched grid may take (kMarchS is the single-grid kernels')
__host__ __device__ inline bool batch_len_ok(int s) { return s == 128 || s == 192 || s == 256; }

template <int A, int NT>
__device__ __forceinline__ void batch_xy(const BatchOp& op, const BatchInst& in, unsigned tile,
                                         unsigned char* smem) {
  if (op.kind == OP_FLUID) {
    if (op.s == 128) batch_fluid_xy_s<A, 128, NT>(op, in, tile, smem);
    else if (op.s == 256) batch_fluid_xy_s<A, 256, NT>(op, in, tile, smem);
    else batch_fluid_xy_s<A, 192, NT>(op, in, tile, smem);
  } else {
    if (op.s == 128) batch_ct_xy_s<A, 128, NT>(op, in, tile, smem);
    else if (op.s == 256) batch_ct_xy_s<A, 256, NT>(op, in, tile, smem);
    else batch_ct_xy_s<A, 192, NT>(op, in, tile, smem);
  }
}

template <int K>
__device__ __forceinline__ void batch_seg_z(const BatchOp& op, const BatchInst& ins,
                                            long long w) {
  if (op.kind == OP_FLUID) {
    if (op.last)
      fluid_seg_z_warp<float, true, PM_FP32, K, false>(op.g, op.in, op.out, ins.gamma, ins.h,
                                                       ins.ds, w);
    else
      fluid_seg_z_warp<float, false, PM_FP32, K, false>(op.g, op.in, op.out, ins.gamma, ins.h,
                                                        ins.ds, w);
  } else {
    ct_seg_z_warp<float, K, false>(op.g, op.in, op.out, ins.h, ins.ds, w);
  }
}

// 16 resident warps per SM (a 128-register cap, with a few bytes of spill) measured 10%
// faster than 12 on the 64-instance batched workload
#ifndef MHD_BATCH_MINB
#define MHD_BATCH_MINB 4
#endif
template <int NT>
__global__ void __launch_bounds__(NT, MHD_BATCH_MINB * 128 / NT) batch_kernel(BatchArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ long long s_id;
  __shared__ int s_go;
  for (;;) {
    if (threadIdx.x == 0) {
      const long long id = (long long)atomicAdd(a.queue, 1ull);
      int go = id < a.nitems ? 1 : 0;
      if (go) {
        const BatchItem it = a.items[id];
        // poll with relaxed loads (cheaper than GPU-scope acquire loads, which must order
        // every later load of the SM), then one acquire load once the count is reached: it
        // reads a value of the counter's release sequence
        if (ld_acquire(a.done + it.inst) < it.need) {
          const long long t0 = clock64();
          while (ld_relaxed(a.done + it.inst) < it.need) {
            if (ld_relaxed(a.abort)) { go = 0; break; }
            if (clock64() - t0 > a.spin_limit) {
              atomicOr(a.status, 1);
              atomicExch(a.abort, 1);
              go = 0;
              break;
            }
            __nanosleep(64);
          }
          if (go) (void)ld_acquire(a.done + it.inst);
        }
      }
      s_id = id;
      s_go = go;
    }
    __syncthreads();
    if (!s_go) break;
    const BatchItem it = a.items[s_id];
    const BatchOp& op = a.ops[it.op];
    const BatchInst& ins = a.inst[it.inst];
    const int warp = threadIdx.x >> 5;
    if (op.kind == OP_DT) {
      if (threadIdx.x == 0) dt_update<float>(ins.ds, ins.cfl_h, ins.h);
    } else if (op.kind == OP_CMAX || op.kind == OP_CTFLAT) {
      constexpr int kFlat = NT * kFlatPerThread;
      const long long N = (long long)op.g.n[0] * op.g.n[1] * op.g.n[2];
      const long long i0 = (long long)it.tile * kFlat;
      const long long i1 = min(i0 + kFlat, N);
      if (op.kind == OP_CMAX) {
        cmax_range<float, PM_FP32>(op.g, op.in, ins.gamma, ins.ds, i0 + threadIdx.x, i1, NT);
      } else {
        const float dth = step_factor<float>(ins.ds, ins.h);
        int st;
        if (op.axis == 0)
          st = ct_flat_range<float, 0>(op.g, op.in, op.out, dth, i0 + threadIdx.x, i1, NT);
        else if (op.axis == 1)
          st = ct_flat_range<float, 1>(op.g, op.in, op.out, dth, i0 + threadIdx.x, i1, NT);
        else
          st = ct_flat_range<float, 2>(op.g, op.in, op.out, dth, i0 + threadIdx.x, i1, NT);
        if (st) atomicOr(&ins.ds->status, st);
      }
    } else if (op.axis < 2) {
      if (op.axis == 0) batch_xy<0, NT>(op, ins, it.tile, smem_raw);
      else batch_xy<1, NT>(op, ins, it.tile, smem_raw);
    } else {
      const long long w0 = (long long)it.tile * op.wpt;
      const long long w1 = min(w0 + op.wpt, op.nwarps);
      for (long long w = w0 + warp; w < w1; w += NT / 32) {
        if (op.segk == 2) batch_seg_z<2>(op, ins, w);
        else batch_seg_z<3>(op, ins, w);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(a.done + it.inst, 1);
    }
  }
}

// dynamic shared memory of the largest tile body at NT threads: the per-element CT march's
// prefetch ring (15 values per iteration), the fluid staging, the shared-row CT
template <int NT>
inline size_t batch_smem() {
  size_t m = sizeof(float) * (size_t)kMarchRing * 15 * NT;
  m = m > march_tile_smem<float>(NT) ? m : march_tile_smem<float>(NT);
  const size_t r = ct_rows_smem<float>(NT / 32);
  return m > r ? m : r;
}

// host entry points of one instantiation (mhd_batch_nt128.cu, mhd_batch_nt256.cu)
struct BatchKernel {
  int nt;
  size_t smem;
  cudaError_t (*prepare)(int* ctas_per_sm);            // attributes + occupancy
  cudaError_t (*launch)(int grid, cudaStream_t s, const BatchArgs& a);
};
const BatchKernel& batch_kernel_nt128();
const BatchKernel& batch_kernel_nt256();

#define MHD_BATCH_INSTANTIATE(NTV)                                                          \
  namespace mhd {                                                                           \
  static cudaError_t batch_prepare_##NTV(int* per_sm) {                                     \
    cudaError_t e = cudaFuncSetAttribute(batch_kernel<NTV>,                                 \
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,       \
                                         (int)batch_smem<NTV>());                           \
    if (e == cudaSuccess)                                                                   \
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, batch_kernel<NTV>, NTV,     \
                                                        batch_smem<NTV>());                 \
    return e;                                                                               \
  }                                                                                         \
  static cudaError_t batch_launch_##NTV(int grid, cudaStream_t s, const BatchArgs& a) {     \
    batch_kernel<NTV><<<grid, NTV, batch_smem<NTV>(), s>>>(a);                              \
    return cudaGetLastError();                                                              \
  }                                                                                         \
  const BatchKernel& batch_kernel_nt##NTV() {                                               \
    static const BatchKernel k{NTV, batch_smem<NTV>(), batch_prepare_##NTV,                 \
                               batch_launch_##NTV};                                         \
    return k;                                                                               \
  }                                                                                         \
  }

}  // namespace mhd
