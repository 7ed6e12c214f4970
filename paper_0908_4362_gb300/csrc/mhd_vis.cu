// Visualization of a state without a graphics API (Sect. 8).
//
// The paper maps the state into OpenGL buffers: a vertex per cell for 1D problems (x
// position, selected value), a pixel per cell of a 2D problem coloured through a transfer
// function, and a texture volume render for 3D.  Here the same products are written into
// device buffers by CUDA kernels: a curve of (x, q) pairs, an RGBA8 colour image of a plane
// of cells, and an orthographic emission-absorption ray cast through the volume (one ray per
// cell column along an axis, front to back).  The selected value q is one of rho, p, E,
// |v|, |B| per cell, with B averaged from the faces to the cell centre.  Arithmetic is in
// the state's precision.
#include <cstring>
#include <string>

#include <cuda_runtime.h>

#include "../../include/mhd.h"
#include "mhd_ctx.h"
#include "mhd_kernels.cuh"

namespace mhd {

// q of cell i (coordinates c)
template <typename T>
__device__ __forceinline__ T vis_value(const GridDesc& g, const FieldSet<T>& f, int quantity,
                                       T gamma, long long i, const int c[3]) {
  const T rho = f.f[0][i];
  if (quantity == MHD_Q_RHO) return rho;
  const T E = f.f[4][i];
  if (quantity == MHD_Q_E) return E;
  const T m0 = f.f[1][i], m1 = f.f[2][i], m2 = f.f[3][i];
  const T mm = m0 * m0 + m1 * m1 + m2 * m2;
  if (quantity == MHD_Q_VMAG) return sqrt(mm) / rho;
  T bb = T(0);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const long long up = i + (long long)(wrap_index(c[a] + 1, g.n[a], g.bc[a]) - c[a]) * g.s[a];
    const T b = T(0.5) * (f.f[5 + a][i] + f.f[5 + a][up]);
    bb += b * b;
  }
  if (quantity == MHD_Q_BMAG) return sqrt(bb);
  return (gamma - T(1)) * (E - T(0.5) * mm / rho - T(0.5) * bb);   // MHD_Q_P
}

__device__ __forceinline__ void cell_coords(const GridDesc& g, long long i, int c[3]) {
  c[2] = (int)(i % g.n[2]);
  const long long xy = i / g.n[2];
  c[1] = (int)(xy % g.n[1]);
  c[0] = (int)(xy / g.n[1]);
}

// transfer function: s in [0, 1] -> colour on a five-stop ramp (dark blue, blue, cyan,
// yellow, red), linear between the stops
template <typename T>
__device__ __forceinline__ void ramp(T s, T rgb[3]) {
  const T stops[5][3] = {{0, 0, T(0.5)}, {0, 0, 1}, {0, 1, 1}, {1, 1, 0}, {1, 0, 0}};
  if (!(s > T(0))) s = T(0);            // also NaN
  else if (s > T(1)) s = T(1);
  const T x = s * T(4);
  int k = (int)x;
  if (k > 3) k = 3;
  const T w = x - T(k);
#pragma unroll
  for (int q = 0; q < 3; ++q) rgb[q] = stops[k][q] + w * (stops[k + 1][q] - stops[k][q]);
}

template <typename T>
__device__ __forceinline__ T normalise(T q, T vmin, T vmax) {
  return (q - vmin) / (vmax - vmin);
}

template <typename T>
__global__ void vis_curve_kernel(GridDesc g, FieldSet<T> f, int quantity, T gamma, int axis,
                                 double h, float* xy) {
  const long long n = g.n[axis];
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n;
       j += (long long)gridDim.x * blockDim.x) {
    int c[3] = {0, 0, 0};
    c[axis] = (int)j;
    const long long i = (long long)j * g.s[axis];
    xy[2 * j] = (float)((j + 0.5) * h);
    xy[2 * j + 1] = (float)vis_value<T>(g, f, quantity, gamma, i, c);
  }
}

// plane normal to `axis` at `index`: image axes u < v are the other two, pixel (row v, col u)
template <typename T>
__global__ void vis_slice_kernel(GridDesc g, FieldSet<T> f, int quantity, T gamma, int axis,
                                 int index, T vmin, T vmax, unsigned char* rgba) {
  const int ua = axis == 0 ? 1 : 0, va = axis == 2 ? 1 : 2;
  const long long w = g.n[ua], npix = w * g.n[va];
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npix;
       p += (long long)gridDim.x * blockDim.x) {
    int c[3];
    c[axis] = index;
    c[ua] = (int)(p % w);
    c[va] = (int)(p / w);
    const long long i = (long long)c[0] * g.s[0] + (long long)c[1] * g.s[1] + c[2];
    T rgb[3];
    ramp<T>(normalise<T>(vis_value<T>(g, f, quantity, gamma, i, c), vmin, vmax), rgb);
#pragma unroll
    for (int q = 0; q < 3; ++q) rgba[4 * p + q] = (unsigned char)(rgb[q] * T(255) + T(0.5));
    rgba[4 * p + 3] = 255;
  }
}

// one ray per column along `axis` (increasing index = front to back): with the cell's
// colour c and opacity alpha = clamp(opacity * s, 0, 1),
//   C += (1 - A) alpha c,  A += (1 - A) alpha
template <typename T>
__global__ void vis_volume_kernel(GridDesc g, FieldSet<T> f, int quantity, T gamma, int axis,
                                  T vmin, T vmax, T opacity, float* rgba) {
  const int ua = axis == 0 ? 1 : 0, va = axis == 2 ? 1 : 2;
  const long long w = g.n[ua], npix = w * g.n[va];
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npix;
       p += (long long)gridDim.x * blockDim.x) {
    int c[3];
    c[ua] = (int)(p % w);
    c[va] = (int)(p / w);
    T C[3] = {0, 0, 0}, A = 0;
    for (int k = 0; k < g.n[axis]; ++k) {
      c[axis] = k;
      const long long i = (long long)c[0] * g.s[0] + (long long)c[1] * g.s[1] + c[2];
      const T s = normalise<T>(vis_value<T>(g, f, quantity, gamma, i, c), vmin, vmax);
      T rgb[3];
      ramp<T>(s, rgb);
      T al = opacity * s;
      if (!(al > T(0))) al = T(0);      // also NaN
      else if (al > T(1)) al = T(1);
      const T wgt = (T(1) - A) * al;
#pragma unroll
      for (int q = 0; q < 3; ++q) C[q] += wgt * rgb[q];
      A += wgt;
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) rgba[4 * p + q] = (float)C[q];
    rgba[4 * p + 3] = (float)A;
  }
}

// min and max of q over the grid (per-block partials, folded by atomics on ordered bits)
__device__ __forceinline__ unsigned long long ordered_bits(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

template <typename T>
__global__ void vis_range_kernel(GridDesc g, FieldSet<T> f, int quantity, T gamma,
                                 unsigned long long* lohi) {
  const long long N = (long long)g.n[0] * g.n[1] * g.n[2];
  double lo = 1e308, hi = -1e308;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    int c[3];
    cell_coords(g, i, c);
    const double q = (double)vis_value<T>(g, f, quantity, gamma, i, c);
    lo = fmin(lo, q);
    hi = fmax(hi, q);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(lohi, ordered_bits(lo));
    atomicMax(lohi + 1, ordered_bits(hi));
  }
}

}  // namespace mhd

using mhd::FieldSet;

namespace {

template <typename T>
FieldSet<T> current_fields(const mhd_ctx* ctx) {
  FieldSet<T> f;
  for (int k = 0; k < 8; ++k) f.f[k] = (T*)ctx->buf[ctx->cur[k]][k];
  return f;
}

unsigned vis_blocks(long long n) {
  long long b = (n + 255) / 256;
  if (b > 152 * 8) b = 152 * 8;
  return (unsigned)(b < 1 ? 1 : b);
}

mhd_status vis_check(mhd_ctx* ctx, int quantity) {
  if (!ctx || quantity < MHD_Q_RHO || quantity > MHD_Q_BMAG) return MHD_ERR_INVALID;
  return MHD_OK;
}

mhd_status vis_done(mhd_ctx* ctx, cudaError_t e, const char* what) {
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) {
    ctx->err = std::string(what) + ": " + cudaGetErrorString(e);
    return MHD_ERR_CUDA;
  }
  return MHD_OK;
}

double ordered_to_double(unsigned long long b) {
  b = (b >> 63) ? (b & 0x7fffffffffffffffull) : ~b;
  double v;
  memcpy(&v, &b, sizeof(v));
  return v;
}

}  // namespace

extern "C" {

mhd_status mhd_vis_curve(mhd_ctx* ctx, int quantity, float* xy) {
  mhd_status s = vis_check(ctx, quantity);
  if (s != MHD_OK) return s;
  if (!xy) return MHD_ERR_INVALID;
  int axis = -1, long_axes = 0;
  for (int a = 0; a < 3; ++a)
    if (ctx->g.n[a] > 1) { axis = a; ++long_axes; }
  if (long_axes > 1) return MHD_ERR_INVALID;     // a curve needs a 1D grid
  if (axis < 0) axis = 0;
  const long long n = ctx->g.n[axis];
  if (ctx->esz == 4)
    mhd::vis_curve_kernel<float><<<vis_blocks(n), 256, 0, ctx->stream>>>(
        ctx->g, current_fields<float>(ctx), quantity, (float)ctx->cfg.gamma, axis, ctx->cfg.h, xy);
  else
    mhd::vis_curve_kernel<double><<<vis_blocks(n), 256, 0, ctx->stream>>>(
        ctx->g, current_fields<double>(ctx), quantity, ctx->cfg.gamma, axis, ctx->cfg.h, xy);
  return vis_done(ctx, cudaGetLastError(), "vis curve");
}

mhd_status mhd_vis_slice(mhd_ctx* ctx, int quantity, int axis, int index, double vmin, double vmax,
                         unsigned char* rgba) {
  mhd_status s = vis_check(ctx, quantity);
  if (s != MHD_OK) return s;
  if (!rgba || axis < 0 || axis > 2 || index < 0 || index >= ctx->g.n[axis] || !(vmax > vmin))
    return MHD_ERR_INVALID;
  const int ua = axis == 0 ? 1 : 0, va = axis == 2 ? 1 : 2;
  const long long npix = (long long)ctx->g.n[ua] * ctx->g.n[va];
  if (ctx->esz == 4)
    mhd::vis_slice_kernel<float><<<vis_blocks(npix), 256, 0, ctx->stream>>>(
        ctx->g, current_fields<float>(ctx), quantity, (float)ctx->cfg.gamma, axis, index,
        (float)vmin, (float)vmax, rgba);
  else
    mhd::vis_slice_kernel<double><<<vis_blocks(npix), 256, 0, ctx->stream>>>(
        ctx->g, current_fields<double>(ctx), quantity, ctx->cfg.gamma, axis, index, vmin, vmax,
        rgba);
  return vis_done(ctx, cudaGetLastError(), "vis slice");
}

mhd_status mhd_vis_volume(mhd_ctx* ctx, int quantity, int axis, double vmin, double vmax,
                          double opacity, float* rgba) {
  mhd_status s = vis_check(ctx, quantity);
  if (s != MHD_OK) return s;
  if (!rgba || axis < 0 || axis > 2 || !(vmax > vmin) || !(opacity >= 0.0)) return MHD_ERR_INVALID;
  const int ua = axis == 0 ? 1 : 0, va = axis == 2 ? 1 : 2;
  const long long npix = (long long)ctx->g.n[ua] * ctx->g.n[va];
  if (ctx->esz == 4)
    mhd::vis_volume_kernel<float><<<vis_blocks(npix), 256, 0, ctx->stream>>>(
        ctx->g, current_fields<float>(ctx), quantity, (float)ctx->cfg.gamma, axis, (float)vmin,
        (float)vmax, (float)opacity, rgba);
  else
    mhd::vis_volume_kernel<double><<<vis_blocks(npix), 256, 0, ctx->stream>>>(
        ctx->g, current_fields<double>(ctx), quantity, ctx->cfg.gamma, axis, vmin, vmax, opacity,
        rgba);
  return vis_done(ctx, cudaGetLastError(), "vis volume");
}

mhd_status mhd_vis_range(mhd_ctx* ctx, int quantity, double* vmin, double* vmax) {
  mhd_status s = vis_check(ctx, quantity);
  if (s != MHD_OK) return s;
  if (!vmin || !vmax) return MHD_ERR_INVALID;
  // the context's FP64 sums scratch holds the two words (it is at least 8 doubles)
  unsigned long long* lohi = (unsigned long long*)ctx->sums_out;
  const unsigned long long init[2] = {~0ull, 0ull};
  cudaError_t e = cudaMemcpyAsync(lohi, init, sizeof(init), cudaMemcpyHostToDevice, ctx->stream);
  const long long N = ctx->N;
  if (e == cudaSuccess) {
    if (ctx->esz == 4)
      mhd::vis_range_kernel<float><<<vis_blocks(N), 256, 0, ctx->stream>>>(
          ctx->g, current_fields<float>(ctx), quantity, (float)ctx->cfg.gamma, lohi);
    else
      mhd::vis_range_kernel<double><<<vis_blocks(N), 256, 0, ctx->stream>>>(
          ctx->g, current_fields<double>(ctx), quantity, ctx->cfg.gamma, lohi);
    e = cudaGetLastError();
  }
  unsigned long long h[2] = {0, 0};
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h, lohi, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream);
  if ((s = vis_done(ctx, e, "vis range")) != MHD_OK) return s;
  *vmin = ordered_to_double(h[0]);
  *vmax = ordered_to_double(h[1]);
  return MHD_OK;
}

}  // extern "C"
