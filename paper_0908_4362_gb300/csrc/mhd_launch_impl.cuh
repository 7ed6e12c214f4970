// Launcher bodies shared by the per-precision translation units.
#pragma once

#include "mhd_kernels.cuh"
#include "mhd_launch.h"

namespace mhd {

template <typename T>
static size_t fluid_smem() {
  constexpr int E = FluidTile<T>::S + 6;
  return sizeof(T) * 23 * (size_t)E * FluidTile<T>::W;
}
template <typename T>
static size_t ct_smem() {
  constexpr int E = CtTile<T>::S + 8, R = 3 * CtTile<T>::W + 1;
  return sizeof(T) * 4 * (size_t)E * R;
}

template <typename T, int A, bool LAST, bool P64>
static cudaError_t set_fluid_attr() {
  return cudaFuncSetAttribute(fluid_kernel<T, A, LAST, P64>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fluid_smem<T>());
}
template <typename T, int A>
static cudaError_t set_ct_attr() {
  return cudaFuncSetAttribute(ct_kernel<T, A>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)ct_smem<T>());
}

template <typename T, bool P64>
static cudaError_t setup_p() {
  cudaError_t e = cudaSuccess;
#define MHD_TRY(x) do { cudaError_t _e = (x); if (_e != cudaSuccess) e = _e; } while (0)
  MHD_TRY((set_fluid_attr<T, 0, false, P64>()));
  MHD_TRY((set_fluid_attr<T, 1, false, P64>()));
  MHD_TRY((set_fluid_attr<T, 2, false, P64>()));
  MHD_TRY((set_fluid_attr<T, 0, true, P64>()));
  MHD_TRY((set_fluid_attr<T, 1, true, P64>()));
  MHD_TRY((set_fluid_attr<T, 2, true, P64>()));
#undef MHD_TRY
  return e;
}

template <typename T>
static dim3 tile_grid(const GridDesc& g, int axis, int S, int W) {
  const int wa = axis_w(axis), oa = axis_o(axis);
  return dim3((unsigned)((g.n[axis] + S - 1) / S), (unsigned)((g.n[wa] + W - 1) / W),
              (unsigned)g.n[oa]);
}

template <typename T, bool LAST, bool P64>
static void fluid_dispatch(const GridDesc& g, const FieldSet<T>& in, const FieldSet<T>& out,
                           T gamma, double h, DevScalars* ds, int axis, cudaStream_t s) {
  const dim3 grid = tile_grid<T>(g, axis, FluidTile<T>::S, FluidTile<T>::W);
  const size_t sm = fluid_smem<T>();
  switch (axis) {
    case 0: fluid_kernel<T, 0, LAST, P64><<<grid, FluidTile<T>::NT, sm, s>>>(g, in, out, gamma, h, ds); break;
    case 1: fluid_kernel<T, 1, LAST, P64><<<grid, FluidTile<T>::NT, sm, s>>>(g, in, out, gamma, h, ds); break;
    default: fluid_kernel<T, 2, LAST, P64><<<grid, FluidTile<T>::NT, sm, s>>>(g, in, out, gamma, h, ds); break;
  }
}

template <typename T>
static cudaError_t fluid_impl(const GridDesc& g, const FieldSet<T>& in, const FieldSet<T>& out,
                              double gamma, double h, DevScalars* ds, int axis, bool last,
                              bool p64, cudaStream_t s) {
  const T gm = (T)gamma;
  if (last) {
    if (p64) fluid_dispatch<T, true, true>(g, in, out, gm, h, ds, axis, s);
    else fluid_dispatch<T, true, false>(g, in, out, gm, h, ds, axis, s);
  } else {
    if (p64) fluid_dispatch<T, false, true>(g, in, out, gm, h, ds, axis, s);
    else fluid_dispatch<T, false, false>(g, in, out, gm, h, ds, axis, s);
  }
  return cudaGetLastError();
}

template <typename T>
static cudaError_t ct_impl(const GridDesc& g, const FieldSet<T>& in, const FieldSet<T>& out,
                           double h, DevScalars* ds, int axis, cudaStream_t s) {
  const dim3 grid = tile_grid<T>(g, axis, CtTile<T>::S, CtTile<T>::W);
  const size_t sm = ct_smem<T>();
  switch (axis) {
    case 0: ct_kernel<T, 0><<<grid, CtTile<T>::NT, sm, s>>>(g, in, out, h, ds); break;
    case 1: ct_kernel<T, 1><<<grid, CtTile<T>::NT, sm, s>>>(g, in, out, h, ds); break;
    default: ct_kernel<T, 2><<<grid, CtTile<T>::NT, sm, s>>>(g, in, out, h, ds); break;
  }
  return cudaGetLastError();
}

template <typename T>
static cudaError_t cmax_impl(const GridDesc& g, const FieldSet<T>& in, double gamma,
                             DevScalars* ds, bool p64, cudaStream_t s) {
  const long long N = (long long)g.n[0] * g.n[1] * g.n[2];
  long long nb = (N + 255) / 256;
  if (nb > 152 * 16) nb = 152 * 16;
  if (p64) cmax_kernel<T, true><<<(unsigned)nb, 256, 0, s>>>(g, in, (T)gamma, ds);
  else cmax_kernel<T, false><<<(unsigned)nb, 256, 0, s>>>(g, in, (T)gamma, ds);
  return cudaGetLastError();
}

template <typename S, typename D>
static cudaError_t convert(const S* src, D* dst, long long n, cudaStream_t s) {
  long long nb = (n + 255) / 256;
  if (nb > 152 * 32) nb = 152 * 32;
  if (nb < 1) nb = 1;
  convert_kernel<S, D><<<(unsigned)nb, 256, 0, s>>>(n, src, dst);
  return cudaGetLastError();
}

#define MHD_INSTANTIATE_LAUNCH(T)                                                            \
  template <> cudaError_t Launch<T>::setup() {                                              \
    cudaError_t e = setup_p<T, false>();                                                    \
    if (sizeof(T) == 4) { cudaError_t e2 = setup_p<T, true>(); if (e2 != cudaSuccess) e = e2; } \
    cudaError_t e3 = set_ct_attr<T, 0>(); if (e3 != cudaSuccess) e = e3;                    \
    e3 = set_ct_attr<T, 1>(); if (e3 != cudaSuccess) e = e3;                                \
    e3 = set_ct_attr<T, 2>(); if (e3 != cudaSuccess) e = e3;                                \
    return e;                                                                               \
  }                                                                                         \
  template <> cudaError_t Launch<T>::fluid(const GridDesc& g, const FieldSet<T>& in,        \
      const FieldSet<T>& out, double gamma, double h, DevScalars* ds, int axis, bool last,  \
      bool p64, cudaStream_t s) {                                                           \
    return fluid_impl<T>(g, in, out, gamma, h, ds, axis, last, p64, s);                     \
  }                                                                                         \
  template <> cudaError_t Launch<T>::ct(const GridDesc& g, const FieldSet<T>& in,           \
      const FieldSet<T>& out, double h, DevScalars* ds, int axis, cudaStream_t s) {         \
    return ct_impl<T>(g, in, out, h, ds, axis, s);                                          \
  }                                                                                         \
  template <> cudaError_t Launch<T>::cmax(const GridDesc& g, const FieldSet<T>& in,         \
      double gamma, DevScalars* ds, bool p64, cudaStream_t s) {                             \
    return cmax_impl<T>(g, in, gamma, ds, p64, s);                                          \
  }                                                                                         \
  template <> cudaError_t Launch<T>::dt(DevScalars* ds, double cfl_h, cudaStream_t s) {     \
    dt_kernel<T><<<1, 1, 0, s>>>(ds, cfl_h);                                                \
    return cudaGetLastError();                                                              \
  }                                                                                         \
  template <> cudaError_t Launch<T>::sums(long long n, const FieldSet<T>& in,               \
      double* partial, int nblocks, double* out, cudaStream_t s) {                          \
    sums_partial_kernel<T><<<nblocks, 256, 0, s>>>(n, in, partial);                         \
    sums_final_kernel<<<1, 32, 0, s>>>(nblocks, partial, out);                              \
    return cudaGetLastError();                                                              \
  }                                                                                         \
  template <> cudaError_t Launch<T>::from(const void* src, int dtype, T* dst, long long n,  \
                                          cudaStream_t s) {                                 \
    if (dtype == 0) return convert<float, T>((const float*)src, dst, n, s);                 \
    return convert<double, T>((const double*)src, dst, n, s);                               \
  }                                                                                         \
  template <> cudaError_t Launch<T>::to(const T* src, void* dst, int dtype, long long n,    \
                                        cudaStream_t s) {                                   \
    if (dtype == 0) return convert<T, float>(src, (float*)dst, n, s);                       \
    return convert<T, double>(src, (double*)dst, n, s);                                     \
  }

}  // namespace mhd
