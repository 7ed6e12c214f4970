// Launcher bodies shared by the per-precision translation units.
#pragma once

#include <cstdlib>

#include "mhd_flat.cuh"
#include "mhd_kernels.cuh"
#include "mhd_launch.h"
#include "mhd_march.cuh"
#include "mhd_segz.cuh"
#include "mhd_tma.cuh"

namespace mhd {

// marching sweeps (x, y): S cells per tile along the sweep, NT pencils per block, shared
// prefetch ring of kMarchRing iterations x NV values per thread
template <typename T> struct MarchCfg { static constexpr int S = kMarchS, NT = 128; };
template <typename T>
static size_t march_smem(int nv) { return sizeof(T) * (size_t)kMarchRing * nv * MarchCfg<T>::NT; }
// warp segments (z): warps per block, cells per lane
constexpr int kSegWarps = 4;
#ifndef MHD_SEG_K_F32
#define MHD_SEG_K_F32 3
#endif
template <typename T> struct SegK { static constexpr int K = sizeof(T) == 4 ? MHD_SEG_K_F32 : 2; };

template <typename T, int A, bool LAST, int PM>
static cudaError_t set_march_attr() {
  cudaError_t e = cudaFuncSetAttribute(
      fluid_march_xy<T, A, LAST, PM, MarchCfg<T>::S, MarchCfg<T>::NT>,
      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)march_tile_smem<T>());
  if constexpr (sizeof(T) == 4) {
    cudaError_t e2 = cudaFuncSetAttribute(
        fluid_march_xy_vec<A, LAST, PM, MarchCfg<T>::S, MarchCfg<T>::NT>,
        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)march_tile_smem<T>());
    if (e2 != cudaSuccess) e = e2;
    e2 = cudaFuncSetAttribute(fluid_march_xy_vec<A, LAST, PM, MarchCfg<T>::S, MarchCfg<T>::NT, true>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)march_tile_smem<T>());
    if (e2 != cudaSuccess) e = e2;
    e2 = cudaFuncSetAttribute(fluid_march_xy_tma<A, LAST, PM, MarchCfg<T>::S>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tma_march_smem());
    if (e2 != cudaSuccess) e = e2;
  }
  return e;
}
template <typename T, int A>
static cudaError_t set_ct_march_attr() {
  return cudaFuncSetAttribute(ct_march_xy<T, A, MarchCfg<T>::S, MarchCfg<T>::NT>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)march_smem<T>(15));
}
// CT with shared EMF rows (ct_rows_xy): warps per block (used where ct_use_rows).  FP32
// launches with at least kRowsWideMin blocks of 16 rows per SM take 16 rows (one block of 512
// threads per SM, 15 updated rows each: 2% faster than 8 at 512^3), smaller ones 8 (16 rows
// left a 256^3 launch at about 2 waves and ran 14% slower); 4 rows were 16% slower at 512^3.
// FP64 always takes 8: its pipelines need 160 registers, which 512 threads cannot have.
#ifndef MHD_ROWS_R
#define MHD_ROWS_R 16
#endif
constexpr int kRowsWide = MHD_ROWS_R, kRowsNarrow = 8, kRowsWideMin = 8;
template <typename T, int A, int R>
static cudaError_t set_ct_rows_attr_r() {
  cudaError_t e = cudaFuncSetAttribute(ct_rows_xy<T, A, MarchCfg<T>::S, R>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)ct_rows_smem<T>(R));
  const cudaError_t e2 = cudaFuncSetAttribute(ct_rows_xy<T, A, MarchCfg<T>::S, R, 2>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)ct_rows_smem<T>(R, 2));
  return e != cudaSuccess ? e : e2;
}
template <typename T, int A>
static cudaError_t set_ct_rows_attr() {
  cudaError_t e = set_ct_rows_attr_r<T, A, kRowsNarrow>();
  if constexpr (sizeof(T) == 4 && kRowsWide != kRowsNarrow) {
    const cudaError_t e2 = set_ct_rows_attr_r<T, A, kRowsWide>();
    if (e2 != cudaSuccess) e = e2;
  }
  return e;
}
// the shared-row CT along axis (0 or 1) with R warps a block, PASSES operator applications
template <typename T, int R, int PASSES>
static cudaError_t launch_ct_rows_r(const GridDesc& g, const FieldSet<T>& in,
                                    const FieldSet<T>& out, double h, DevScalars* ds, int axis,
                                    cudaStream_t s) {
  constexpr int S = MarchCfg<T>::S;
  const int o = axis == 0 ? 1 : 0;
  const long long nb = (long long)((g.n[2] + 30) / 31) * ((g.n[o] + R - 2) / (R - 1));
  const dim3 grid((unsigned)nb, (unsigned)((g.n[axis] + S - 1) / S));
  const size_t sm = ct_rows_smem<T>(R, PASSES);
  if (axis == 0) ct_rows_xy<T, 0, S, R, PASSES><<<grid, 32 * R, sm, s>>>(g, in, out, h, ds);
  else ct_rows_xy<T, 1, S, R, PASSES><<<grid, 32 * R, sm, s>>>(g, in, out, h, ds);
  return cudaGetLastError();
}
template <typename T, int PASSES>
static cudaError_t launch_ct_rows(const GridDesc& g, const FieldSet<T>& in,
                                  const FieldSet<T>& out, double h, DevScalars* ds, int axis,
                                  cudaStream_t s) {
  if constexpr (sizeof(T) == 4 && kRowsWide != kRowsNarrow) {
    static int sms = 0;
    if (sms == 0) {
      int dev = 0;
      if (cudaGetDevice(&dev) != cudaSuccess ||
          cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        sms = 152;
    }
    const int o = axis == 0 ? 1 : 0;
    const long long wide = (long long)((g.n[2] + 30) / 31) *
                           ((g.n[o] + kRowsWide - 2) / (kRowsWide - 1)) *
                           ((g.n[axis] + MarchCfg<T>::S - 1) / MarchCfg<T>::S);
    if (wide >= (long long)kRowsWideMin * sms)
      return launch_ct_rows_r<T, kRowsWide, PASSES>(g, in, out, h, ds, axis, s);
  }
  return launch_ct_rows_r<T, kRowsNarrow, PASSES>(g, in, out, h, ds, axis, s);
}

template <typename T, int PM>
static cudaError_t setup_p() {
  cudaError_t e = cudaSuccess;
#define MHD_TRY(x) do { cudaError_t _e = (x); if (_e != cudaSuccess) e = _e; } while (0)
  MHD_TRY((set_march_attr<T, 0, false, PM>()));
  MHD_TRY((set_march_attr<T, 1, false, PM>()));
  MHD_TRY((set_march_attr<T, 0, true, PM>()));
  MHD_TRY((set_march_attr<T, 1, true, PM>()));
#undef MHD_TRY
  return e;
}


template <typename T, bool LAST, int PM>
static void fluid_dispatch(const GridDesc& g, const FieldSet<T>& in, const FieldSet<T>& out,
                           T gamma, double h, DevScalars* ds, int axis, cudaStream_t s,
                           const void* tmaps) {
  constexpr int S = MarchCfg<T>::S, NT = MarchCfg<T>::NT;
  if (axis == 0 || axis == 1) {
    const int o = axis == 0 ? 1 : 0;
    const long long np = (long long)g.n[2] * g.n[o];
    const dim3 grid((unsigned)((np + NT - 1) / NT), (unsigned)((g.n[axis] + S - 1) / S));
    const size_t sm = march_tile_smem<T>();
    if constexpr (sizeof(T) == 4) {
      if (MHD_TMA_MARCH && tmaps && g.n[2] % 128 == 0) {
        const TmaMaps* m = static_cast<const TmaMaps*>(tmaps);
        const int A = axis, T1 = (A + 1) % 3, T2 = (A + 2) % 3;
        TmaRows rows;
        const int f[9] = {0, 1 + A, 1 + T1, 1 + T2, 4, 5 + A, 5 + T1, 5 + T2, 5 + o};
        for (int r = 0; r < 9; ++r) {
          rows.g[r] = A == 0 ? m->gx[f[r]] : m->gy[f[r]];
          rows.one[r] = m->one[f[r]];
        }
        const size_t tsm = tma_march_smem();
        if (axis == 0)
          fluid_march_xy_tma<0, LAST, PM, S><<<grid, 128, tsm, s>>>(g, in, out, gamma, h, ds, rows);
        else
          fluid_march_xy_tma<1, LAST, PM, S><<<grid, 128, tsm, s>>>(g, in, out, gamma, h, ds, rows);
        return;
      }
      if (march_vec<T>(g)) {
        const bool o32 = MHD_OFF32_XY && field_off32<T>(g);
        if (axis == 0 && o32)
          fluid_march_xy_vec<0, LAST, PM, S, NT, true><<<grid, NT, sm, s>>>(g, in, out, gamma, h, ds);
        else if (axis == 0)
          fluid_march_xy_vec<0, LAST, PM, S, NT><<<grid, NT, sm, s>>>(g, in, out, gamma, h, ds);
        else if (o32)
          fluid_march_xy_vec<1, LAST, PM, S, NT, true><<<grid, NT, sm, s>>>(g, in, out, gamma, h, ds);
        else
          fluid_march_xy_vec<1, LAST, PM, S, NT><<<grid, NT, sm, s>>>(g, in, out, gamma, h, ds);
        return;
      }
    }
    if (axis == 0) fluid_march_xy<T, 0, LAST, PM, S, NT><<<grid, NT, sm, s>>>(g, in, out, gamma, h, ds);
    else fluid_march_xy<T, 1, LAST, PM, S, NT><<<grid, NT, sm, s>>>(g, in, out, gamma, h, ds);
    return;
  }
  if (sizeof(T) == 4 && seg_k_for(g.n[2]) == 2) {
    constexpr int K = 2, SEG = 32 * K - 6;
    const long long warps = (long long)g.n[0] * g.n[1] * ((g.n[2] + SEG - 1) / SEG);
    const unsigned nb = (unsigned)((warps + kSegWarps - 1) / kSegWarps);
    if (field_off32<T>(g))
      fluid_seg_z<T, LAST, PM, kSegWarps, K, true><<<nb, 32 * kSegWarps, 0, s>>>(g, in, out, gamma, h, ds);
    else
      fluid_seg_z<T, LAST, PM, kSegWarps, K><<<nb, 32 * kSegWarps, 0, s>>>(g, in, out, gamma, h, ds);
    return;
  }
  constexpr int K = SegK<T>::K, SEG = 32 * K - 6;
  const long long warps = (long long)g.n[0] * g.n[1] * ((g.n[2] + SEG - 1) / SEG);
  const unsigned nb = (unsigned)((warps + kSegWarps - 1) / kSegWarps);
  if (field_off32<T>(g))
    fluid_seg_z<T, LAST, PM, kSegWarps, K, true><<<nb, 32 * kSegWarps, 0, s>>>(g, in, out, gamma, h, ds);
  else
    fluid_seg_z<T, LAST, PM, kSegWarps, K><<<nb, 32 * kSegWarps, 0, s>>>(g, in, out, gamma, h, ds);
}

template <typename T>
static cudaError_t cmax_impl(const GridDesc& g, const FieldSet<T>& in, double gamma,
                             DevScalars* ds, int pm, cudaStream_t s);

template <typename T>
static cudaError_t fluid_impl(const GridDesc& g, const FieldSet<T>& in, const FieldSet<T>& out,
                              double gamma, double h, DevScalars* ds, int axis, bool last,
                              int pm, cudaStream_t s, const void* tmaps) {
  if (axis_is_flat(g, axis))   // identity (mhd_flat.cuh); the caller does not swap buffers
    return last ? cmax_impl<T>(g, in, gamma, ds, pm, s) : cudaSuccess;
  const T gm = (T)gamma;
  if constexpr (sizeof(T) == 4) {
    if (pm == PM_FP64) {
      if (last) fluid_dispatch<T, true, PM_FP64>(g, in, out, gm, h, ds, axis, s, tmaps);
      else fluid_dispatch<T, false, PM_FP64>(g, in, out, gm, h, ds, axis, s, tmaps);
      return cudaGetLastError();
    }
    if (pm == PM_COMP) {
      if (last) fluid_dispatch<T, true, PM_COMP>(g, in, out, gm, h, ds, axis, s, tmaps);
      else fluid_dispatch<T, false, PM_COMP>(g, in, out, gm, h, ds, axis, s, tmaps);
      return cudaGetLastError();
    }
  }
  if (last) fluid_dispatch<T, true, PM_FP32>(g, in, out, gm, h, ds, axis, s, tmaps);
  else fluid_dispatch<T, false, PM_FP32>(g, in, out, gm, h, ds, axis, s, tmaps);
  return cudaGetLastError();
}

// FP32 constrained transport along z by the marching shared-row kernel (ct_rows_z), one or
// two passes; false where its grid does not fit, or where the environment variable
// MHD_CTZ_SEG is "1" (read at each launch: the tests compare both forms bit for bit), and
// the caller then takes ct_seg_z
template <int PASSES>
static bool ct_rows_z_launch(const GridDesc& g, const FieldSet<float>& in,
                             const FieldSet<float>& out, double h, DevScalars* ds,
                             cudaStream_t s) {
  if (!MHD_CTZ_ROWS) return false;
  const char* seg = std::getenv("MHD_CTZ_SEG");
  if (seg && seg[0] == '1') return false;
  constexpr int Q = MHD_CTZ_Q, L = MHD_CTZ_L;
  const bool o32 = field_off32<float>(g), clamp = PASSES == 2 && g.bc[2] == 1;
  dim3 grid;
  if (seg_k_for(g.n[2]) == 2) {
    constexpr int K = 2;
    if (!ct_rows_z_grid<K, PASSES>(g, Q, L, &grid)) return false;
    if (clamp && o32) ct_rows_z<K, Q, PASSES, true, true><<<grid, 32 * Q, 0, s>>>(g, in, out, h, ds, L);
    else if (clamp) ct_rows_z<K, Q, PASSES, true, false><<<grid, 32 * Q, 0, s>>>(g, in, out, h, ds, L);
    else if (o32) ct_rows_z<K, Q, PASSES, false, true><<<grid, 32 * Q, 0, s>>>(g, in, out, h, ds, L);
    else ct_rows_z<K, Q, PASSES, false, false><<<grid, 32 * Q, 0, s>>>(g, in, out, h, ds, L);
    return true;
  }
  constexpr int K = 3;
  if (!ct_rows_z_grid<K, PASSES>(g, Q, L, &grid)) return false;
  if (clamp && o32) ct_rows_z<K, Q, PASSES, true, true><<<grid, 32 * Q, 0, s>>>(g, in, out, h, ds, L);
  else if (clamp) ct_rows_z<K, Q, PASSES, true, false><<<grid, 32 * Q, 0, s>>>(g, in, out, h, ds, L);
  else if (o32) ct_rows_z<K, Q, PASSES, false, true><<<grid, 32 * Q, 0, s>>>(g, in, out, h, ds, L);
  else ct_rows_z<K, Q, PASSES, false, false><<<grid, 32 * Q, 0, s>>>(g, in, out, h, ds, L);
  return true;
}

template <typename T>
static cudaError_t ct_impl(const GridDesc& g, const FieldSet<T>& in, const FieldSet<T>& out,
                           double h, DevScalars* ds, int axis, cudaStream_t s) {
  constexpr int S = MarchCfg<T>::S, NT = MarchCfg<T>::NT;
  if (axis_is_flat(g, axis)) {   // B_A only (mhd_flat.cuh); the caller swaps B_A alone
    const long long N = (long long)g.n[0] * g.n[1] * g.n[2];
    long long nb = (N + 255) / 256;
    if (nb > 152 * 16) nb = 152 * 16;
    if (axis == 0) ct_flat_kernel<T, 0><<<(unsigned)nb, 256, 0, s>>>(g, in, out, h, ds);
    else if (axis == 1) ct_flat_kernel<T, 1><<<(unsigned)nb, 256, 0, s>>>(g, in, out, h, ds);
    else ct_flat_kernel<T, 2><<<(unsigned)nb, 256, 0, s>>>(g, in, out, h, ds);
    return cudaGetLastError();
  }
  if (ct_use_rows(g, axis)) return launch_ct_rows<T, 1>(g, in, out, h, ds, axis, s);
  if (axis == 0 || axis == 1) {
    const int o = axis == 0 ? 1 : 0;
    const long long np = (long long)g.n[2] * g.n[o];
    const dim3 grid((unsigned)((np + NT - 1) / NT), (unsigned)((g.n[axis] + S - 1) / S));
    const size_t sm = march_smem<T>(15);
    if (axis == 0) ct_march_xy<T, 0, S, NT><<<grid, NT, sm, s>>>(g, in, out, h, ds);
    else ct_march_xy<T, 1, S, NT><<<grid, NT, sm, s>>>(g, in, out, h, ds);
    return cudaGetLastError();
  }
  if constexpr (sizeof(T) == 4)
    if (ct_rows_z_launch<1>(g, in, out, h, ds, s)) return cudaGetLastError();
  if (sizeof(T) == 4 && seg_k_for(g.n[2]) == 2) {
    constexpr int K = 2, SEG = 32 * K - 8;
    const long long warps = (long long)g.n[0] * g.n[1] * ((g.n[2] + SEG - 1) / SEG);
    const unsigned nb = (unsigned)((warps + kSegWarps - 1) / kSegWarps);
    if (field_off32<T>(g))
      ct_seg_z<T, kSegWarps, K, 1, false, true><<<nb, 32 * kSegWarps, 0, s>>>(g, in, out, h, ds);
    else
      ct_seg_z<T, kSegWarps, K><<<nb, 32 * kSegWarps, 0, s>>>(g, in, out, h, ds);
    return cudaGetLastError();
  }
  {
    constexpr int K = SegK<T>::K, SEG = 32 * K - 8;
    const long long warps = (long long)g.n[0] * g.n[1] * ((g.n[2] + SEG - 1) / SEG);
    const unsigned nb = (unsigned)((warps + kSegWarps - 1) / kSegWarps);
    if (field_off32<T>(g))
      ct_seg_z<T, kSegWarps, K, 1, false, true><<<nb, 32 * kSegWarps, 0, s>>>(g, in, out, h, ds);
    else
      ct_seg_z<T, kSegWarps, K><<<nb, 32 * kSegWarps, 0, s>>>(g, in, out, h, ds);
    return cudaGetLastError();
  }
}

// the two-pass z segments: outflow z re-clamps its ghost cells between the passes
template <typename T, int K>
static cudaError_t ct2_seg_z_launch(const GridDesc& g, const FieldSet<T>& in,
                                    const FieldSet<T>& out, double h, DevScalars* ds,
                                    unsigned nb, bool clamp, cudaStream_t s) {
  const bool o32 = field_off32<T>(g);
  if (clamp && o32) ct_seg_z<T, kSegWarps, K, 2, true, true><<<nb, 32 * kSegWarps, 0, s>>>(g, in, out, h, ds);
  else if (clamp) ct_seg_z<T, kSegWarps, K, 2, true><<<nb, 32 * kSegWarps, 0, s>>>(g, in, out, h, ds);
  else if (o32) ct_seg_z<T, kSegWarps, K, 2, false, true><<<nb, 32 * kSegWarps, 0, s>>>(g, in, out, h, ds);
  else ct_seg_z<T, kSegWarps, K, 2, false><<<nb, 32 * kSegWarps, 0, s>>>(g, in, out, h, ds);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t ct2_impl(const GridDesc& g, const FieldSet<T>& in, const FieldSet<T>& out,
                            double h, DevScalars* ds, int axis, cudaStream_t s) {
  if (axis_is_flat(g, axis)) return cudaErrorNotSupported;
  if (axis < 2) {
    if (!ct_use_rows(g, axis) || g.bc[axis] != 0) return cudaErrorNotSupported;
    return launch_ct_rows<T, 2>(g, in, out, h, ds, axis, s);
  }
  if constexpr (sizeof(T) == 4)
    if (ct_rows_z_launch<2>(g, in, out, h, ds, s)) return cudaGetLastError();
  const bool clamp = g.bc[2] == 1;
  if (sizeof(T) == 4 && seg_k_for(g.n[2]) == 2) {
    constexpr int K = 2, SEG = 32 * K - 16;
    const long long warps = (long long)g.n[0] * g.n[1] * ((g.n[2] + SEG - 1) / SEG);
    const unsigned nb = (unsigned)((warps + kSegWarps - 1) / kSegWarps);
    return ct2_seg_z_launch<T, K>(g, in, out, h, ds, nb, clamp, s);
  }
  constexpr int K = SegK<T>::K, SEG = 32 * K - 16;
  const long long warps = (long long)g.n[0] * g.n[1] * ((g.n[2] + SEG - 1) / SEG);
  const unsigned nb = (unsigned)((warps + kSegWarps - 1) / kSegWarps);
  return ct2_seg_z_launch<T, K>(g, in, out, h, ds, nb, clamp, s);
}

template <typename T>
static cudaError_t ct_fluid_impl(const GridDesc& g, const FieldSet<T>& in,
                                 const FieldSet<T>& out, double gamma, double h,
                                 DevScalars* ds, int axis, int pm, cudaStream_t s) {
  if constexpr (sizeof(T) != 4) {
    return cudaErrorNotSupported;
  } else {
    if (axis != 2 || axis_is_flat(g, 2) || pm != PM_FP32) return cudaErrorNotSupported;
    constexpr int Q = MHD_LOPZ_Q, L = MHD_CTZ_L;
    const bool o32 = field_off32<float>(g), clamp = g.bc[2] == 1;
    const float gm = (float)gamma;
    dim3 grid;
    if (seg_k_for(g.n[2]) == 2) {
      constexpr int K = 2;
      if (!ct_fluid_rows_z_grid<K>(g, Q, L, &grid)) return cudaErrorNotSupported;
      if (clamp && o32) ct_fluid_rows_z<K, Q, PM_FP32, true, true><<<grid, 32 * Q, 0, s>>>(g, in, out, gm, h, ds, L);
      else if (clamp) ct_fluid_rows_z<K, Q, PM_FP32, true, false><<<grid, 32 * Q, 0, s>>>(g, in, out, gm, h, ds, L);
      else if (o32) ct_fluid_rows_z<K, Q, PM_FP32, false, true><<<grid, 32 * Q, 0, s>>>(g, in, out, gm, h, ds, L);
      else ct_fluid_rows_z<K, Q, PM_FP32, false, false><<<grid, 32 * Q, 0, s>>>(g, in, out, gm, h, ds, L);
      return cudaGetLastError();
    }
    constexpr int K = 3;
    if (!ct_fluid_rows_z_grid<K>(g, Q, L, &grid)) return cudaErrorNotSupported;
    if (clamp && o32) ct_fluid_rows_z<K, Q, PM_FP32, true, true><<<grid, 32 * Q, 0, s>>>(g, in, out, gm, h, ds, L);
    else if (clamp) ct_fluid_rows_z<K, Q, PM_FP32, true, false><<<grid, 32 * Q, 0, s>>>(g, in, out, gm, h, ds, L);
    else if (o32) ct_fluid_rows_z<K, Q, PM_FP32, false, true><<<grid, 32 * Q, 0, s>>>(g, in, out, gm, h, ds, L);
    else ct_fluid_rows_z<K, Q, PM_FP32, false, false><<<grid, 32 * Q, 0, s>>>(g, in, out, gm, h, ds, L);
    return cudaGetLastError();
  }
}

template <typename T>
static cudaError_t cmax_impl(const GridDesc& g, const FieldSet<T>& in, double gamma,
                             DevScalars* ds, int pm, cudaStream_t s) {
  const long long N = (long long)g.n[0] * g.n[1] * g.n[2];
  long long nb = (N + 255) / 256;
  if (nb > 152 * 16) nb = 152 * 16;
  if (sizeof(T) == 4 && pm == PM_FP64)
    cmax_kernel<T, PM_FP64><<<(unsigned)nb, 256, 0, s>>>(g, in, (T)gamma, ds);
  else if (sizeof(T) == 4 && pm == PM_COMP)
    cmax_kernel<T, PM_COMP><<<(unsigned)nb, 256, 0, s>>>(g, in, (T)gamma, ds);
  else
    cmax_kernel<T, PM_FP32><<<(unsigned)nb, 256, 0, s>>>(g, in, (T)gamma, ds);
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
    cudaError_t e = setup_p<T, PM_FP32>();                                                  \
    if (sizeof(T) == 4) {                                                                   \
      cudaError_t e2 = setup_p<T, PM_FP64>(); if (e2 != cudaSuccess) e = e2;                \
      e2 = setup_p<T, PM_COMP>(); if (e2 != cudaSuccess) e = e2;                            \
    }                                                                                       \
    cudaError_t e3 = set_ct_march_attr<T, 0>(); if (e3 != cudaSuccess) e = e3;              \
    e3 = set_ct_march_attr<T, 1>(); if (e3 != cudaSuccess) e = e3;                          \
    e3 = set_ct_rows_attr<T, 0>(); if (e3 != cudaSuccess) e = e3;                           \
    e3 = set_ct_rows_attr<T, 1>(); if (e3 != cudaSuccess) e = e3;                           \
    return e;                                                                               \
  }                                                                                         \
  template <> cudaError_t Launch<T>::fluid(const GridDesc& g, const FieldSet<T>& in,        \
      const FieldSet<T>& out, double gamma, double h, DevScalars* ds, int axis, bool last,  \
      int pm, cudaStream_t s, const void* tmaps) {                                          \
    return fluid_impl<T>(g, in, out, gamma, h, ds, axis, last, pm, s, tmaps);              \
  }                                                                                         \
  template <> cudaError_t Launch<T>::ct(const GridDesc& g, const FieldSet<T>& in,           \
      const FieldSet<T>& out, double h, DevScalars* ds, int axis, cudaStream_t s) {         \
    return ct_impl<T>(g, in, out, h, ds, axis, s);                                          \
  }                                                                                         \
  template <> cudaError_t Launch<T>::ct2(const GridDesc& g, const FieldSet<T>& in,          \
      const FieldSet<T>& out, double h, DevScalars* ds, int axis, cudaStream_t s) {         \
    return ct2_impl<T>(g, in, out, h, ds, axis, s);                                         \
  }                                                                                         \
  template <> cudaError_t Launch<T>::ct_fluid(const GridDesc& g, const FieldSet<T>& in,     \
      const FieldSet<T>& out, double gamma, double h, DevScalars* ds, int axis, int pm,     \
      cudaStream_t s) {                                                                     \
    return ct_fluid_impl<T>(g, in, out, gamma, h, ds, axis, pm, s);                         \
  }                                                                                         \
  template <> cudaError_t Launch<T>::cmax(const GridDesc& g, const FieldSet<T>& in,         \
      double gamma, DevScalars* ds, int pm, cudaStream_t s) {                             \
    return cmax_impl<T>(g, in, gamma, ds, pm, s);                                          \
  }                                                                                         \
  template <> cudaError_t Launch<T>::dt(DevScalars* ds, double cfl_h, double h,           \
                                        cudaStream_t s) {                                   \
    dt_kernel<T><<<1, 1, 0, s>>>(ds, cfl_h, h);                                             \
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
