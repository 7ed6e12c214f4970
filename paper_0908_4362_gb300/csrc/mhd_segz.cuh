// z sweeps as warp-cooperative segments.  The z pencil is the contiguous axis, so the 32
// lanes of a warp hold 32 K consecutive cells of one pencil (lane l: cells lK .. lK+K-1):
// loads coalesce along z, neighbours inside a lane are registers, and the one neighbour
// per shift that lives in the next or previous lane comes from a warp shuffle.  Each warp
// updates the cells whose full stencil lies inside its window: 32K - 6 for the fluid sweep
// (halo 3 per side), 32K - 8 for the constrained transport (halo 4).
// Per-cell arithmetic and its order are the oracle's (Algorithms 1 and 2).
#pragma once

#include <type_traits>

#include "mhd_kernels.cuh"
#include "mhd_march.cuh"

namespace mhd {

// Cells per lane of the FP32 z segments, chosen per grid: a window of 32K cells updates
// 32K - 6 (fluid) or 32K - 8 (CT) of them, so short pencils waste part of a K = 3 window.
// Work per pencil ~ windows x 32K x (cost per window cell), with the measured relative
// costs 1.0 (K = 3) and 1.12 (K = 2); the cheaper choice is taken (the CT uses the fluid's
// choice).  FP64 keeps K = 2.
#ifndef MHD_SEG_K_AUTO
#define MHD_SEG_K_AUTO 1
#endif
__host__ __device__ inline int seg_k_for(int nz) {
  if (!MHD_SEG_K_AUTO) return 3;
  const long long w3 = (nz + 89) / 90, w2 = (nz + 57) / 58;
  return w2 * 64 * 112 < w3 * 96 * 100 ? 2 : 3;
}

// Which window a warp takes: segment s of pencil (x, y), the segments of a pencil on
// consecutive warps (ordering consecutive warps along y at a fixed segment, so that a
// block's warps share their y-neighbour rows in L1, measured 2.6% slower for the fluid).
// Warps past the end are inactive and take the last window for their arithmetic.
struct SegPlace {
  int s0, x, y;
  bool active;
};
template <bool DIV32 = false>
__device__ __forceinline__ SegPlace seg_place(const GridDesc& g, int nz, int seg, long long wid) {
  const int nseg = (nz + seg - 1) / seg;
  const long long total = (long long)g.n[0] * g.n[1] * nseg;
  SegPlace p;
  p.active = wid < total;
  const long long w = p.active ? wid : total - 1;
  if (DIV32 && total <= 0xFFFFFFFFll) {
    // 32-bit unsigned divisions: every lane computes its warp's window, and a 64-bit
    // division per lane and window was a measurable share of the fluid segments (-1.3%;
    // the CT segments, at a 56-register cap, were 6.7% slower this way and keep 64 bits)
    const unsigned w32 = (unsigned)w, ns = (unsigned)nseg, n1 = (unsigned)g.n[1];
    const unsigned pencil = w32 / ns;
    p.s0 = (int)(w32 - pencil * ns) * seg;
    p.x = (int)(pencil / n1);
    p.y = (int)(pencil - (unsigned)p.x * n1);
  } else {
    const long long pencil = w / nseg;
    p.s0 = (int)(w % nseg) * seg;
    p.x = (int)(pencil / g.n[1]);
    p.y = (int)(pencil % g.n[1]);
  }
  return p;
}

// global loads: the read-only path in standalone kernels (NC), plain coherent loads where
// the same launch writes the data earlier (the persistent batched kernel)
template <bool NC, typename T>
__device__ __forceinline__ T ldx(const T* p) {
  if constexpr (NC) return __ldg(p);
  else return *p;
}

template <typename T>
__device__ __forceinline__ T shdown(T v) { return __shfl_down_sync(0xffffffffu, v, 1); }
template <typename T>
__device__ __forceinline__ T shup(T v) { return __shfl_up_sync(0xffffffffu, v, 1); }

// value of the next cell (to the right along z) for each of the lane's K cells
template <typename T, int K>
__device__ __forceinline__ void next_cell(const T (&x)[K], T (&xn)[K]) {
  const T from_next_lane = shdown(x[0]);
#pragma unroll
  for (int i = 0; i < K; ++i) xn[i] = (i + 1 < K) ? x[i + 1] : from_next_lane;
}
// value of the previous cell for each of the lane's K cells
template <typename T, int K>
__device__ __forceinline__ void prev_cell(const T (&x)[K], T (&xp)[K]) {
  const T from_prev_lane = shup(x[K - 1]);
#pragma unroll
  for (int i = 0; i < K; ++i) xp[i] = (i > 0) ? x[i - 1] : from_prev_lane;
}

// next/previous cell of packed pairs: two shuffles per shift
template <int K>
__device__ __forceinline__ void next_cell2(const float2 (&x)[K], float2 (&xn)[K]) {
  const float2 from_next_lane = make_float2(shdown(x[0].x), shdown(x[0].y));
#pragma unroll
  for (int i = 0; i < K; ++i) xn[i] = (i + 1 < K) ? x[i + 1] : from_next_lane;
}
template <int K>
__device__ __forceinline__ void prev_cell2(const float2 (&x)[K], float2 (&xp)[K]) {
  const float2 from_prev_lane = make_float2(shup(x[K - 1].x), shup(x[K - 1].y));
#pragma unroll
  for (int i = 0; i < K; ++i) xp[i] = (i > 0) ? x[i - 1] : from_prev_lane;
}
// Component loops of the fluid segments (packing component pairs into f32x2 was measured
// slower here: 1.91 -> 2.02 ms at 512^3, the pair moves and the lower occupancy cost more
// than the halved arithmetic).
template <typename T> struct Vec {
  static __device__ __forceinline__ T sub(T a, T b) { return a - b; }
  static __device__ __forceinline__ T add(T a, T b) { return a + b; }
  static __device__ __forceinline__ T fnma(T s, T a, T b) { return ffms(s, a, b); }   // b - s a
  static __device__ __forceinline__ T add_hv(T base, T a, T b) { return plus_half_vanleer(base, a, b); }
  static __device__ __forceinline__ T sub_hv(T base, T a, T b) { return minus_half_vanleer(base, a, b); }
  static __device__ __forceinline__ T splat(T v) { return v; }
  template <int K>
  static __device__ __forceinline__ void next(const T (&x)[K], T (&xn)[K]) { next_cell<T, K>(x, xn); }
  template <int K>
  static __device__ __forceinline__ void prev(const T (&x)[K], T (&xp)[K]) { prev_cell<T, K>(x, xp); }
};
// stage 1 of one component: first-order fluxes and the half step
template <typename V, int K>
__device__ __forceinline__ void seg_stage1(const V (&fr)[K], const V (&fl)[K], const V (&u)[K],
                                           V hd, V (&uh)[K]) {
  V fln[K], g1[K], g1p[K];
  Vec<V>::template next<K>(fl, fln);
#pragma unroll
  for (int i = 0; i < K; ++i) g1[i] = Vec<V>::sub(fr[i], fln[i]);   // first-order flux at +1/2
  Vec<V>::template prev<K>(g1, g1p);
#pragma unroll
  for (int i = 0; i < K; ++i) uh[i] = Vec<V>::fnma(hd, Vec<V>::sub(g1[i], g1p[i]), u[i]);
}

// stage 2 of one component: limited fluxes and the full update
template <typename V, int K>
__device__ __forceinline__ void seg_stage2(const V (&fr2)[K], const V (&fl2)[K], const V (&u)[K],
                                           V dth, V (&un)[K]) {
  V frn[K], dR[K], dRp[K], fln[K], dL[K], dLn[K], g2[K], g2p[K];
  Vec<V>::template next<K>(fr2, frn);
#pragma unroll
  for (int i = 0; i < K; ++i) dR[i] = Vec<V>::sub(frn[i], fr2[i]);   // FR2(w+1) - FR2(w)
  Vec<V>::template prev<K>(dR, dRp);
  Vec<V>::template next<K>(fl2, fln);
#pragma unroll
  for (int i = 0; i < K; ++i) dL[i] = Vec<V>::sub(fln[i], fl2[i]);   // FL2(w+1) - FL2(w)
  Vec<V>::template next<K>(dL, dLn);
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const V right = Vec<V>::add_hv(fr2[i], dRp[i], dR[i]);
    const V left = Vec<V>::sub_hv(fln[i], dL[i], dLn[i]);
    g2[i] = Vec<V>::sub(right, left);                                // limited flux at +1/2
  }
  Vec<V>::template prev<K>(g2, g2p);
#pragma unroll
  for (int i = 0; i < K; ++i) un[i] = Vec<V>::fnma(dth, Vec<V>::sub(g2[i], g2p[i]), u[i]);
}

// The two stages of the fluid sweep over a warp's window (Algorithm 1): u[K][5] the
// conserved fluid variables of the lane's cells in local order (rho, m_n, m_t1, m_t2, E),
// b[K][3] the cell-centred B (n, t1, t2); un the updated variables, valid on window cells
// 3 .. 32K-4 when u and b are valid on the whole window.  Returns the status bits of the
// flux evaluations at the window cells [v0, v1] (stage 1) and [v0 + 1, v1 - 1] (stage 2),
// the cells whose operands are real (v0 = 0, v1 = 32K - 1 where u and b are valid
// everywhere).
template <typename T, int PM, int K>
__device__ __forceinline__ int fluid_seg_core(const T (&u)[K][5], const T (&b)[K][3], T gamma,
                                              T dth, T hd, int lane, int v0, int v1,
                                              T (&un)[K][5]) {
  int st = 0;
  // stage 1: first-order fluxes, half step
  T uh[K][5];
  {
    T fr[5][K], fl[5][K];
#pragma unroll
    for (int i = 0; i < K; ++i) {
      T a[5], c[5];
      const int s1 = cell_flux<T, PM>(u[i], b[i], gamma, a, c);
      const int w1 = lane * K + i;
      if (w1 >= v0 && w1 <= v1) st |= s1;
#pragma unroll
      for (int q = 0; q < 5; ++q) { fr[q][i] = a[q]; fl[q][i] = c[q]; }
    }
    T uq[5][K], uhq[5][K];
#pragma unroll
    for (int q = 0; q < 5; ++q)
#pragma unroll
      for (int i = 0; i < K; ++i) uq[q][i] = u[i][q];
#pragma unroll
    for (int q = 0; q < 5; ++q) seg_stage1<T, K>(fr[q], fl[q], uq[q], hd, uhq[q]);
#pragma unroll
    for (int q = 0; q < 5; ++q)
#pragma unroll
      for (int i = 0; i < K; ++i) uh[i][q] = uhq[q][i];
  }
  // stage 2: limited fluxes of u^{t+dt/2}, full update
  {
    T fr2[5][K], fl2[5][K];
#pragma unroll
    for (int i = 0; i < K; ++i) {
      T a[5], c[5];
      const int s2 = cell_flux<T, PM>(uh[i], b[i], gamma, a, c);
      const int w = lane * K + i;
      if (w >= v0 + 1 && w <= v1 - 1) st |= s2;
#pragma unroll
      for (int q = 0; q < 5; ++q) { fr2[q][i] = a[q]; fl2[q][i] = c[q]; }
    }
    T uq[5][K], unq[5][K];
#pragma unroll
    for (int q = 0; q < 5; ++q)
#pragma unroll
      for (int i = 0; i < K; ++i) uq[q][i] = u[i][q];
#pragma unroll
    for (int q = 0; q < 5; ++q) seg_stage2<T, K>(fr2[q], fl2[q], uq[q], dth, unq[q]);
#pragma unroll
    for (int q = 0; q < 5; ++q)
#pragma unroll
      for (int i = 0; i < K; ++i) un[i][q] = unq[q][i];
  }
  return st;
}

// one warp: window `wid` (seg_place); all 32 lanes call it
template <typename T, bool LAST, int PM, int K, bool NC, bool OFF32 = false>
__device__ __forceinline__ void fluid_seg_z_warp(const GridDesc& g, const FieldSet<T>& in,
                                                 const FieldSet<T>& out, T gamma, double h,
                                                 DevScalars* ds, long long wid) {
  using AD = FieldAddr<T, OFF32>;
  constexpr int H = 3, SEG = 32 * K - 2 * H;
  const int lane = threadIdx.x & 31;
  const int nz = g.n[2], bcz = g.bc[2];
  const SegPlace sp = seg_place<true>(g, nz, SEG, wid);
  const int s0 = sp.s0, x = sp.x, y = sp.y;
  const bool warp_active = sp.active;
  const T dth = step_factor<T>(ds, h) * T(FluxScale<T>::inv);   // for cell_flux's flux scale
  const T hd = T(0.5) * dth;
  const typename AD::I row = AD::of((long long)x * g.s[0] + (long long)y * g.s[1]);
  const typename AD::I r1 =
      row + AD::of((long long)(wrap_index(x + 1, g.n[0], g.bc[0]) - x) * g.s[0]);
  const typename AD::I r2 =
      row + AD::of((long long)(wrap_index(y + 1, g.n[1], g.bc[1]) - y) * g.s[1]);
  const int z0 = s0 - H + lane * K;     // the lane's first cell
  // local coordinates of a z sweep: n = z, t1 = x, t2 = y
  T u[K][5], b[K][3];
  int st = 0;
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const typename AD::I zc = AD::of(wrap_index(z0 + i, nz, bcz));
    const typename AD::I zn = AD::of(wrap_index(z0 + i + 1, nz, bcz));
    const typename AD::I c = row + zc;
    u[i][0] = ldx<NC>(AD::at(in.f[0], c));
    u[i][1] = ldx<NC>(AD::at(in.f[3], c));
    u[i][2] = ldx<NC>(AD::at(in.f[1], c));
    u[i][3] = ldx<NC>(AD::at(in.f[2], c));
    u[i][4] = ldx<NC>(AD::at(in.f[4], c));
    b[i][0] = T(0.5) * (ldx<NC>(AD::at(in.f[7], c)) + ldx<NC>(AD::at(in.f[7], row + zn)));
    b[i][1] = T(0.5) * (ldx<NC>(AD::at(in.f[5], c)) + ldx<NC>(AD::at(in.f[5], r1 + zc)));
    b[i][2] = T(0.5) * (ldx<NC>(AD::at(in.f[6], c)) + ldx<NC>(AD::at(in.f[6], r2 + zc)));
  }
  T un[K][5];
  st |= fluid_seg_core<T, PM, K>(u, b, gamma, dth, hd, lane, 0, 32 * K - 1, un);
  T cm = T(0);
  bool nan_seen = false;
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const int w = lane * K + i, z = z0 + i;
    if (warp_active && w >= H && w < H + SEG && z < nz) {
      const typename AD::I co = row + AD::of(z);
      *AD::at(out.f[0], co) = un[i][0];
      *AD::at(out.f[3], co) = un[i][1];
      *AD::at(out.f[1], co) = un[i][2];
      *AD::at(out.f[2], co) = un[i][3];
      *AD::at(out.f[4], co) = un[i][4];
      if (!(un[i][0] > T(0))) st |= ST_UNPHYSICAL;
      if (LAST) {
        const T v = cell_cmax<T, PM>(un[i][0], un[i][1], un[i][2], un[i][3], un[i][4], b[i][0],
                                      b[i][1], b[i][2], gamma, &st);
        if (v != v) nan_seen = true; else cm = fmax(cm, v);
      }
    }
  }
  if (LAST) block_max_to_global(cm, nan_seen, ds);
  if (warp_active && st) atomicOr(&ds->status, st);
}

// Minimum resident blocks per SM asked of the compiler for the FP32 z segments (register
// caps: 64 registers for the fluid, 56 for the CT; 0 leaves the bound unset).  Measured at
// 512^3: fluid z 1.91 -> 1.81 ms, CT z 1.43 -> 1.37 ms against the uncapped 72 and 64
// registers; tighter caps spill more than the extra resident warps recover.
#ifndef MHD_SEG_MINB
#define MHD_SEG_MINB 8
#endif
#ifndef MHD_CTSEG_MINB
#define MHD_CTSEG_MINB 9
#endif
template <typename T> struct SegMinBlocks {
  static constexpr int fluid = sizeof(T) == 4 ? MHD_SEG_MINB : 0;
  static constexpr int ct = sizeof(T) == 4 ? MHD_CTSEG_MINB : 0;
};
template <typename T, bool LAST, int PM, int NW, int K, bool OFF32 = false>
__global__ void __launch_bounds__(32 * NW, SegMinBlocks<T>::fluid)
fluid_seg_z(GridDesc g, FieldSet<T> in, FieldSet<T> out, T gamma, double h, DevScalars* ds) {
  fluid_seg_z_warp<T, LAST, PM, K, true, OFF32>(g, in, out, gamma, h, ds,
                                                 (long long)blockIdx.x * NW + (threadIdx.x >> 5));
}

// one EMF pipeline over the window: bt[] becomes the advected B_t (valid on window cells
// 4 .. 32K-5) and e2m[] the limited EMF at each cell's lower face (4 .. 32K-4)
template <typename T, int K>
__device__ __forceinline__ void emf_seg(const T (&vf)[K], T (&bt)[K], T dth, T hd, T (&e2m)[K]) {
  T vn[K], vp[K], vs[K], vsn[K], f[K], fn[K], e1[K], e1p[K], gg[K], ggn[K], d[K], dp[K], P[K], Pn[K];
  next_cell<T, K>(vf, vn);
  prev_cell<T, K>(vf, vp);
#pragma unroll
  for (int i = 0; i < K; ++i) vs[i] = T(0.25) * ((vn[i] + vp[i]) + T(2) * vf[i]);
  next_cell<T, K>(vs, vsn);
#pragma unroll
  for (int i = 0; i < K; ++i) f[i] = vs[i] * bt[i];
  next_cell<T, K>(f, fn);
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const T ve = T(0.5) * (vs[i] + vsn[i]);                       // edge velocity at +1/2
    e1[i] = ve > T(0) ? f[i] : fn[i];                             // first-order EMF
  }
  prev_cell<T, K>(e1, e1p);
#pragma unroll
  for (int i = 0; i < K; ++i) gg[i] = vs[i] * (bt[i] - hd * (e1[i] - e1p[i]));   // vs B_half
  next_cell<T, K>(gg, ggn);
#pragma unroll
  for (int i = 0; i < K; ++i) d[i] = ggn[i] - gg[i];
  prev_cell<T, K>(d, dp);
#pragma unroll
  for (int i = 0; i < K; ++i) P[i] = half_vanleer(dp[i], d[i]);
  next_cell<T, K>(P, Pn);
  T e2[K];
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const T ve = T(0.5) * (vs[i] + vsn[i]);
    e2[i] = ve > T(0) ? gg[i] + P[i] : ggn[i] - Pn[i];          // limited EMF at +1/2
  }
  prev_cell<T, K>(e2, e2m);
#pragma unroll
  for (int i = 0; i < K; ++i) bt[i] = bt[i] - dth * (e2[i] - e2m[i]);
}

// emf_seg<float> of two pipelines at once (lane x and lane y of each float2), f32x2
// arithmetic, with the scales of EmfPipe2: vs kept as 4 vs, EMFs kEmf2Scale x emf_seg's,
// ndth and nhd divided by kEmf2Scale (powers of two: no packed operation rounds differently)
template <int K>
__device__ __forceinline__ void emf_seg2(const float2 (&vf)[K], float2 (&bt)[K], float2 ndth,
                                         float2 nhd, float2 (&e2m)[K]) {
  float2 vn[K], vp[K], vs[K], vsn[K], f[K], fn[K], e1[K], e1p[K], gg[K], ggn[K], d[K], dp[K],
      P[K], Pn[K], ve[K];
  next_cell2<K>(vf, vn);
  prev_cell2<K>(vf, vp);
#pragma unroll
  for (int i = 0; i < K; ++i) vs[i] = fma2(splat2(2.f), vf[i], add2(vn[i], vp[i]));   // 4 vs
  next_cell2<K>(vs, vsn);
#pragma unroll
  for (int i = 0; i < K; ++i) f[i] = mul2(vs[i], bt[i]);
  next_cell2<K>(f, fn);
#pragma unroll
  for (int i = 0; i < K; ++i) {
    ve[i] = add2(vs[i], vsn[i]);                                 // 8 x edge velocity
    e1[i] = sel_pos2(ve[i], f[i], fn[i]);                        // first-order EMF
  }
  prev_cell2<K>(e1, e1p);
#pragma unroll
  for (int i = 0; i < K; ++i) gg[i] = mul2(vs[i], fma2(nhd, sub2(e1[i], e1p[i]), bt[i]));
  next_cell2<K>(gg, ggn);
#pragma unroll
  for (int i = 0; i < K; ++i) d[i] = sub2(ggn[i], gg[i]);
  prev_cell2<K>(d, dp);
#pragma unroll
  for (int i = 0; i < K; ++i) P[i] = half_vanleer2(dp[i], d[i]);
  next_cell2<K>(P, Pn);
  float2 e2[K];
#pragma unroll
  for (int i = 0; i < K; ++i)
    e2[i] = sel_pos2(ve[i], add2(gg[i], P[i]), sub2(ggn[i], Pn[i]));   // limited EMF at +1/2
  prev_cell2<K>(e2, e2m);
#pragma unroll
  for (int i = 0; i < K; ++i) bt[i] = fma2(ndth, sub2(e2[i], e2m[i]), bt[i]);
}

// the value of window cell idx (lane idx / K, element idx % K) of a per-lane K array, in
// every lane
template <typename V, int K>
__device__ __forceinline__ V window_cell(const V (&x)[K], int idx) {
  const int e = idx % K;
  V v = x[0];
#pragma unroll
  for (int i = 1; i < K; ++i) v = (e == i) ? x[i] : v;
  if constexpr (std::is_same<V, float2>::value) {
    return V{__shfl_sync(0xffffffffu, v.x, idx / K), __shfl_sync(0xffffffffu, v.y, idx / K)};
  } else {
    return __shfl_sync(0xffffffffu, v, idx / K);
  }
}

// Between the two passes of an outflow z axis, window cells outside the grid must hold their
// edge cell's first-pass values (a second single pass would read them clamped from the first
// pass's output): copy the edge cell's values over, where the edge cell's first-pass value is
// valid (window cells 4 .. 32K-5).
template <typename V, int K>
__device__ __forceinline__ void reclamp_window(V (&x)[K], int zw0, int z0, int nz) {
  const int lo = -zw0, hi = nz - 1 - zw0;    // window indices of the cells z = 0, nz - 1
  if (lo >= 4 && lo < 32 * K - 4) {
    const V v = window_cell<V, K>(x, lo);
#pragma unroll
    for (int i = 0; i < K; ++i)
      if (z0 + i < 0) x[i] = v;
  }
  if (hi >= 4 && hi < 32 * K - 4) {
    const V v = window_cell<V, K>(x, hi);
#pragma unroll
    for (int i = 0; i < K; ++i)
      if (z0 + i >= nz) x[i] = v;
  }
}

// PASSES = 2: the constrained transport along z applied twice with the same dt (the two
// CT_z operators that meet in the middle of a step whose axis order ends with z, Eq.
// "eq:L_sequence": forward L_z ends with CT_z, reverse L_z starts with it).  The fluid is
// frozen, so both passes use the same face velocities; the second pass takes the first
// pass's advected B_t of the pencil and of its upper rows (the warp's upper-row pipelines
// advect exactly what the neighbouring pencils' own pipelines advect) and adds its EMF
// differences to the first pass's B_z.  Every cell runs the operations of two single passes
// in the same order, so the result is the same bits; the halo doubles (8 cells per side).
template <typename T, int K, bool NC, int PASSES = 1, bool CLAMPZ = false, bool OFF32 = false>
__device__ __forceinline__ void ct_seg_z_warp(const GridDesc& g, const FieldSet<T>& in,
                                              const FieldSet<T>& out, double h, DevScalars* ds,
                                              long long wid) {
  using AD = FieldAddr<T, OFF32>;
  constexpr int H = 4 * PASSES, SEG = 32 * K - 2 * H;
  const int lane = threadIdx.x & 31;
  const int nz = g.n[2], bcz = g.bc[2];
  const SegPlace sp = seg_place(g, nz, SEG, wid);
  const int s0 = sp.s0, x = sp.x, y = sp.y;
  const bool warp_active = sp.active;
  const T dth = step_factor<T>(ds, h);
  const T hd = T(0.5) * dth;
  const typename AD::I row = AD::of((long long)x * g.s[0] + (long long)y * g.s[1]);
  const TransverseOffsets o1 = transverse_offsets(x, g.n[0], g.bc[0], g.s[0]);
  const TransverseOffsets o2 = transverse_offsets(y, g.n[1], g.bc[1], g.s[1]);
  const typename AD::I l1 = AD::of(o1.lo), h1 = AD::of(o1.hi), l2 = AD::of(o2.lo),
                       h2 = AD::of(o2.hi);
  const int z0 = s0 - H + lane * K;
  const T* pr = in.f[0];
  const T* pm = in.f[3];
  // face velocities of the four EMF rows (own and upper row, for t1 = x and t2 = y) and
  // the transverse face fields; B_z for the constraint
  T vo1[K], vn1[K], vo2[K], vn2[K], b1o[K], b1h[K], b2o[K], b2h[K], ba[K];
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const typename AD::I c = row + AD::of(wrap_index(z0 + i, nz, bcz));
    const typename AD::I cl1 = c + l1, ch1 = c + h1, cl2 = c + l2, ch2 = c + h2;
    T r[5], m[5];
    r[0] = ldx<NC>(AD::at(pr, c));     m[0] = ldx<NC>(AD::at(pm, c));
    r[1] = ldx<NC>(AD::at(pr, cl1));   m[1] = ldx<NC>(AD::at(pm, cl1));
    r[2] = ldx<NC>(AD::at(pr, ch1));   m[2] = ldx<NC>(AD::at(pm, ch1));
    r[3] = ldx<NC>(AD::at(pr, cl2));   m[3] = ldx<NC>(AD::at(pm, cl2));
    r[4] = ldx<NC>(AD::at(pr, ch2));   m[4] = ldx<NC>(AD::at(pm, ch2));
    b1o[i] = ldx<NC>(AD::at(in.f[5], c));
    b1h[i] = ldx<NC>(AD::at(in.f[5], ch1));
    b2o[i] = ldx<NC>(AD::at(in.f[6], c));
    b2h[i] = ldx<NC>(AD::at(in.f[6], ch2));
    ba[i] = ldx<NC>(AD::at(in.f[7], c));
    // the upper row's face velocity: across its lower face, the own cell, or (outflow
    // upper edge) the lower neighbour; the operands are chosen first, one quotient each
    const T mx1 = o1.hi_across_lo ? m[1] : m[0], rx1 = o1.hi_across_lo ? r[1] : r[0];
    const T mx2 = o2.hi_across_lo ? m[3] : m[0], rx2 = o2.hi_across_lo ? r[3] : r[0];
    vo1[i] = Num<T>::div(m[0] + m[1], r[0] + r[1]);
    vn1[i] = Num<T>::div(m[2] + mx1, r[2] + rx1);
    vo2[i] = Num<T>::div(m[0] + m[3], r[0] + r[3]);
    vn2[i] = Num<T>::div(m[4] + mx2, r[4] + rx2);
  }
  T eo1[K], en1[K], eo2[K], en2[K];
  constexpr bool PACK = sizeof(T) == 4 && MHD_CT_PACK;
  const T dc = PACK ? dth * T(kEmf2Inv) : dth;   // constraint factor for the EMFs' scale
  T bA[K];
#pragma unroll
  for (int i = 0; i < K; ++i) bA[i] = ba[i];
  if constexpr (PACK) {
    // the own-row pipelines of t1 and t2 as one packed pair, the upper-row ones as another
    float2 vo[K], vn[K], bo[K], bh[K], eo[K], en[K];
#pragma unroll
    for (int i = 0; i < K; ++i) {
      vo[i] = make_float2(vo1[i], vo2[i]);
      vn[i] = make_float2(vn1[i], vn2[i]);
      bo[i] = make_float2(b1o[i], b2o[i]);
      bh[i] = make_float2(b1h[i], b2h[i]);
    }
    const float2 ndth2 = splat2(-(float)dth * kEmf2Inv);
    const float2 nhd2 = splat2(-(float)hd * kEmf2Inv);
#pragma unroll
    for (int pass = 0; pass < PASSES; ++pass) {
      emf_seg2<K>(vo, bo, ndth2, nhd2, eo);
      emf_seg2<K>(vn, bh, ndth2, nhd2, en);
#pragma unroll
      for (int i = 0; i < K; ++i) {
        bA[i] = ffma(dc, en[i].x - eo[i].x, bA[i]);   // constraint from t1 = x, then t2 = y
        bA[i] = ffma(dc, en[i].y - eo[i].y, bA[i]);
      }
      if (CLAMPZ && pass + 1 < PASSES) {
        reclamp_window<float2, K>(bo, s0 - H, z0, nz);
        reclamp_window<float2, K>(bh, s0 - H, z0, nz);
        reclamp_window<T, K>(bA, s0 - H, z0, nz);
      }
    }
#pragma unroll
    for (int i = 0; i < K; ++i) {
      b1o[i] = bo[i].x; b2o[i] = bo[i].y;
    }
  } else {
#pragma unroll
    for (int pass = 0; pass < PASSES; ++pass) {
      emf_seg<T, K>(vo1, b1o, dth, hd, eo1);
      emf_seg<T, K>(vn1, b1h, dth, hd, en1);
      emf_seg<T, K>(vo2, b2o, dth, hd, eo2);
      emf_seg<T, K>(vn2, b2h, dth, hd, en2);
#pragma unroll
      for (int i = 0; i < K; ++i) {
        bA[i] = ffma(dc, en1[i] - eo1[i], bA[i]);     // constraint from t1 = x, then t2 = y
        bA[i] = ffma(dc, en2[i] - eo2[i], bA[i]);
      }
      if (CLAMPZ && pass + 1 < PASSES) {
        reclamp_window<T, K>(b1o, s0 - H, z0, nz);
        reclamp_window<T, K>(b1h, s0 - H, z0, nz);
        reclamp_window<T, K>(b2o, s0 - H, z0, nz);
        reclamp_window<T, K>(b2h, s0 - H, z0, nz);
        reclamp_window<T, K>(bA, s0 - H, z0, nz);
      }
    }
  }
  int st = 0;
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const int w = lane * K + i, z = z0 + i;
    if (warp_active && w >= H && w < H + SEG && z < nz) {
      const typename AD::I co = row + AD::of(z);
      *AD::at(out.f[5], co) = b1o[i];
      *AD::at(out.f[6], co) = b2o[i];
      *AD::at(out.f[7], co) = bA[i];
      if (!(b1o[i] == b1o[i]) || !(b2o[i] == b2o[i]) || !(bA[i] == bA[i])) st |= ST_NONFINITE;
    }
  }
  if (st) atomicOr(&ds->status, st);
}

// CLAMPZ: the z axis is outflow (the two-pass form re-clamps its ghost cells between passes)
template <typename T, int NW, int K, int PASSES = 1, bool CLAMPZ = false, bool OFF32 = false>
__global__ void __launch_bounds__(32 * NW, SegMinBlocks<T>::ct)
ct_seg_z(GridDesc g, FieldSet<T> in, FieldSet<T> out, double h, DevScalars* ds) {
  ct_seg_z_warp<T, K, true, PASSES, CLAMPZ, OFF32>(g, in, out, h, ds,
                                                   (long long)blockIdx.x * NW + (threadIdx.x >> 5));
}


// ------------------------------------------------------------------------------------
// Constrained transport along z with shared EMF rows (FP32): ct_rows_z.
//
// ct_seg_z runs four EMF pipelines per pencil: the own row's and the upper row's, for each
// transverse component; the upper rows' pipelines are the neighbouring pencils' own ones
// (same operands, the packed lanes independent).  Here a block of Q warps covers Q
// neighbouring y rows (warp w: pencil y = yb + w) of one z window and marches along x over L
// rows, and each warp runs only its own pair of pipelines (t1 = x, t2 = y):
//   - the y-face EMF of the upper y row comes from warp w + 1 through shared memory (double
//     buffered by row parity, one block barrier per row); warp Q - 1 only supplies it;
//   - the x-face EMF of the upper x row is the own x-face EMF of the next row of the march,
//     so the constraint on B_z of row r completes one row later (three values per cell
//     carried in registers: B_z, the x-face EMF, and the y-face EMF difference);
//   - the face velocity of the x-face takes rho and m_z of the previous row from registers;
//     that of the y-face loads the lower y row (the same data warp w - 1 loads: an L1 hit).
// Per cell: 2 pipelines x Q/(Q-1) x (L+1)/L and 7 loads, against 4 pipelines and 15 loads.
// At the outflow upper edge of x or y the upper row's pipeline is the own one (the upper row
// clamps onto the row itself and its face velocity is taken across its lower face), as in
// ct_seg_z.  Every output value comes from the same operations on the same operands as in
// ct_seg_z, in the same order, so the two kernels give the same bits; PASSES = 2 is the
// middle pair of a step (two passes with the same dt, ghost cells re-clamped between passes
// on an outflow z axis).
// ------------------------------------------------------------------------------------
#ifndef MHD_CTZ_ROWS
#define MHD_CTZ_ROWS 1
#endif
#ifndef MHD_CTZ_Q
#define MHD_CTZ_Q 8
#endif
#ifndef MHD_CTZ_L
#define MHD_CTZ_L 16
#endif
// resident blocks asked of the compiler: by default a 64-register cap (32 / Q blocks of Q
// warps per SM)
#ifndef MHD_CTZ_MINB
#define MHD_CTZ_MINB 0
#endif
// load the operands of the next row of the march while the current one computes (measured
// at 512^3: the one-pass kernel 0.977 -> 0.966 ms with a 79-register cap, 1.21 ms at 64
// registers; the two-pass pair 1.29 -> 1.36-1.90 ms: off)
#ifndef MHD_CTZ_PREFETCH
#define MHD_CTZ_PREFETCH 0
#endif
#ifndef MHD_CTZ2_MINB
#define MHD_CTZ2_MINB 0
#endif
template <int Q, int PASSES> struct CtRowsZMinBlocks {
  static constexpr int m = PASSES == 2 ? MHD_CTZ2_MINB : MHD_CTZ_MINB;
  static constexpr int value = m > 0 ? m : (Q <= 32 ? 32 / Q : 1);
};

template <int K, int Q, int PASSES = 1, bool CLAMPZ = false, bool OFF32 = false>
__global__ void __launch_bounds__(32 * Q, CtRowsZMinBlocks<Q, PASSES>::value)
ct_rows_z(GridDesc g, FieldSet<float> in, FieldSet<float> out, double h, DevScalars* ds, int L) {
  using AD = FieldAddr<float, OFF32>;
  using I = typename AD::I;
  constexpr int H = 4 * PASSES, W = 32 * K, SEG = W - 2 * H;
  __shared__ float se[2][PASSES][Q][W];   // y-face EMF of each warp's own pipelines
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const int bcx = g.bc[0], bcy = g.bc[1], bcz = g.bc[2];
  const int yw = (int)blockIdx.x * (Q - 1) + w;          // unwrapped y of the warp's pencil
  const int s0 = (int)blockIdx.y * SEG;
  const int xb = (int)blockIdx.z * L;
  const int xe = min(xb + L, nx);
  const int y = wrap_index(yw, ny, bcy), ylo = wrap_index(y - 1, ny, bcy);
  // the upper y row's across-face cell is the lower neighbour: its pipeline is the own one
  const bool y_edge = wrap_index(wrap_index(y + 1, ny, bcy) - 1, ny, bcy) != y;
  const bool writer = w < Q - 1 && yw < ny;
  const int wn = w + 1 < Q ? w + 1 : w;
  // outflow upper x edge in this block: the last row's upper-row pipeline is its own
  const bool x_edge = xe == nx && bcx == 1;
  const float dth = step_factor<float>(ds, h), hd = 0.5f * dth;
  const float2 ndth2 = splat2(-dth * kEmf2Inv), nhd2 = splat2(-hd * kEmf2Inv);
  const float dc = dth * kEmf2Inv;                        // the packed EMFs are kEmf2Scale x
  const int z0 = s0 - H + lane * K;
  I zc[K];
#pragma unroll
  for (int i = 0; i < K; ++i) zc[i] = AD::of(wrap_index(z0 + i, nz, bcz));
  const I ys = AD::of((long long)y * g.s[1]), ylos = AD::of((long long)ylo * g.s[1]);
  // rho and m_z of the row below the first one
  float rp[K], mp[K];
  {
    const I row = AD::of((long long)wrap_index(xb - 1, nx, bcx) * g.s[0]) + ys;
#pragma unroll
    for (int i = 0; i < K; ++i) {
      rp[i] = __ldg(AD::at(in.f[0], row + zc[i]));
      mp[i] = __ldg(AD::at(in.f[3], row + zc[i]));
    }
  }
  // carried from row r - 1 to row r: B_z, own x-face EMF and y-face EMF difference per pass
  float bap[K], e1p[PASSES][K], d2p[PASSES][K];
#pragma unroll
  for (int i = 0; i < K; ++i) {
    bap[i] = 0.f;
#pragma unroll
    for (int p = 0; p < PASSES; ++p) e1p[p][i] = d2p[p][i] = 0.f;
  }
  I xop = 0;                      // x offset of the previous row
  int st = 0;
  // output cells of the window: w in [H, H + SEG), z < nz
  bool outc[K];
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const int wc = lane * K + i;
    outc[i] = writer && wc >= H && wc < H + SEG && z0 + i < nz;
  }
  // B_z of the previous row from its carried values and this row's x-face EMF (en1)
  auto finish_bz = [&](const float (&en1)[PASSES][K]) {
    float b[K];
#pragma unroll
    for (int i = 0; i < K; ++i) b[i] = bap[i];
#pragma unroll
    for (int p = 0; p < PASSES; ++p) {
#pragma unroll
      for (int i = 0; i < K; ++i) {
        b[i] = ffma(dc, en1[p][i] - e1p[p][i], b[i]);   // constraint from t1 = x, then t2 = y
        b[i] = ffma(dc, d2p[p][i], b[i]);
      }
      if (CLAMPZ && p + 1 < PASSES) reclamp_window<float, K>(b, s0 - H, z0, nz);
    }
#pragma unroll
    for (int i = 0; i < K; ++i)
      if (outc[i]) {
        const I co = xop + ys + AD::of(z0 + i);
        *AD::at(out.f[7], co) = b[i];
        if (!(b[i] == b[i])) st |= ST_NONFINITE;
      }
  };
  const int rlast = x_edge ? xe - 1 : xe;
  // the operands of a row: rho, m_z, B_x, B_y, B_z of the pencil, rho and m_z of the row
  // below across y; with MHD_CTZ_PREFETCH those of row r + 1 are loaded while row r computes
  float q0[K], q1[K], q2[K], q3[K], q4[K], q5[K], q6[K];
  auto load_row = [&](int r) {
    const I xo = AD::of((long long)wrap_index(r, nx, bcx) * g.s[0]);
    const I row = xo + ys, rowlo = xo + ylos;
#pragma unroll
    for (int i = 0; i < K; ++i) {
      const I c = row + zc[i], cl = rowlo + zc[i];
      q0[i] = __ldg(AD::at(in.f[0], c));
      q1[i] = __ldg(AD::at(in.f[3], c));
      q2[i] = __ldg(AD::at(in.f[0], cl));
      q3[i] = __ldg(AD::at(in.f[3], cl));
      q4[i] = __ldg(AD::at(in.f[5], c));
      q5[i] = __ldg(AD::at(in.f[6], c));
      q6[i] = __ldg(AD::at(in.f[7], c));
    }
  };
  if (MHD_CTZ_PREFETCH) load_row(xb);
  for (int r = xb; r <= rlast; ++r) {
    const I xo = AD::of((long long)wrap_index(r, nx, bcx) * g.s[0]);
    const I row = xo + ys;
    if (!MHD_CTZ_PREFETCH) load_row(r);
    float r0[K], m0[K], bz[K];
    float2 vo[K], bo[K];
#pragma unroll
    for (int i = 0; i < K; ++i) {
      r0[i] = q0[i];
      m0[i] = q1[i];
      bo[i] = make_float2(q4[i], q5[i]);
      bz[i] = q6[i];
      vo[i] = make_float2(Num<float>::div(m0[i] + mp[i], r0[i] + rp[i]),
                          Num<float>::div(m0[i] + q3[i], r0[i] + q2[i]));
    }
    if (MHD_CTZ_PREFETCH && r < rlast) load_row(r + 1);
    float2 eo[PASSES][K];
#pragma unroll
    for (int p = 0; p < PASSES; ++p) {
      emf_seg2<K>(vo, bo, ndth2, nhd2, eo[p]);
      if (CLAMPZ && p + 1 < PASSES) reclamp_window<float2, K>(bo, s0 - H, z0, nz);
    }
    if (r > xb) {
      float en1[PASSES][K];
#pragma unroll
      for (int p = 0; p < PASSES; ++p)
#pragma unroll
        for (int i = 0; i < K; ++i) en1[p][i] = eo[p][i].x;
      finish_bz(en1);
    }
    if (r < xe) {
#pragma unroll
      for (int i = 0; i < K; ++i)
        if (outc[i]) {
          const I co = row + AD::of(z0 + i);
          *AD::at(out.f[5], co) = bo[i].x;
          *AD::at(out.f[6], co) = bo[i].y;
          if (!(bo[i].x == bo[i].x) || !(bo[i].y == bo[i].y)) st |= ST_NONFINITE;
        }
      float(&sw)[PASSES][Q][W] = se[r & 1];
#pragma unroll
      for (int p = 0; p < PASSES; ++p)
#pragma unroll
        for (int i = 0; i < K; ++i) sw[p][w][lane * K + i] = eo[p][i].y;
      __syncthreads();
#pragma unroll
      for (int p = 0; p < PASSES; ++p)
#pragma unroll
        for (int i = 0; i < K; ++i) {
          const float en2 = y_edge ? eo[p][i].y : sw[p][wn][lane * K + i];
          d2p[p][i] = en2 - eo[p][i].y;
          e1p[p][i] = eo[p][i].x;
        }
#pragma unroll
      for (int i = 0; i < K; ++i) bap[i] = bz[i];
      xop = xo;
    }
#pragma unroll
    for (int i = 0; i < K; ++i) { rp[i] = r0[i]; mp[i] = m0[i]; }
  }
  if (x_edge) finish_bz(e1p);   // the last row's upper-row x-face EMF is its own
  if (st) atomicOr(&ds->status, st);
}

// ct_rows_z launch geometry: blocks of Q warps over (y rows, z windows, x row groups)
template <int K, int PASSES>
__host__ inline bool ct_rows_z_grid(const GridDesc& g, int Q, int L, dim3* grid) {
  constexpr int SEG = 32 * K - 8 * PASSES;
  const long long gx = (g.n[1] + Q - 2) / (Q - 1), gy = (g.n[2] + SEG - 1) / SEG,
                  gz = (g.n[0] + L - 1) / L;
  if (gx > 0x7FFFFFFFll || gy > 65535 || gz > 65535) return false;
  *grid = dim3((unsigned)gx, (unsigned)gy, (unsigned)gz);
  return true;
}


// ------------------------------------------------------------------------------------
// The reverse z operator L_z (CT_z, then fluid_z) in one launch, FP32: ct_fluid_rows_z.
//
// The march of ct_rows_z, with the fluid sweep of each pencil run as soon as the B it
// needs is final: the fluid of row r needs the advected B_x of its own and of the next row
// (its cell-centred B_x), the advected B_y of its own and of the upper y row (the warp above,
// through shared memory), and B_z, whose constraint completes with the x-face EMF of row r + 1.
// So in iteration r a warp runs the CT of row r and then the fluid of row r - 1, whose rho
// and m_z it loaded as CT operands one iteration earlier.  Unlike the forward order (fluid,
// then CT), no pencil's fluid is evaluated twice across x or y: the face velocities come from
// the input state.  The window pays instead: the fluid's stencil reaches 3 cells and B_z the
// CT's 4, so a window of 32K cells updates 32K - 14 (against 32K - 6 and 32K - 8 for the two
// operators apart).  Every value is the same operation on the same operands as ct_seg_z
// followed by fluid_seg_z (ghost cells of an outflow z axis re-clamped to their edge cells,
// as the fluid's clamped loads of the CT's output would read them), so the result is the same
// bits.  Not the last sweep of a step (no c_max reduction).
// ------------------------------------------------------------------------------------
#ifndef MHD_LOPZ_Q
#define MHD_LOPZ_Q 8
#endif
#ifndef MHD_LOPZ_MINB
#define MHD_LOPZ_MINB 2
#endif

template <int K, int Q, int PM, bool CLAMPZ = false, bool OFF32 = false>
__global__ void __launch_bounds__(32 * Q, MHD_LOPZ_MINB)
ct_fluid_rows_z(GridDesc g, FieldSet<float> in, FieldSet<float> out, float gamma, double h,
                DevScalars* ds, int L) {
  using AD = FieldAddr<float, OFF32>;
  using I = typename AD::I;
  constexpr int HL = 7, W = 32 * K, SEG = W - 14;
  __shared__ float se[2][Q][W];   // y-face EMF of each warp's own pipeline
  __shared__ float sb[2][Q][W];   // advected B_y of each warp's pencil (the lower warp's fluid)
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const int bcx = g.bc[0], bcy = g.bc[1], bcz = g.bc[2];
  const int yw = (int)blockIdx.x * (Q - 1) + w;
  const int s0 = (int)blockIdx.y * SEG;
  const int xb = (int)blockIdx.z * L;
  const int xe = min(xb + L, nx);
  const int y = wrap_index(yw, ny, bcy), ylo = wrap_index(y - 1, ny, bcy);
  const int yup = wrap_index(y + 1, ny, bcy);
  const bool y_edge = wrap_index(yup - 1, ny, bcy) != y;   // upper EMF row = own
  const bool y_self = yup == y;                             // upper B_y row = own
  const bool writer = w < Q - 1 && yw < ny;
  const int wn = w + 1 < Q ? w + 1 : w;
  const bool x_edge = xe == nx && bcx == 1;
  const float dts = step_factor<float>(ds, h);
  const float2 ndth2 = splat2(-dts * kEmf2Inv), nhd2 = splat2(-(0.5f * dts) * kEmf2Inv);
  const float dc = dts * kEmf2Inv;
  const float fdth = dts * float(FluxScale<float>::inv), fhd = 0.5f * fdth;
  const int z0 = s0 - HL + lane * K;
  I zc[K];
#pragma unroll
  for (int i = 0; i < K; ++i) zc[i] = AD::of(wrap_index(z0 + i, nz, bcz));
  const I ys = AD::of((long long)y * g.s[1]), ylos = AD::of((long long)ylo * g.s[1]);
  float rp[K], mp[K];
  {
    const I row = AD::of((long long)wrap_index(xb - 1, nx, bcx) * g.s[0]) + ys;
#pragma unroll
    for (int i = 0; i < K; ++i) {
      rp[i] = __ldg(AD::at(in.f[0], row + zc[i]));
      mp[i] = __ldg(AD::at(in.f[3], row + zc[i]));
    }
  }
  // carried from row r - 1: B_z, x-face EMF, y-face EMF difference (the constraint), the
  // advected B_x and B_y of the pencil and B_y of the upper y row (the fluid's cell-centred B)
  float bap[K], e1p[K], d2p[K], bxp[K], byp[K], byu[K];
#pragma unroll
  for (int i = 0; i < K; ++i) bap[i] = e1p[i] = d2p[i] = bxp[i] = byp[i] = byu[i] = 0.f;
  I xop = 0;
  int st = 0;
  bool outc[K];
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const int wc = lane * K + i;
    outc[i] = writer && wc >= HL && wc < HL + SEG && z0 + i < nz;
  }
  // B_z of row r - 1 (stored), then its fluid sweep; en1: x-face EMF of the upper x row,
  // bxu: advected B_x of the upper x row
  auto finish_row = [&](const float (&en1)[K], const float (&bxu)[K]) {
    float bz[K];
#pragma unroll
    for (int i = 0; i < K; ++i) {
      float b = ffma(dc, en1[i] - e1p[i], bap[i]);   // constraint from t1 = x, then t2 = y
      bz[i] = ffma(dc, d2p[i], b);
    }
#pragma unroll
    for (int i = 0; i < K; ++i)
      if (outc[i]) {
        *AD::at(out.f[7], xop + ys + AD::of(z0 + i)) = bz[i];
        if (!(bz[i] == bz[i])) st |= ST_NONFINITE;
      }
    if (CLAMPZ) reclamp_window<float, K>(bz, s0 - HL, z0, nz);
    float bzn[K];
    next_cell<float, K>(bz, bzn);
    float u[K][5], bb[K][3], un[K][5];
#pragma unroll
    for (int i = 0; i < K; ++i) {
      const I c = xop + ys + zc[i];
      u[i][0] = rp[i];
      u[i][1] = mp[i];
      u[i][2] = __ldg(AD::at(in.f[1], c));
      u[i][3] = __ldg(AD::at(in.f[2], c));
      u[i][4] = __ldg(AD::at(in.f[4], c));
      bb[i][0] = 0.5f * (bz[i] + bzn[i]);
      bb[i][1] = 0.5f * (bxp[i] + bxu[i]);
      bb[i][2] = 0.5f * (byp[i] + byu[i]);
    }
    // the CT's output, hence the cell-centred B, is valid on window cells 4 .. 32K-5
    st |= fluid_seg_core<float, PM, K>(u, bb, gamma, fdth, fhd, lane, 4, W - 5, un);
#pragma unroll
    for (int i = 0; i < K; ++i)
      if (outc[i]) {
        const I co = xop + ys + AD::of(z0 + i);
        *AD::at(out.f[0], co) = un[i][0];
        *AD::at(out.f[3], co) = un[i][1];
        *AD::at(out.f[1], co) = un[i][2];
        *AD::at(out.f[2], co) = un[i][3];
        *AD::at(out.f[4], co) = un[i][4];
        if (!(un[i][0] > 0.f)) st |= ST_UNPHYSICAL;
      }
  };
  const int rlast = x_edge ? xe - 1 : xe;
  for (int r = xb; r <= rlast; ++r) {
    const I xo = AD::of((long long)wrap_index(r, nx, bcx) * g.s[0]);
    const I row = xo + ys, rowlo = xo + ylos;
    float r0[K], m0[K], bz[K];
    float2 vo[K], bo[K], eo[K];
#pragma unroll
    for (int i = 0; i < K; ++i) {
      const I c = row + zc[i], cl = rowlo + zc[i];
      r0[i] = __ldg(AD::at(in.f[0], c));
      m0[i] = __ldg(AD::at(in.f[3], c));
      const float rl = __ldg(AD::at(in.f[0], cl)), ml = __ldg(AD::at(in.f[3], cl));
      bo[i] = make_float2(__ldg(AD::at(in.f[5], c)), __ldg(AD::at(in.f[6], c)));
      bz[i] = __ldg(AD::at(in.f[7], c));
      vo[i] = make_float2(Num<float>::div(m0[i] + mp[i], r0[i] + rp[i]),
                          Num<float>::div(m0[i] + ml, r0[i] + rl));
    }
    emf_seg2<K>(vo, bo, ndth2, nhd2, eo);
    if (CLAMPZ) reclamp_window<float2, K>(bo, s0 - HL, z0, nz);
    if (r > xb) {
      float en1[K], bxu[K];
#pragma unroll
      for (int i = 0; i < K; ++i) { en1[i] = eo[i].x; bxu[i] = bo[i].x; }
      finish_row(en1, bxu);
    }
    if (r < xe) {
#pragma unroll
      for (int i = 0; i < K; ++i)
        if (outc[i]) {
          const I co = row + AD::of(z0 + i);
          *AD::at(out.f[5], co) = bo[i].x;
          *AD::at(out.f[6], co) = bo[i].y;
          if (!(bo[i].x == bo[i].x) || !(bo[i].y == bo[i].y)) st |= ST_NONFINITE;
        }
      float(&swe)[Q][W] = se[r & 1];
      float(&swb)[Q][W] = sb[r & 1];
#pragma unroll
      for (int i = 0; i < K; ++i) {
        swe[w][lane * K + i] = eo[i].y;
        swb[w][lane * K + i] = bo[i].y;
      }
      __syncthreads();
#pragma unroll
      for (int i = 0; i < K; ++i) {
        const float en2 = y_edge ? eo[i].y : swe[wn][lane * K + i];
        d2p[i] = en2 - eo[i].y;
        e1p[i] = eo[i].x;
        byu[i] = y_self ? bo[i].y : swb[wn][lane * K + i];
        bap[i] = bz[i];
        bxp[i] = bo[i].x;
        byp[i] = bo[i].y;
      }
      xop = xo;
    }
#pragma unroll
    for (int i = 0; i < K; ++i) { rp[i] = r0[i]; mp[i] = m0[i]; }
  }
  if (x_edge) {
    // the last row: its upper x row is itself (outflow), for the EMF and for B_x
    float en1[K], bxu[K];
#pragma unroll
    for (int i = 0; i < K; ++i) { en1[i] = e1p[i]; bxu[i] = bxp[i]; }
    finish_row(en1, bxu);
  }
  if (st) atomicOr(&ds->status, st);
}

template <int K>
__host__ inline bool ct_fluid_rows_z_grid(const GridDesc& g, int Q, int L, dim3* grid) {
  constexpr int SEG = 32 * K - 14;
  const long long gx = (g.n[1] + Q - 2) / (Q - 1), gy = (g.n[2] + SEG - 1) / SEG,
                  gz = (g.n[0] + L - 1) / L;
  if (gx > 0x7FFFFFFFll || gy > 65535 || gz > 65535) return false;
  *grid = dim3((unsigned)gx, (unsigned)gy, (unsigned)gz);
  return true;
}

}  // namespace mhd
