// Marching fluid sweep: one thread per pencil, walking along the sweep axis with a sliding
// register window (Algorithm 1 evaluated cell by cell as the pencil streams in).
//
// At iteration k the thread has loaded cell j = js + k and holds, in registers,
//   u(j-1..j-3), cell-centred B (j-1..j-3), the stage-1 right-moving flux of j-1, the
//   first-order interface flux at (j-2)+1/2, the stage-2 fluxes and their differences
//   around j-3, and the limited interface flux at (j-4)+1/2.
// It then forms the stage-1 fluxes of j, the first-order flux at (j-1)+1/2, the half step
// u^{t+dt/2}(j-1) (Eq. "eq:Delta_u_half"), its stage-2 fluxes, the limited interface flux at
// (j-3)+1/2 (Eqs. "eq:Delta_F", "eq:limiter", "eq:F_n" and the mirrored left-moving form)
// and the full update of cell j-3 (Eq. "eq:Delta_u_full").  Every flux is evaluated once.
//
// The operation order of each expression matches the oracle (phi(a/2, b/2) is evaluated
// as phi(a, b)/2, which is the same rounded value), so the FP64 build without FMA
// contraction reproduces it bit for bit.  In FP32 every flux in the window is doubled
// (cell_flux, FluxScale) and dth, hd come halved.
#pragma once

#include "mhd_kernels.cuh"

namespace mhd {

template <typename T, int PM, bool LAST>
struct FluidPencil {
  T u1[5], u2[5], u3[5];   // u(j-1), u(j-2), u(j-3)
  T b1[3], b2[3], b3[3];   // cell-centred B at j-1, j-2, j-3
  T fr1[5];                // stage-1 FR(j-1)
  T g1[5];                 // first-order interface flux at (j-2)+1/2
  T frA[5], frB[5];        // stage-2 FR(j-3), FR(j-2)
  T dRp[5];                // FR2(j-3) - FR2(j-4)
  T flL[5], dLp[5];        // FL2(j-2), FL2(j-2) - FL2(j-3)
  T g2[5];                 // limited interface flux at (j-4)+1/2
  int st;

  __device__ __forceinline__ void init() {
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      u1[c] = u2[c] = u3[c] = T(0);
      fr1[c] = g1[c] = frA[c] = frB[c] = dRp[c] = flL[c] = dLp[c] = g2[c] = T(0);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) b1[c] = b2[c] = b3[c] = T(0);
    st = 0;
  }

  // Push cell j (iteration k).  Returns true when `out` holds u^{t+dt} of cell j-3, and
  // then `bout` its cell-centred B (for the fused CFL speed).
  __device__ __forceinline__ bool push(int k, const T u0[5], const T b0[3], T gamma, T dth,
                                       T hd, T out[5], T bout[3]) {
    T fr0[5], fl0[5];
    st |= cell_flux<T, PM>(u0, b0, gamma, fr0, fl0);
    T uh[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      const T g1c = fr1[c] - fl0[c];                 // first-order flux at (j-1)+1/2
      uh[c] = ffms(hd, g1c - g1[c], u1[c]);          // u^{t+dt/2}(j-1)
      g1[c] = g1c;
      fr1[c] = fr0[c];
    }
    T fr2[5], fl2[5];
    const int s2 = cell_flux<T, PM>(uh, b1, gamma, fr2, fl2);
    if (k >= 2) st |= s2;
    T g2c[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      const T dRc = frB[c] - frA[c];                 // FR2(j-2) - FR2(j-3)
      const T right = plus_half_vanleer(frA[c], dRp[c], dRc);
      const T dLc = fl2[c] - flL[c];                 // FL2(j-1) - FL2(j-2)
      const T left = minus_half_vanleer(flL[c], dLp[c], dLc);
      g2c[c] = right - left;                         // limited flux at (j-3)+1/2
      dRp[c] = dRc;
      frA[c] = frB[c];
      frB[c] = fr2[c];
      dLp[c] = dLc;
      flL[c] = fl2[c];
    }
    const bool valid = k >= 6;
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      out[c] = ffms(dth, g2c[c] - g2[c], u3[c]);
      g2[c] = g2c[c];
      u3[c] = u2[c];
      u2[c] = u1[c];
      u1[c] = u0[c];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      bout[c] = b3[c];
      if (LAST) {
        b3[c] = b2[c];
        b2[c] = b1[c];
      }
      b1[c] = b0[c];
    }
    if (!LAST) {
      // b3 only feeds the CFL speed of the LAST variant
    }
    return valid;
  }
};

template <typename T>
__device__ __forceinline__ long long wrap_off(int i, int n, int bc, long long stride) {
  return (long long)wrap_index(i, n, bc) * stride;
}

// Offset of the next row along the sweep axis that a march stages: rows advance by the
// axis stride, and take the axis' wrap only where they cross its ends (one compare per row
// instead of a wrap and a 64-bit product; the index arithmetic is a large share of the
// issue-bound marches)
struct RowCursor {
  int a, n, bc;
  long long s, off;
  __device__ __forceinline__ RowCursor(int a0, int n_, int bc_, long long s_)
      : a(a0), n(n_), bc(bc_), s(s_), off((long long)wrap_index(a0, n_, bc_) * s_) {}
  __device__ __forceinline__ void advance() {
    if ((unsigned)a < (unsigned)(n - 1)) off += s;      // a and a + 1 inside the axis
    else off = (long long)wrap_index(a + 1, n, bc) * s;
    ++a;
  }
};

// Asynchronous global -> shared copies (cp.async): each thread prefetches the inputs of
// the iterations D ahead of the one it computes into its own slots of a shared ring, so
// that the loads of a march stay in flight while the arithmetic of earlier cells runs.
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* smem, const T* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  if (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// prefetch depth (iterations ahead) and ring length of the marching kernels
// (at 512^3, 3 iterations ahead run 1.2% faster for the fluid and 1.1% for the CT than 4;
// 5 was no better, 6 slower)
#ifndef MHD_MARCH_DEPTH
#define MHD_MARCH_DEPTH 3
#endif
constexpr int kMarchDepth = MHD_MARCH_DEPTH;
constexpr int kMarchRing = kMarchDepth + 1;
// cells per marching tile along the sweep (the halo of 6 or 8 cells is recomputed per
// tile).  The single-grid kernels and the batched kernel use the same length, so that a
// grid's FP32 result does not depend on which of them advanced it.
#ifndef MHD_MARCH_S
#define MHD_MARCH_S 192
#endif
constexpr int kMarchS = MHD_MARCH_S;

// unroll factors of the marching loops: a window of depth d shifts without register moves
// when the loop body is repeated a multiple of d times
#ifndef MHD_FLUID_UNROLL
#define MHD_FLUID_UNROLL 3
#endif
#ifndef MHD_CT_UNROLL
#define MHD_CT_UNROLL 4
#endif
// minimum resident blocks per SM requested from the compiler (register cap) for the
// fluid and CT marches; 0 names no minimum.  The fluid march names none: the compiler then
// fits it in 128 registers without spills (4 blocks per SM), where naming one block gave 160
// registers and 3 blocks, 0.5% (512^3) to 4.7% (256^3) slower with identical results.
#ifndef MHD_MARCH_MINB
#define MHD_MARCH_MINB 0
#endif
#ifndef MHD_CT_MINB
#define MHD_CT_MINB 4
#endif
constexpr int kFluidUnroll = MHD_FLUID_UNROLL;
constexpr int kCtUnroll = MHD_CT_UNROLL;

// ------------------------------------------------------------------------------------
// x or y sweep (A = 0, 1): threads take consecutive positions of the transverse plane with
// z fastest (coalesced rows per field); each thread marches its pencil over S cells plus
// the 6-cell halo.  blockIdx.y selects the tile along the sweep.
// ------------------------------------------------------------------------------------
// one tile: pencils bx*NT .. bx*NT+NT-1 of the transverse plane, cells by*S .. by*S+S-1
// along the sweep; smem_raw holds the prefetch ring (march_ring_bytes)
template <typename T, int A, bool LAST, int PM, int S, int NT>
__device__ __forceinline__ void fluid_march_xy_tile_elem(const GridDesc& g, const FieldSet<T>& in,
                                                         const FieldSet<T>& out, T gamma, double h,
                                                         DevScalars* ds, unsigned bx, unsigned by,
                                                         unsigned char* smem_raw) {
  static_assert(A == 0 || A == 1, "x or y sweep");
  constexpr int O = (A == 0) ? 1 : 0;       // the transverse axis that is not z
  constexpr int T1 = axis_t1(A), T2 = axis_t2(A);
  const long long p = (long long)bx * NT + threadIdx.x;
  const int z = (int)(p % g.n[2]);
  const long long o_ = p / g.n[2];
  const int o = (int)(o_ < g.n[O] ? o_ : g.n[O]);
  const int a0 = by * S;
  const int nA = g.n[A], bcA = g.bc[A];
  const bool active = o_ < g.n[O];
  const T dth = step_factor<T>(ds, h) * T(FluxScale<T>::inv);   // for cell_flux's flux scale
  const T hd = T(0.5) * dth;
  const int zc = min(z, g.n[2] - 1), oc = min(o, g.n[O] - 1);
  const long long base = (long long)zc + (long long)oc * g.s[O];
  // offsets of the +1 neighbour across the t1 and t2 faces (for the cell-centred B)
  const long long s1 = (T1 == 2) ? (long long)(wrap_index(zc + 1, g.n[2], g.bc[2]) - zc)
                                 : (long long)(wrap_index(oc + 1, g.n[O], g.bc[O]) - oc) * g.s[O];
  const long long s2 = (T2 == 2) ? (long long)(wrap_index(zc + 1, g.n[2], g.bc[2]) - zc)
                                 : (long long)(wrap_index(oc + 1, g.n[O], g.bc[O]) - oc) * g.s[O];
  const T* __restrict__ pr = in.f[0];
  const T* __restrict__ pn = in.f[1 + A];
  const T* __restrict__ p1 = in.f[1 + T1];
  const T* __restrict__ p2 = in.f[1 + T2];
  const T* __restrict__ pe = in.f[4];
  const T* __restrict__ bn = in.f[5 + A];
  const T* __restrict__ bt1 = in.f[5 + T1];
  const T* __restrict__ bt2 = in.f[5 + T2];
  const long long sA = g.s[A];

  FluidPencil<T, PM, LAST> P;
  P.init();
  const int js = a0 - 3;
  const int kend = min(S, nA - a0) + 6;       // iterations needed for this tile
  // shared ring: [slot][value][thread], 10 values per iteration (u, B_n(j+1), B_t1 x2, B_t2 x2)
  T* ring = reinterpret_cast<T*>(smem_raw);
  constexpr int NV = 10;
  RowCursor rc(js, nA, bcA, sA), rn(js + 1, nA, bcA, sA);
  auto issue = [&](int kk) {
    if (kk < kend) {
      const long long c = base + rc.off;
      const long long cn = base + rn.off;
      rc.advance();
      rn.advance();
      T* slot = ring + (size_t)((unsigned)kk % kMarchRing) * NV * NT + threadIdx.x;
      cp_async_elem(slot + 0 * NT, pr + c);
      cp_async_elem(slot + 1 * NT, pn + c);
      cp_async_elem(slot + 2 * NT, p1 + c);
      cp_async_elem(slot + 3 * NT, p2 + c);
      cp_async_elem(slot + 4 * NT, pe + c);
      cp_async_elem(slot + 5 * NT, bn + cn);
      cp_async_elem(slot + 6 * NT, bt1 + c);
      cp_async_elem(slot + 7 * NT, bt1 + c + s1);
      cp_async_elem(slot + 8 * NT, bt2 + c);
      cp_async_elem(slot + 9 * NT, bt2 + c + s2);
    }
    cp_async_commit();
  };
#pragma unroll
  for (int d = 0; d < kMarchDepth; ++d) issue(d);
  // B_n of the first cell (each iteration brings B_n one cell ahead)
  T bn_cur = bn[base + wrap_off<T>(js, nA, bcA, sA)];
  T cm = T(0);
  bool nan_seen = false;
#pragma unroll kFluidUnroll
  for (int k = 0; k < kend; ++k) {
    issue(k + kMarchDepth);
    cp_async_wait<kMarchDepth>();
    const T* slot = ring + (size_t)((unsigned)k % kMarchRing) * NV * NT + threadIdx.x;
    const int j = js + k;
    T u0[5], b0[3];
#pragma unroll
    for (int c = 0; c < 5; ++c) u0[c] = slot[c * NT];
    const T bn_next = slot[5 * NT];
    b0[0] = T(0.5) * (bn_cur + bn_next);
    b0[1] = T(0.5) * (slot[6 * NT] + slot[7 * NT]);
    b0[2] = T(0.5) * (slot[8 * NT] + slot[9 * NT]);
    bn_cur = bn_next;
    T un[5], bo[3];
    if (P.push(k, u0, b0, gamma, dth, hd, un, bo)) {
      const int ia = j - 3;
      if (active) {
        const long long co = base + (long long)ia * sA;
        out.f[0][co] = un[0];
        out.f[1 + A][co] = un[1];
        out.f[1 + T1][co] = un[2];
        out.f[1 + T2][co] = un[3];
        out.f[4][co] = un[4];
        if (!(un[0] > T(0))) P.st |= ST_UNPHYSICAL;
        if (LAST) {
          const T v = cell_cmax<T, PM>(un[0], un[1], un[2], un[3], un[4], bo[0], bo[1], bo[2],
                                        gamma, &P.st);
          if (v != v) nan_seen = true; else cm = fmax(cm, v);
        }
      }
    }
  }
  cp_async_wait<0>();
  if (LAST) block_max_to_global(cm, nan_seen, ds);
  if (active && P.st) atomicOr(&ds->status, P.st);
}

// 16-byte staging (FP32, nz a multiple of 4).  Each warp stages its own 32 pencils: 8 groups
// of 4 consecutive z positions, which never straddle a z row and start on a 16-byte
// boundary.  Per cell along the sweep the warp needs 9 rows of 32 values (u, B_n one cell
// ahead, B_t1, B_t2, and the B across the other transverse axis O one row up); lane l copies
// group l % 8 of rows l / 8 and 4 + l / 8 (lanes 0-7 also row 8) with one 16-byte cp.async
// each: about 2.3 copies and addresses per thread and cell instead of 10.  The z + 1
// neighbour of B_z is the next lane's B_z, except for lane 31 and at the end of a z row
// (wrapped or clamped), where the thread copies it itself into row 9.  Lanes read each
// other's copies after their own cp.async wait and a warp barrier; no block barrier, so
// warps march independently as in the per-element staging.
constexpr int kVecRows = 10;

// 16-byte copies allocate in L1 (.ca, MHD_STAGE_L1 = 1: neighbouring warps' halo rows hit
// there) or go through L2 only (.cg, 0)
#ifndef MHD_STAGE_L1
#define MHD_STAGE_L1 0
#endif
__device__ __forceinline__ void cp_async_16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
#if MHD_STAGE_L1
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
#else
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
#endif
}

template <int A, bool LAST, int PM, int S, int NT, bool OFF32 = false>
__device__ __forceinline__ void fluid_march_xy_tile_vec(const GridDesc& g, const FieldSet<float>& in,
                                                        const FieldSet<float>& out, float gamma,
                                                        double h, DevScalars* ds, unsigned bx,
                                                        unsigned by, unsigned char* smem_raw) {
  using AD = FieldAddr<float, OFF32>;
  static_assert(A == 0 || A == 1, "x or y sweep");
  static_assert(NT % 32 == 0, "whole warps");
  using T = float;
  constexpr int O = (A == 0) ? 1 : 0;       // the transverse axis that is not z
  constexpr int T1 = axis_t1(A), T2 = axis_t2(A);
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int nz = g.n[2], nO = g.n[O];
  const long long ntr = (long long)nz * nO;  // pencils of the transverse plane
  const long long p = (long long)bx * NT + tid;
  const bool active = p < ntr;
  const int z = (int)(p % nz);
  const int o = active ? (int)(p / nz) : nO - 1;
  const int a0 = by * S;
  const int nA = g.n[A], bcA = g.bc[A];
  const T dth = step_factor<T>(ds, h) * T(FluxScale<T>::inv);
  const T hd = T(0.5) * dth;
  const long long sA = g.s[A], sO = g.s[O];
  // this lane's copies: group q of rows r and r + 4 (and of row 8 for lanes 0-7)
  const int q = lane & 7, r = lane >> 3;
  const long long pq = (long long)bx * NT + 32 * w + 4 * q;
  const bool gq = pq < ntr;
  const int zq = (int)(pq % nz), oq = gq ? (int)(pq / nz) : 0;
  const long long tq = (long long)zq + (long long)oq * sO;
  const long long tq8 = (long long)zq + (long long)wrap_index(oq + 1, nO, g.bc[O]) * sO;
  // rows 0-3: rho, m_A, m_T1, m_T2; rows 4-7: E, B_A (one cell ahead), B_T1, B_T2; row 8:
  // the B across O, one O row up
  const float* src0 = (r == 0 ? in.f[0] : r == 1 ? in.f[1 + A] : r == 2 ? in.f[1 + T1]
                                                                         : in.f[1 + T2]) + tq;
  const float* src1 = (r == 0 ? in.f[4] : r == 1 ? in.f[5 + A] : r == 2 ? in.f[5 + T1]
                                                                         : in.f[5 + T2]) + tq;
  const float* src2 = in.f[5 + (A == 0 ? T1 : T2)] + tq8;
  // the z + 1 neighbour of B_z that the next lane does not hold
  const bool special = active && (lane == 31 || z == nz - 1);
  const float* srcs = in.f[7] + (long long)wrap_index(z + 1, nz, g.bc[2]) + (long long)o * sO;
  constexpr int RS = kVecRows * 32;          // floats per ring slot of a warp
  float* ring = reinterpret_cast<float*>(smem_raw) + (size_t)w * kMarchRing * RS;
  const int js = a0 - 3;
  const int kend = min(S, nA - a0) + 6;
  // offsets of the next row to stage (an) and of the row after it (B_A, one cell ahead):
  // rows advance by sA and take the wrap of the axis only where they cross its ends
  int an = js;
  long long offc = (long long)wrap_index(an, nA, bcA) * sA;
  long long offn = (long long)wrap_index(an + 1, nA, bcA) * sA;
  auto issue = [&](int kk) {
    if (kk < kend) {
      float* slot = ring + (size_t)((unsigned)kk % kMarchRing) * RS + 4 * q;
      if (gq) {
        const long long off1 = r == 1 ? offn : offc;
        cp_async_16(slot + r * 32, src0 + offc);
        cp_async_16(slot + (4 + r) * 32, src1 + off1);
        if (lane < 8) cp_async_16(slot + 8 * 32, src2 + offc);
      }
      if (special) cp_async_elem(ring + (size_t)((unsigned)kk % kMarchRing) * RS + 9 * 32 + lane, srcs + offc);
      offc = offn;
      ++an;
      if ((unsigned)an < (unsigned)(nA - 1)) offn += sA;   // an and an + 1 inside the axis
      else offn = (long long)wrap_index(an + 1, nA, bcA) * sA;
    }
    cp_async_commit();
  };
#pragma unroll
  for (int d = 0; d < kMarchDepth; ++d) issue(d);
  FluidPencil<T, PM, LAST> P;
  P.init();
  const long long base = (long long)z + (long long)o * sO;
  T bn_cur = in.f[5 + A][base + wrap_off<T>(js, nA, bcA, sA)];
  T cm = T(0);
  bool nan_seen = false;
  constexpr int ZROW = (A == 0) ? 7 : 6;     // the row holding B_z (B_t2 for x, B_t1 for y)
  const int nb_idx = special ? 9 * 32 + lane : ZROW * 32 + lane + 1;
  // output offset of iteration k (cell j - 3 = a0 - 6 + k; used from k = 6 on, inside the
  // tile), advanced by one row per iteration
  typename AD::I co = AD::of(base + (long long)(a0 - 6) * sA);
  const typename AD::I dco = AD::of(sA);
#pragma unroll kFluidUnroll
  for (int k = 0; k < kend; ++k, co += dco) {
    cp_async_wait<kMarchDepth - 1>();
    __syncwarp();
    issue(k + kMarchDepth);
    const float* slot = ring + (size_t)((unsigned)k % kMarchRing) * RS;
    T u0[5], b0[3];
#pragma unroll
    for (int c = 0; c < 5; ++c) u0[c] = slot[c * 32 + lane];
    const T bn_next = slot[5 * 32 + lane];
    const T zb_nb = slot[nb_idx];
    const T ob_nb = slot[8 * 32 + lane];
    b0[0] = T(0.5) * (bn_cur + bn_next);
    b0[1] = T(0.5) * (slot[6 * 32 + lane] + (A == 0 ? ob_nb : zb_nb));
    b0[2] = T(0.5) * (slot[7 * 32 + lane] + (A == 0 ? zb_nb : ob_nb));
    bn_cur = bn_next;
    T un[5], bo[3];
    if (P.push(k, u0, b0, gamma, dth, hd, un, bo)) {
      if (active) {
        *AD::at(out.f[0], co) = un[0];
        *AD::at(out.f[1 + A], co) = un[1];
        *AD::at(out.f[1 + T1], co) = un[2];
        *AD::at(out.f[1 + T2], co) = un[3];
        *AD::at(out.f[4], co) = un[4];
        if (!(un[0] > T(0))) P.st |= ST_UNPHYSICAL;
        if (LAST) {
          const T v = cell_cmax<T, PM>(un[0], un[1], un[2], un[3], un[4], bo[0], bo[1], bo[2],
                                        gamma, &P.st);
          if (v != v) nan_seen = true; else cm = fmax(cm, v);
        }
      }
    }
  }
  cp_async_wait<0>();
  if (LAST) block_max_to_global(cm, nan_seen, ds);
  if (active && P.st) atomicOr(&ds->status, P.st);
}

// FP32 grids whose z extent is a multiple of 4 take the 16-byte staging, others the
// per-element one; both feed the same arithmetic in the same order (identical results)
template <typename T>
__host__ __device__ inline bool march_vec(const GridDesc& g) {
  return sizeof(T) == 4 && g.n[2] % 4 == 0;
}
template <typename T>
static size_t march_tile_smem(int nt = 128) {
  return sizeof(T) * (size_t)kMarchRing * kVecRows * nt;    // both stagings: 10 values per cell
}

template <typename T, int A, bool LAST, int PM, int S, int NT>
__device__ __forceinline__ void fluid_march_xy_tile(const GridDesc& g, const FieldSet<T>& in,
                                                    const FieldSet<T>& out, T gamma, double h,
                                                    DevScalars* ds, unsigned bx, unsigned by,
                                                    unsigned char* smem_raw) {
  if constexpr (sizeof(T) == 4) {
    if (march_vec<T>(g)) {
      fluid_march_xy_tile_vec<A, LAST, PM, S, NT>(g, in, out, gamma, h, ds, bx, by, smem_raw);
      return;
    }
  }
  fluid_march_xy_tile_elem<T, A, LAST, PM, S, NT>(g, in, out, gamma, h, ds, bx, by, smem_raw);
}

template <typename T, int A, bool LAST, int PM, int S, int NT>
__global__ void __launch_bounds__(NT, MHD_MARCH_MINB)
fluid_march_xy(GridDesc g, FieldSet<T> in, FieldSet<T> out, T gamma, double h, DevScalars* ds) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  fluid_march_xy_tile_elem<T, A, LAST, PM, S, NT>(g, in, out, gamma, h, ds, blockIdx.x,
                                                   blockIdx.y, smem_raw);
}

// the 16-byte staging as a kernel of its own (its register allocation does not carry the
// per-element path's); MHD_VEC_MINB resident blocks per SM asked of the compiler
#ifndef MHD_VEC_MINB
#define MHD_VEC_MINB 4
#endif
template <int A, bool LAST, int PM, int S, int NT, bool OFF32 = false>
__global__ void __launch_bounds__(NT, MHD_VEC_MINB)
fluid_march_xy_vec(GridDesc g, FieldSet<float> in, FieldSet<float> out, float gamma, double h,
                   DevScalars* ds) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  fluid_march_xy_tile_vec<A, LAST, PM, S, NT, OFF32>(g, in, out, gamma, h, ds, blockIdx.x,
                                                      blockIdx.y, smem_raw);
}

}  // namespace mhd

namespace mhd {

// ------------------------------------------------------------------------------------
// Marching constrained transport (Algorithm 2; Eqs. "eq:averaging_x", "eq:first_flux").
// One EMF pipeline follows one pencil of a transverse face component B_t along the sweep.
// The (1,2,1) smoothing adds the two outer face velocities first: the smoothed velocity is
// then exactly odd under a reflection of the sweep axis, so the edge velocity on a mirror
// face is exactly 0 in every precision and the upwind rule of Eq. "eq:first_flux" (0 takes
// the right cell) decides it the same way in FP32 as in FP64.
// Pushing cell j (face velocity vf(j) across the t-face and B_t(j)) yields, 4 cells
// behind, the advected B_t(j-4) and the limited EMF at the A-face (j-4)+1/2; the EMF at
// (j-5)+1/2 (the previous one) is what the constraint on B_A(j-4) uses.
// Operation order matches the oracle expression by expression.
// ------------------------------------------------------------------------------------
template <typename T>
struct EmfPipe {
  T vf1, vf2;          // vf(j-1), vf(j-2)
  T vs1, vs2, vs3;     // vs(j-2), vs(j-3), vs(j-4)
  T b1, b2, b3, b4;    // B_t(j-1), B_t(j-2), B_t(j-3), B_t(j-4)
  T e1p;               // first-order EMF at (j-3)+1/2
  T g3, g4;            // g(j-3), g(j-4)  (g = vs * B_t at t + dt/2)
  T dp;                // g(j-3) - g(j-4)
  T pp;                // phi(g(j-4) - g(j-5), g(j-3) - g(j-4)) / 2
  T e2p;               // limited EMF at (j-5)+1/2

  __device__ __forceinline__ void init() {
    vf1 = vf2 = vs1 = vs2 = vs3 = b1 = b2 = b3 = b4 = e1p = g3 = g4 = dp = pp = e2p = T(0);
  }

  // returns the advected B_t(j-4); e2_prev receives the EMF at (j-5)+1/2
  __device__ __forceinline__ T push(T vf0, T b0, T dth, T hd, T* e2_prev) {
    const T vs0 = T(0.25) * ((vf0 + vf2) + T(2) * vf1);         // vs(j-1)
    const T ve1 = T(0.5) * (vs1 + vs0);                           // edge velocity (j-2)+1/2
    const T e1 = ve1 > T(0) ? vs1 * b2 : vs0 * b1;               // first-order EMF (j-2)+1/2
    const T bh = b2 - hd * (e1 - e1p);                            // B_t(j-2) at t + dt/2
    const T g2 = vs1 * bh;                                        // g(j-2)
    const T dn = g2 - g3;                                         // g(j-2) - g(j-3)
    const T pn = half_vanleer(dp, dn);                            // phi/2 at (j-3)
    const T ve4 = T(0.5) * (vs3 + vs2);                           // edge velocity (j-4)+1/2
    const T e2 = ve4 > T(0) ? g4 + pp : g3 - pn;
    const T bt = b4 - dth * (e2 - e2p);                           // advected B_t(j-4)
    *e2_prev = e2p;
    // shift
    vf2 = vf1; vf1 = vf0;
    vs3 = vs2; vs2 = vs1; vs1 = vs0;
    b4 = b3; b3 = b2; b2 = b1; b1 = b0;
    e1p = e1;
    g4 = g3; g3 = g2;
    dp = dn;
    pp = pn;
    e2p = e2;
    return bt;
  }
};

// Packed FP32 arithmetic on float pairs (f32x2 instructions of sm_100+): two independent
// EMF pipelines advance in one instruction stream, lane x and lane y.
#ifndef MHD_CT_PACK
#define MHD_CT_PACK 1
#endif
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  float2 d;
  asm("{.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\t"
      "mov.b64 rb, {%4, %5};\n\t"
      "sub.rn.f32x2 rd, ra, rb;\n\t"
      "mov.b64 {%0, %1}, rd;}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 splat2(float v) { return make_float2(v, v); }
// lane-wise c > 0 ? a : b
__device__ __forceinline__ float2 sel_pos2(float2 c, float2 a, float2 b) {
  return make_float2(c.x > 0.f ? a.x : b.x, c.y > 0.f ? a.y : b.y);
}
// lane-wise phi(a, b) / 2 (half_vanleer<float>)
__device__ __forceinline__ float2 half_vanleer2(float2 a, float2 b) {
  const float2 ab = mul2(a, b), s = add2(a, b);
  const float2 q = mul2(ab, make_float2(__fdividef(1.f, s.x), __fdividef(1.f, s.y)));
  return make_float2(ab.x > 0.f ? q.x : 0.f, ab.y > 0.f ? q.y : 0.f);
}

// Two EmfPipe<float> in one: lane x and lane y are independent pipelines (same steps), with
// the smoothed velocity kept as 4 vs (the (1,2,1) sum without its 1/4), so that g and every
// EMF come out 4x EmfPipe's; ndth and nhd come divided by kEmf2Scale, and the edge velocity's
// sign is that of vs(j) + vs(j+1).  The scales are powers of two, so they change the
// rounding of none of the packed operations.
constexpr float kEmf2Scale = 4.f, kEmf2Inv = 0.25f;
struct EmfPipe2 {
  float2 vf1, vf2, vs1, vs2, vs3, b1, b2, b3, b4, e1p, g3, g4, dp, pp, e2p;

  __device__ __forceinline__ void init() {
    vf1 = vf2 = vs1 = vs2 = vs3 = b1 = b2 = b3 = b4 = e1p = g3 = g4 = dp = pp = e2p =
        make_float2(0.f, 0.f);
  }

  // ndth = -dt/(4h), nhd = -dt/(8h) in both lanes (dt/h and dt/(2h) over kEmf2Scale)
  __device__ __forceinline__ float2 push(float2 vf0, float2 b0, float2 ndth, float2 nhd,
                                         float2* e2_prev) {
    const float2 vs0 = fma2(splat2(2.f), vf1, add2(vf0, vf2));   // 4 vs(j-1)
    const float2 ve1 = add2(vs1, vs0);                            // 8 x edge velocity
    const float2 e1 = sel_pos2(ve1, mul2(vs1, b2), mul2(vs0, b1));
    const float2 bh = fma2(nhd, sub2(e1, e1p), b2);
    const float2 g2 = mul2(vs1, bh);
    const float2 dn = sub2(g2, g3);
    const float2 pn = half_vanleer2(dp, dn);
    const float2 ve4 = add2(vs3, vs2);
    const float2 e2 = sel_pos2(ve4, add2(g4, pp), sub2(g3, pn));
    const float2 bt = fma2(ndth, sub2(e2, e2p), b4);
    *e2_prev = e2p;
    vf2 = vf1; vf1 = vf0;
    vs3 = vs2; vs2 = vs1; vs1 = vs0;
    b4 = b3; b3 = b2; b2 = b1; b1 = b0;
    e1p = e1;
    g4 = g3; g3 = g2;
    dp = dn;
    pp = pn;
    e2p = e2;
    return bt;
  }
};

// Offsets of the four cells a thread needs across one transverse axis t: the row itself
// (own), its lower neighbour (the across-face cell of its EMF row), its upper neighbour
// (the row whose EMF enters the constraint) and that row's across-face cell, which is
// always either the own cell or the lower neighbour (wrap or clamp).
struct TransverseOffsets {
  long long lo, hi;      // offsets of the lower and upper neighbour rows
  bool hi_across_lo;     // the upper row's across-face cell is the lower neighbour
};

__device__ __forceinline__ TransverseOffsets transverse_offsets(int c, int n, int bc,
                                                               long long stride) {
  TransverseOffsets t;
  const int lo = wrap_index(c - 1, n, bc), hi = wrap_index(c + 1, n, bc);
  const int hi_across = wrap_index(hi - 1, n, bc);
  t.lo = (long long)(lo - c) * stride;
  t.hi = (long long)(hi - c) * stride;
  t.hi_across_lo = (hi_across != c);
  return t;
}

template <typename T>
struct CtColumn {
  static constexpr bool PACK = MHD_CT_PACK && sizeof(T) == 4;
  EmfPipe<T> own1, nb1, own2, nb2;
  EmfPipe2 ownp, nbp;     // FP32: (own1, own2) and (nb1, nb2) as packed pairs
  T ba1, ba2, ba3, ba4;   // B_A(j-1..j-4)

  __device__ __forceinline__ void init() {
    own1.init(); nb1.init(); own2.init(); nb2.init();
    ownp.init(); nbp.init();
    ba1 = ba2 = ba3 = ba4 = T(0);
  }

  // r[5], m[5]: rho and m_A at (own, lo1, hi1, lo2, hi2); b1o/b1h: B_t1 at own/hi1 row,
  // b2o/b2h: B_t2 at own/hi2 row; ba: B_A(j).  Outputs for cell j-4.
  __device__ __forceinline__ void push(const T r[5], const T m[5], T b1o, T b1h, T b2o, T b2h,
                                       T ba, bool hx1, bool hx2, T dth, T hd, T* bt1, T* bt2,
                                       T* bA) {
    // the upper row's face velocity: across its lower face, the own cell, or (outflow upper
    // edge) the lower neighbour; the operands are chosen first, one quotient each
    const T mx1 = hx1 ? m[1] : m[0], rx1 = hx1 ? r[1] : r[0];
    const T mx2 = hx2 ? m[3] : m[0], rx2 = hx2 ? r[3] : r[0];
    const T vo1 = Num<T>::div(m[0] + m[1], r[0] + r[1]);
    const T vn1 = Num<T>::div(m[2] + mx1, r[2] + rx1);
    const T vo2 = Num<T>::div(m[0] + m[3], r[0] + r[3]);
    const T vn2 = Num<T>::div(m[4] + mx2, r[4] + rx2);
    T eo1, en1, eo2, en2;
    if constexpr (PACK) {
      const float2 ndth = splat2(-(float)dth * kEmf2Inv), nhd = splat2(-(float)hd * kEmf2Inv);
      float2 eo, en;
      const float2 bt = ownp.push(make_float2((float)vo1, (float)vo2),
                                  make_float2((float)b1o, (float)b2o), ndth, nhd, &eo);
      nbp.push(make_float2((float)vn1, (float)vn2), make_float2((float)b1h, (float)b2h), ndth,
               nhd, &en);
      *bt1 = bt.x; *bt2 = bt.y;
      eo1 = eo.x; eo2 = eo.y; en1 = en.x; en2 = en.y;
    } else {
      *bt1 = own1.push(vo1, b1o, dth, hd, &eo1);
      nb1.push(vn1, b1h, dth, hd, &en1);
      *bt2 = own2.push(vo2, b2o, dth, hd, &eo2);
      nb2.push(vn2, b2h, dth, hd, &en2);
    }
    const T dc = PACK ? dth * T(kEmf2Inv) : dth;   // the packed EMFs are kEmf2Scale x
    T b = ffma(dc, en1 - eo1, ba4);          // constraint from t1, then t2
    b = ffma(dc, en2 - eo2, b);
    *bA = b;
    ba4 = ba3; ba3 = ba2; ba2 = ba1; ba1 = ba;
  }
};

// x or y sweep of the constrained transport; thread layout as fluid_march_xy
template <typename T, int A, int S, int NT>
__device__ __forceinline__ void ct_march_xy_tile(const GridDesc& g, const FieldSet<T>& in,
                                                 const FieldSet<T>& out, double h, DevScalars* ds,
                                                 unsigned bx, unsigned by, unsigned char* smem_raw) {
  static_assert(A == 0 || A == 1, "x or y sweep");
  constexpr int O = (A == 0) ? 1 : 0;
  constexpr int T1 = axis_t1(A), T2 = axis_t2(A);
  const long long p = (long long)bx * NT + threadIdx.x;
  const int z = (int)(p % g.n[2]);
  const long long o_ = p / g.n[2];
  const int oc = (int)(o_ < g.n[O] ? o_ : g.n[O] - 1);
  const int a0 = by * S;
  const int nA = g.n[A], bcA = g.bc[A];
  const bool active = o_ < g.n[O];
  const T dth = (T)(ds->dt / h);   // step_factor's value; a division once per tile here
  const T hd = T(0.5) * dth;
  const long long base = (long long)z + (long long)oc * g.s[O];
  const int c1 = (T1 == 2) ? z : oc, c2 = (T2 == 2) ? z : oc;
  const TransverseOffsets o1 = transverse_offsets(c1, g.n[T1], g.bc[T1], g.s[T1]);
  const TransverseOffsets o2 = transverse_offsets(c2, g.n[T2], g.bc[T2], g.s[T2]);
  const T* __restrict__ pr = in.f[0];
  const T* __restrict__ pm = in.f[1 + A];
  const T* __restrict__ pb1 = in.f[5 + T1];
  const T* __restrict__ pb2 = in.f[5 + T2];
  const T* __restrict__ pba = in.f[5 + A];
  const long long sA = g.s[A];
  CtColumn<T> col;
  col.init();
  const int js = a0 - 4;
  const int kend = min(S, nA - a0) + 8;
  T* ring = reinterpret_cast<T*>(smem_raw);
  constexpr int NV = 15;
  RowCursor rc(js, nA, bcA, sA);
  auto issue = [&](int kk) {
    if (kk < kend) {
      const long long c = base + rc.off;
      rc.advance();
      T* slot = ring + (size_t)((unsigned)kk % kMarchRing) * NV * NT + threadIdx.x;
      cp_async_elem(slot + 0 * NT, pr + c);
      cp_async_elem(slot + 1 * NT, pr + c + o1.lo);
      cp_async_elem(slot + 2 * NT, pr + c + o1.hi);
      cp_async_elem(slot + 3 * NT, pr + c + o2.lo);
      cp_async_elem(slot + 4 * NT, pr + c + o2.hi);
      cp_async_elem(slot + 5 * NT, pm + c);
      cp_async_elem(slot + 6 * NT, pm + c + o1.lo);
      cp_async_elem(slot + 7 * NT, pm + c + o1.hi);
      cp_async_elem(slot + 8 * NT, pm + c + o2.lo);
      cp_async_elem(slot + 9 * NT, pm + c + o2.hi);
      cp_async_elem(slot + 10 * NT, pb1 + c);
      cp_async_elem(slot + 11 * NT, pb1 + c + o1.hi);
      cp_async_elem(slot + 12 * NT, pb2 + c);
      cp_async_elem(slot + 13 * NT, pb2 + c + o2.hi);
      cp_async_elem(slot + 14 * NT, pba + c);
    }
    cp_async_commit();
  };
#pragma unroll
  for (int d = 0; d < kMarchDepth; ++d) issue(d);
  int st = 0;
#pragma unroll kCtUnroll
  for (int k = 0; k < kend; ++k) {
    issue(k + kMarchDepth);
    cp_async_wait<kMarchDepth>();
    const T* slot = ring + (size_t)((unsigned)k % kMarchRing) * NV * NT + threadIdx.x;
    const int j = js + k;
    T r[5], m[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      r[q] = slot[q * NT];
      m[q] = slot[(5 + q) * NT];
    }
    T bt1, bt2, bA;
    col.push(r, m, slot[10 * NT], slot[11 * NT], slot[12 * NT], slot[13 * NT], slot[14 * NT],
             o1.hi_across_lo, o2.hi_across_lo, dth, hd, &bt1, &bt2, &bA);
    if (k >= 8 && active) {
      const long long co = base + (long long)(j - 4) * sA;
      out.f[5 + T1][co] = bt1;
      out.f[5 + T2][co] = bt2;
      out.f[5 + A][co] = bA;
      if (!(bt1 == bt1) || !(bt2 == bt2) || !(bA == bA)) st |= ST_NONFINITE;
    }
  }
  cp_async_wait<0>();
  if (active && st) atomicOr(&ds->status, st);
}

template <typename T, int A, int S, int NT>
__global__ void __launch_bounds__(NT, MHD_CT_MINB)
ct_march_xy(GridDesc g, FieldSet<T> in, FieldSet<T> out, double h, DevScalars* ds) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ct_march_xy_tile<T, A, S, NT>(g, in, out, h, ds, blockIdx.x, blockIdx.y, smem_raw);
}

// ------------------------------------------------------------------------------------
// x or y sweep of the constrained transport with every EMF row evaluated once.
//
// A block holds R warps; warp w follows transverse row o0 + w of the axis O (the
// transverse axis that is not z), lane l the pencil z0 + l; both coordinates are wrapped
// or clamped at the grid's edges like any neighbour index.  Each thread runs the EMF
// pipelines of its own pencil for t1 and t2.  The constraint on B_A (Algorithm 2) needs, for
// each transverse axis, the EMF of the row above as well: across z that is lane l+1's
// (warp shuffle), across O it is warp w+1's (shared memory, one barrier per cell).  So
// lane 31 and warp R-1 only supply EMFs to their neighbours, and a block updates 31 x (R-1)
// pencils.  Where the row above is clamped onto the row itself (outflow top edge), the
// neighbour's pipeline sees the same inputs as the thread's own, which is what the
// per-thread form (ct_march_xy) computes there too.  Results are identical to ct_march_xy.
// ------------------------------------------------------------------------------------
// the EMF exchange of the shared-row CT synchronises row pairs with named barriers instead
// of the whole block (1), or uses the block barrier (0)
#ifndef MHD_CT_PAIR_BARRIERS
#define MHD_CT_PAIR_BARRIERS 1
#endif
// the shared-row form pays off when a z chunk of 31 pencils and several rows are filled
constexpr int kRowsMinNz = 48, kRowsMinRows = 4;
__host__ __device__ inline bool ct_use_rows(const GridDesc& g, int axis) {
  return axis < 2 && g.n[2] >= kRowsMinNz && g.n[axis == 0 ? 1 : 0] >= kRowsMinRows;
}

// PASSES = 2: the CT along A applied twice with the same dt in one march (the pair of CT
// operators in the middle of a step whose axis order ends with A, Eq. "eq:L_sequence"), for a
// periodic axis A.  A second pair of pipelines runs 4 cells behind the first, fed with the
// first pass's advected B_t and the same face velocities (the fluid is frozen); its EMFs are
// exchanged with the first pass's at the same barriers, and its constraint adds to the first
// pass's B_A.  Each cell gets the operations of two single passes in the same order (the same
// bits); the tile's halo along A doubles to 8 cells.
template <typename T, int A, int S, int R, int PASSES = 1>
__device__ __forceinline__ void ct_rows_xy_tile(const GridDesc& g, const FieldSet<T>& in,
                                                const FieldSet<T>& out, double h, DevScalars* ds,
                                                unsigned bx, unsigned by,
                                                unsigned char* smem_raw) {
  static_assert(PASSES == 1 || PASSES == 2, "one or two passes");
  static_assert(A == 0 || A == 1, "x or y sweep");
  constexpr int O = (A == 0) ? 1 : 0;
  constexpr int T1 = axis_t1(A), T2 = axis_t2(A);
  constexpr int NT = 32 * R;
  constexpr bool Z1 = (T1 == 2);             // the t1 pipeline runs across z (y sweep)
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nzc = (g.n[2] + 30) / 31;
  const int z0 = (int)(bx % nzc) * 31;
  const int zr = z0 + lane;
  const int orow = (int)(bx / nzc) * (R - 1) + w;
  const int zc = wrap_index(zr, g.n[2], g.bc[2]);
  const int oc = wrap_index(orow, g.n[O], g.bc[O]);
  const bool out_ok = lane < 31 && zr < g.n[2] && w < R - 1 && orow < g.n[O];
  const bool halo_row = (w == R - 1);        // supplies the O-row EMF only
  const int a0 = by * S;
  const int nA = g.n[A], bcA = g.bc[A];
  const T dth = (T)(ds->dt / h);   // step_factor's value; a division once per tile here
  const T hd = T(0.5) * dth;
  const long long base = (long long)zc + (long long)oc * g.s[O];
  const int oc_lo = wrap_index(oc - 1, g.n[O], g.bc[O]);
  const long long lo_z = (long long)(wrap_index(zc - 1, g.n[2], g.bc[2]) - zc);
  const long long lo_o = (long long)(oc_lo - oc) * g.s[O];
  const long long lo1 = Z1 ? lo_z : lo_o, lo2 = Z1 ? lo_o : lo_z;
  const T* __restrict__ pr = in.f[0];
  const T* __restrict__ pm = in.f[1 + A];
  const T* __restrict__ pb1 = in.f[5 + T1];
  const T* __restrict__ pb2 = in.f[5 + T2];
  const T* __restrict__ pba = in.f[5 + A];
  const long long sA = g.s[A];
  constexpr bool PACK = MHD_CT_PACK && sizeof(T) == 4;
  EmfPipe<T> p1, p2, q1, q2;                 // q: the second pass (PASSES = 2)
  EmfPipe2 pp2, qq2;
  p1.init();
  p2.init();
  pp2.init();
  q1.init();
  q2.init();
  qq2.init();
  const float2 ndth2 = splat2(-(float)dth * kEmf2Inv), nhd2 = splat2(-(float)hd * kEmf2Inv);
  const T dc = PACK ? dth * T(kEmf2Inv) : dth;   // constraint factor for the EMFs' scale
  T ba1 = T(0), ba2 = T(0), ba3 = T(0), ba4 = T(0);
  // the second pass: face velocities of the last 4 cells, first-pass B_A of the last 4
  T wv1[4] = {T(0), T(0), T(0), T(0)}, wv2[4] = {T(0), T(0), T(0), T(0)};
  T wb1 = T(0), wb2 = T(0), wb3 = T(0), wb4 = T(0);
  constexpr int H = 4 * PASSES;              // halo along A
  const int js = a0 - H;
  const int kend = min(S, nA - a0) + 2 * H;
  T* ring = reinterpret_cast<T*>(smem_raw);
  T* xbuf = ring + (size_t)kMarchRing * 9 * NT;   // [2][PASSES][NT] EMF of the O pipelines
  int st = 0;
  // the pipelines of one pass for one cell: face velocities vf1, vf2 and B_t in; the
  // advected B_t (4 cells behind) and the EMFs at its lower A face out
  auto pipes = [&](EmfPipe<T>& a1, EmfPipe<T>& a2, EmfPipe2& aa, T vf1, T vf2, T b1in,
                   T b2in, T& bt1, T& bt2, T& e1, T& e2) {
    if constexpr (PACK) {
      float2 e12;
      const float2 bt = aa.push(make_float2((float)vf1, (float)vf2),
                                make_float2((float)b1in, (float)b2in), ndth2, nhd2, &e12);
      bt1 = bt.x; bt2 = bt.y; e1 = e12.x; e2 = e12.y;
    } else {
      // the halo row only feeds the O pipeline's EMF to the row below
      if (!halo_row || !Z1) bt1 = a1.push(vf1, b1in, dth, hd, &e1);
      if (!halo_row || Z1) bt2 = a2.push(vf2, b2in, dth, hd, &e2);
    }
  };
  // one cell of the march: face velocities, the EMF pipelines, the EMF exchange and the
  // constraint on B_A; r = rho (own, lo1, lo2), m = m_A (same), b1, b2, ba the face fields
  auto cell = [&](int k, T r0, T r1, T r2, T m0, T m1, T m2, T b1in, T b2in, T bain) {
    const int j = js + k;
    const T vf1 = Num<T>::div(m0 + m1, r0 + r1);     // face velocities below the pencil
    const T vf2 = Num<T>::div(m0 + m2, r0 + r2);
    T bt1 = T(0), bt2 = T(0), e1 = T(0), e2 = T(0);
    pipes(p1, p2, pp2, vf1, vf2, b1in, b2in, bt1, bt2, e1, e2);
    // second pass, 4 cells behind: first-pass B_t of cell j-4 with its face velocities
    T ct1 = T(0), ct2 = T(0), f1 = T(0), f2 = T(0);
    if constexpr (PASSES == 2) pipes(q1, q2, qq2, wv1[3], wv2[3], bt1, bt2, ct1, ct2, f1, f2);
    T* xb = xbuf + (k & 1) * PASSES * NT;
    xb[threadIdx.x] = Z1 ? e2 : e1;                  // EMF of the O pipeline
    if constexpr (PASSES == 2) xb[NT + threadIdx.x] = Z1 ? f2 : f1;
#if MHD_CT_PAIR_BARRIERS
    // warp w hands its value to warp w-1 (barrier w) and takes warp w+1's (barrier w+1):
    // each named barrier joins just the two warps of one row pair (64 threads)
    if (w > 0) asm volatile("bar.sync %0, 64;" ::"r"(w) : "memory");
    if (w < R - 1) asm volatile("bar.sync %0, 64;" ::"r"(w + 1) : "memory");
#else
    __syncthreads();
#endif
    const int up = halo_row ? threadIdx.x : threadIdx.x + 32;
    const T eo_up = xb[up];
    const T ez_up = __shfl_down_sync(0xffffffffu, Z1 ? e1 : e2, 1);
    const T en1 = Z1 ? ez_up : eo_up, en2 = Z1 ? eo_up : ez_up;
    T b = ffma(dc, en1 - e1, ba4);           // constraint from t1, then t2
    b = ffma(dc, en2 - e2, b);
    ba4 = ba3; ba3 = ba2; ba2 = ba1; ba1 = bain;
    if constexpr (PASSES == 2) {
      const T fo_up = xb[NT + up];
      const T fz_up = __shfl_down_sync(0xffffffffu, Z1 ? f1 : f2, 1);
      const T fn1 = Z1 ? fz_up : fo_up, fn2 = Z1 ? fo_up : fz_up;
      T b2 = ffma(dc, fn1 - f1, wb4);        // the second pass's constraint on cell j-8
      b2 = ffma(dc, fn2 - f2, b2);
      wb4 = wb3; wb3 = wb2; wb2 = wb1; wb1 = b;
      wv1[3] = wv1[2]; wv1[2] = wv1[1]; wv1[1] = wv1[0]; wv1[0] = vf1;
      wv2[3] = wv2[2]; wv2[2] = wv2[1]; wv2[1] = wv2[0]; wv2[0] = vf2;
      if (k >= 2 * H && out_ok) {
        const long long co = base + (long long)(j - 8) * sA;
        out.f[5 + T1][co] = ct1;
        out.f[5 + T2][co] = ct2;
        out.f[5 + A][co] = b2;
        if (!(ct1 == ct1) || !(ct2 == ct2) || !(b2 == b2)) st |= ST_NONFINITE;
      }
    } else if (k >= 8 && out_ok) {
      const long long co = base + (long long)(j - 4) * sA;
      out.f[5 + T1][co] = bt1;
      out.f[5 + T2][co] = bt2;
      out.f[5 + A][co] = b;
      if (!(bt1 == bt1) || !(bt2 == bt2) || !(b == b)) st |= ST_NONFINITE;
    }
  };
  // 16-byte staging (FP32, nz a multiple of 4, a z chunk that needs no wrap): each warp
  // copies, per cell, 7 rows of the 36 aligned z positions around its 32 pencils (rho, m_A
  // of its own row and of the row below across O, B_t1, B_t2, B_A), 9 groups of 4 each:
  // two 16-byte copies per lane instead of 9 single values; the z - 1 neighbours of rho and
  // m_A are the row's previous positions.  Lanes read each other's copies after their own
  // wait and a warp barrier.
  // staged z range [zb, zb + 36): aligned, holding z0 - 1 .. z0 + 31, inside the row
  const int zb = (z0 - 1) & ~3;
  bool vec = false;
  if constexpr (sizeof(T) == 4) vec = g.n[2] % 4 == 0 && z0 >= 1 && zb + 36 <= g.n[2];
  if (vec) {
    constexpr int VW = 36, VR = 7;           // values per row, rows per cell
    const int zo = z0 - zb;                  // this warp's first pencil in the row (1..4)
    float* wring = reinterpret_cast<float*>(smem_raw) + (size_t)w * kMarchRing * VR * VW;
    // this lane's copies: c = lane and lane + 32 of the 63 (row c / 9, group c % 9)
    const float* src[2];
    int dst[2];
    bool has[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int c = lane + 32 * q;
      has[q] = c < VR * 9;
      const int row = has[q] ? c / 9 : 0, grp = c % 9;
      const float* f = (const float*)(row == 0 || row == 2 ? in.f[0] : row == 1 || row == 3
                                      ? in.f[1 + A] : row == 4 ? in.f[5 + T1] : row == 5
                                      ? in.f[5 + T2] : in.f[5 + A]);
      const int orow_c = (row == 2 || row == 3) ? oc_lo : oc;
      src[q] = f + (long long)orow_c * g.s[O] + zb + 4 * grp;
      dst[q] = row * VW + 4 * grp;
    }
    RowCursor rc(js, nA, bcA, sA);
    auto issue = [&](int kk) {
      if (kk < kend) {
        const long long off = rc.off;
        rc.advance();
        float* slot = wring + (size_t)((unsigned)kk % kMarchRing) * VR * VW;
#pragma unroll
        for (int q = 0; q < 2; ++q)
          if (has[q]) cp_async_16(slot + dst[q], src[q] + off);
      }
      cp_async_commit();
    };
#pragma unroll
    for (int d = 0; d < kMarchDepth; ++d) issue(d);
    const int own = zo + lane, lz = own - 1;
    const int l1 = Z1 ? lz : 2 * VW + own, l2 = Z1 ? 2 * VW + own : lz;   // lo1, lo2 of rho
#pragma unroll kCtUnroll
    for (int k = 0; k < kend; ++k) {
      cp_async_wait<kMarchDepth - 1>();
      __syncwarp();
      issue(k + kMarchDepth);
      const float* sl = wring + (size_t)((unsigned)k % kMarchRing) * VR * VW;
      cell(k, (T)sl[own], (T)sl[l1], (T)sl[l2], (T)sl[VW + own], (T)sl[VW + l1],
           (T)sl[VW + l2], (T)sl[4 * VW + own], (T)sl[5 * VW + own], (T)sl[6 * VW + own]);
    }
  } else {
    constexpr int NV = 9;
    RowCursor rc(js, nA, bcA, sA);
    auto issue = [&](int kk) {
      if (kk < kend) {
        const long long c = base + rc.off;
        rc.advance();
        T* slot = ring + (size_t)((unsigned)kk % kMarchRing) * NV * NT + threadIdx.x;
        cp_async_elem(slot + 0 * NT, pr + c);
        cp_async_elem(slot + 1 * NT, pr + c + lo1);
        cp_async_elem(slot + 2 * NT, pr + c + lo2);
        cp_async_elem(slot + 3 * NT, pm + c);
        cp_async_elem(slot + 4 * NT, pm + c + lo1);
        cp_async_elem(slot + 5 * NT, pm + c + lo2);
        cp_async_elem(slot + 6 * NT, pb1 + c);
        cp_async_elem(slot + 7 * NT, pb2 + c);
        cp_async_elem(slot + 8 * NT, pba + c);
      }
      cp_async_commit();
    };
#pragma unroll
    for (int d = 0; d < kMarchDepth; ++d) issue(d);
#pragma unroll kCtUnroll
    for (int k = 0; k < kend; ++k) {
      issue(k + kMarchDepth);
      cp_async_wait<kMarchDepth>();
      const T* slot = ring + (size_t)((unsigned)k % kMarchRing) * NV * NT + threadIdx.x;
      cell(k, slot[0], slot[1 * NT], slot[2 * NT], slot[3 * NT], slot[4 * NT], slot[5 * NT],
           slot[6 * NT], slot[7 * NT], slot[8 * NT]);
    }
  }
  cp_async_wait<0>();
  if (st) atomicOr(&ds->status, st);
}

template <typename T>
static size_t ct_rows_smem(int R, int passes = 1) {
  return sizeof(T) * ((size_t)kMarchRing * 9 * 32 * R + 2 * (size_t)passes * 32 * R);
}

// resident blocks per SM asked of the compiler: for the two-pass form 2 (at most 128
// registers a thread) or, with 16 rows (512 threads), 1; MHD_ROWS1_MINB for the FP32 one-pass form (0: none; the compiler
// takes 88 registers, 2 blocks of 256 threads per SM; a cap at 3 blocks, 79 registers, was
// 5% slower at 512^3)
#ifndef MHD_ROWS1_MINB
#define MHD_ROWS1_MINB 0
#endif
template <typename T, int A, int S, int R, int PASSES = 1>
__global__ void __launch_bounds__(32 * R, PASSES == 2 ? (R >= 16 ? 1 : 2) : (sizeof(T) == 4 ? MHD_ROWS1_MINB : 0))
ct_rows_xy(GridDesc g, FieldSet<T> in, FieldSet<T> out, double h, DevScalars* ds) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ct_rows_xy_tile<T, A, S, R, PASSES>(g, in, out, h, ds, blockIdx.x, blockIdx.y, smem_raw);
}

}  // namespace mhd
