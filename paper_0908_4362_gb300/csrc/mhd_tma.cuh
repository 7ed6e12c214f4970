// x or y fluid sweep staged by the tensor memory accelerator (TMA, cp.async.bulk.tensor):
// FP32 grids whose z extent is a multiple of 128, so that a block's 128 pencils are 128
// consecutive z positions of one row of the other transverse axis O.
//
// Per cell along the sweep the block needs 9 rows of 128 values (u at j, B_A at j + 1, B_t1,
// B_t2, and the B across O one O row up).  The march is staged in groups of kTmaG cells: one
// thread issues, per group, one box of 128 x kTmaG values per row (9 boxes), or, where the
// group's cells wrap or clamp at the ends of the sweep axis, one 128-value box per cell and
// row at the mapped coordinate; the loads complete on the slot's "full" mbarrier, which the
// threads wait on before reading.  After a group every thread arrives on the slot's "empty"
// mbarrier, and the thread that refills the slot waits on that first.  The issuing thread
// rotates over the warps group by group.  The z + 1 neighbour of B_z is the next thread's
// value, except for the block's last thread and at the end of a z row, where the thread
// copies it itself (cp.async).  The arithmetic is FluidPencil's, in the same order as the
// other stagings (identical results).
//
// Every mbarrier wait is bounded: a wait that gives up sets ST_TIMEOUT in the context's
// status and the block stops issuing, so the launch ends instead of hanging.
#pragma once

#include <cuda.h>

#include "mhd_march.cuh"

// The x/y fluid sweeps take this staging where the context has tensor maps (1), or always
// the 16-byte cp.async staging (0, the default: measured faster at 512^3, 1.45 ms against
// 1.87 ms for the best ring shape here, kTmaG = 2, kTmaRing = 4, kTmaLag = 2)
#ifndef MHD_TMA_MARCH
#define MHD_TMA_MARCH 0
#endif

namespace mhd {

// the 9 staged rows' tensor maps (rho, m_A, m_T1, m_T2, E, B_A, B_T1, B_T2, B across O), with
// boxes of 128 x kTmaG cells (g) and of 128 x 1 (one)
#ifndef MHD_TMA_G
#define MHD_TMA_G 2
#endif
#ifndef MHD_TMA_RING
#define MHD_TMA_RING 4
#endif
#ifndef MHD_TMA_LAG
#define MHD_TMA_LAG 2
#endif
constexpr int kTmaG = MHD_TMA_G;
struct TmaRows {
  CUtensorMap g[9];
  CUtensorMap one[9];
};

// the tensor maps of a state's 8 input buffers, as the launcher receives them: boxes of
// 128 x 1 x 1, of 128 x 1 x kTmaG (x sweeps) and of 128 x kTmaG x 1 (y sweeps)
struct TmaMaps {
  CUtensorMap one[8], gx[8], gy[8];
};

// slots of kTmaG cells; a slot is refilled kTmaLag groups after it was read (so that the
// refilling thread rarely waits for the slowest warp), kTmaRing - kTmaLag groups ahead
constexpr int kTmaRing = MHD_TMA_RING, kTmaLag = MHD_TMA_LAG;
static_assert(kTmaRing > kTmaLag && kTmaLag >= 1, "ring");
constexpr int kTmaRowBytes = 128 * 4;
constexpr int kTmaSlotFloats = 10 * kTmaG * 128;   // rows 0-8 boxed, row 9 the z + 1 copies
// polls of a wait before it gives up (a suspend-time hint on the polls, letting the warp sleep
// in the barrier unit, measured 1.8x slower: the wake-up comes late)
constexpr int kTmaSpin = 1 << 24;

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(
                   smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
          smem_u32(bar)),
      "r"(bytes)
      : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// wait for the phase of the given parity to complete; false if it did not within the limit
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
  for (int i = 0; i < kTmaSpin; ++i)
    if (mbar_test(bar, parity)) return true;
  return false;
}
// one box of the 3D tensor (z, y, x) at coordinates (c0, c1, c2) into shared memory
__device__ __forceinline__ void tma_box(float* dst, const CUtensorMap* tm, int c0, int c1, int c2,
                                        unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<unsigned long long>(tm)), "r"(c0), "r"(c1), "r"(c2),
      "r"(smem_u32(bar))
      : "memory");
}

// shared memory of the TMA-staged march: the ring (10 rows of 128 floats per slot, row 9
// for the z + 1 neighbours the threads copy themselves) and 2 mbarriers per slot
constexpr size_t tma_march_smem() {
  return 128 + (size_t)kTmaRing * kTmaSlotFloats * 4 + 2 * kTmaRing * sizeof(unsigned long long);
}

template <int A, bool LAST, int PM, int S>
__device__ __forceinline__ void fluid_march_xy_tile_tma(const GridDesc& g, const FieldSet<float>& in,
                                                        const FieldSet<float>& out, float gamma,
                                                        double h, DevScalars* ds,
                                                        const TmaRows& tm, unsigned bx,
                                                        unsigned by, unsigned char* smem_raw) {
  static_assert(A == 0 || A == 1, "x or y sweep");
  using T = float;
  constexpr int NT = 128;
  constexpr int O = (A == 0) ? 1 : 0;
  constexpr int T1 = axis_t1(A), T2 = axis_t2(A);
  constexpr int R = kTmaRing, G = kTmaG, PF = kTmaRing - kTmaLag;   // PF: groups ahead
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int nz = g.n[2], nO = g.n[O];
  const long long p0 = (long long)bx * NT;
  const int z0 = (int)(p0 % nz), o = (int)(p0 / nz);   // nz % 128 == 0: one O row
  const int z = z0 + tid;
  const int oup = wrap_index(o + 1, nO, g.bc[O]);
  const int a0 = by * S;
  const int nA = g.n[A], bcA = g.bc[A];
  const T dth = step_factor<T>(ds, h) * T(FluxScale<T>::inv);
  const T hd = T(0.5) * dth;
  const long long sA = g.s[A], sO = g.s[O];
  // the ring on a 128-byte boundary of the shared window (box destinations)
  unsigned char* sm = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  float* ring = reinterpret_cast<float*>(sm);
  unsigned long long* full =
      reinterpret_cast<unsigned long long*>(sm + (size_t)R * kTmaSlotFloats * 4);
  unsigned long long* empty = full + R;
  const int js = a0 - 3;
  const int kend = min(S, nA - a0) + 6;
  const int ngroups = (kend + G - 1) / G;
  if (tid == 0) {
    for (int r = 0; r < R; ++r) {
      mbar_init(full + r, 1);
      mbar_init(empty + r, NT);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  bool ok = true;
  // slot layout: row r, cell c of the group at (r * G + c) * 128 (a box of 128 x G cells
  // lands as G consecutive rows of 128)
  auto issue_group = [&](int q) {
    const int s = q % R;
    if (q >= R && !mbar_wait(empty + s, (unsigned)((q / R - 1) & 1))) {
      ok = false;
      return;
    }
    float* slot = ring + (size_t)s * kTmaSlotFloats;
    mbar_arrive_tx(full + s, 9 * G * kTmaRowBytes);
    const int jg = js + q * G;               // the group's first cell along A
#pragma unroll
    for (int r = 0; r < 9; ++r) {
      const int j0 = r == 5 ? jg + 1 : jg;   // B_A one cell ahead
      const int co = r == 8 ? oup : o;
      if (j0 >= 0 && j0 + G <= nA) {
        const int cy = A == 0 ? co : j0, cx = A == 0 ? j0 : co;
        tma_box(slot + r * G * NT, &tm.g[r], z0, cy, cx, full + s);
      } else {
#pragma unroll
        for (int c = 0; c < G; ++c) {
          const int ja = wrap_index(j0 + c, nA, bcA);
          const int cy = A == 0 ? co : ja, cx = A == 0 ? ja : co;
          tma_box(slot + (r * G + c) * NT, &tm.one[r], z0, cy, cx, full + s);
        }
      }
    }
  };
  // the z + 1 neighbour of B_z that the next thread does not hold, copied by the thread
  // itself for a whole group (row 9)
  const bool special = tid == NT - 1 || z == nz - 1;
  const float* srcs = in.f[7] + (long long)wrap_index(z + 1, nz, g.bc[2]) + (long long)o * sO;
  auto issue_special = [&](int q) {
    if (q < ngroups && special) {
      float* d = ring + (size_t)(q % R) * kTmaSlotFloats + 9 * G * NT + tid;
#pragma unroll
      for (int c = 0; c < G; ++c)
        cp_async_elem(d + c * NT, srcs + (long long)wrap_index(js + q * G + c, nA, bcA) * sA);
    }
    cp_async_commit();
  };
  if (tid == 0)
    for (int q = 0; q < PF && q < ngroups; ++q) issue_group(q);
#pragma unroll
  for (int q = 0; q < PF; ++q) issue_special(q);
  FluidPencil<T, PM, LAST> P;
  P.init();
  const long long base = (long long)z + (long long)o * sO;
  T bn_cur = in.f[5 + A][base + wrap_off<T>(js, nA, bcA, sA)];
  T cm = T(0);
  bool nan_seen = false;
  constexpr int ZROW = (A == 0) ? 7 : 6;     // the row holding B_z (B_t2 for x, B_t1 for y)
  for (int q = 0; q < ngroups; ++q) {
    // the next group's boxes, by lane 0 of a rotating warp
    if (lane == 0 && w == (q & 3) && ok && q + PF < ngroups) issue_group(q + PF);
    issue_special(q + PF);
    cp_async_wait<PF>();
    const int s = q % R;
    if (ok && !mbar_wait(full + s, (unsigned)((q / R) & 1))) ok = false;
    const float* slot = ring + (size_t)s * kTmaSlotFloats;
#pragma unroll
    for (int c = 0; c < G; ++c) {
      const int k = q * G + c;
      if (k < kend) {
        const int j = js + k;
        const float* cl = slot + c * NT + tid;        // row r of this cell at cl[r * G * NT]
        T u0[5], b0[3];
#pragma unroll
        for (int r = 0; r < 5; ++r) u0[r] = cl[r * G * NT];
        const T bn_next = cl[5 * G * NT];
        const T zb_nb = special ? cl[9 * G * NT] : cl[ZROW * G * NT + 1];
        const T ob_nb = cl[8 * G * NT];
        b0[0] = T(0.5) * (bn_cur + bn_next);
        b0[1] = T(0.5) * (cl[6 * G * NT] + (A == 0 ? ob_nb : zb_nb));
        b0[2] = T(0.5) * (cl[7 * G * NT] + (A == 0 ? zb_nb : ob_nb));
        bn_cur = bn_next;
        T un[5], bo[3];
        if (P.push(k, u0, b0, gamma, dth, hd, un, bo)) {
          const long long co = base + (long long)(j - 3) * sA;
          out.f[0][co] = un[0];
          out.f[1 + A][co] = un[1];
          out.f[1 + T1][co] = un[2];
          out.f[1 + T2][co] = un[3];
          out.f[4][co] = un[4];
          if (!(un[0] > T(0))) P.st |= ST_UNPHYSICAL;
          if (LAST) {
            const T v = cell_cmax<T, PM>(un[0], un[1], un[2], un[3], un[4], bo[0], bo[1],
                                         bo[2], gamma, &P.st);
            if (v != v) nan_seen = true; else cm = fmax(cm, v);
          }
        }
      }
    }
    mbar_arrive(empty + s);
  }
  cp_async_wait<0>();
  if (LAST) block_max_to_global(cm, nan_seen, ds);
  if (!ok) P.st |= ST_TIMEOUT;
  if (P.st) atomicOr(&ds->status, P.st);
}

template <int A, bool LAST, int PM, int S>
__global__ void __launch_bounds__(128, MHD_VEC_MINB)
fluid_march_xy_tma(GridDesc g, FieldSet<float> in, FieldSet<float> out, float gamma, double h,
                   DevScalars* ds, const __grid_constant__ TmaRows tm) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  fluid_march_xy_tile_tma<A, LAST, PM, S>(g, in, out, gamma, h, ds, tm, blockIdx.x, blockIdx.y,
                                          smem_raw);
}

}  // namespace mhd
