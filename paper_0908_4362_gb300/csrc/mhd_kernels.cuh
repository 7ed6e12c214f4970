// Device code of the relaxing-TVD ideal-MHD sweeps for sm_103a.
//
// Method: Wong, Wong, Feng & Tang, arXiv:0908.4362, Sect. 3 (numerical scheme) and
// Sect. 4.3 (sweeping operations; Algorithms 1 and 2).  Every sweep is written once in
// local coordinates: normal n = A, transverse t1 = (A+1)%3, t2 = (A+2)%3.
//
// Memory layout: 8 separate field arrays (rho, mx, my, mz, E, Bx, By, Bz), flat index
// (x*ny + y)*nz + z, z contiguous (Sect. 4.1).  B is face centred: Bx[i] on the x-face
// i-1/2, etc. (Eq. "equat_b").  Every sweep kernel is out of place: it reads the current
// buffer of a field and writes the other one, so no thread reads what another writes.
// This header holds the per-cell arithmetic shared by the sweep kernels (mhd_march.cuh for
// x and y sweeps, mhd_segz.cuh for z sweeps) and the auxiliary kernels.
//
// Boundaries per axis: periodic (wrap) or outflow (every array index clamped to [0,N-1]).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mhd {

enum : int { ST_UNPHYSICAL = 1, ST_NONFINITE = 2, ST_BAD_DT = 4, ST_TIMEOUT = 8 };

struct GridDesc {
  int n[3];
  int bc[3];      // 0 periodic, 1 outflow
  long long s[3]; // strides in elements
};

template <typename T>
struct FieldSet {
  T* f[8];
};

// Device-resident step scalars: the time step is computed and applied on the device, so
// a step needs no host round trip (the paper reads dt back every step, Sect. 4.2 step 6).
struct DevScalars {
  double t;                  // current time
  double dt;                 // dt of the step in flight (0: step is a no-op)
  double dt_last;            // dt of the last step that advanced t
  double t_end;              // < 0: none
  unsigned long long cmax;   // bits of the c_max of the current state (float or double)
  int steps_done;            // steps that advanced t
  int status;                // sticky ST_* bits
  float dt_h;                // (float)(dt / h): the step factor of the FP32 sweeps
  int pad_;
  // partial maxima of the running c_max: warps fold their maximum into one of these slots
  // (atomicMax), spreading what would be one contended address over kCmaxSlots; dt_update
  // and the host fold them into cmax
  unsigned long long cmax_part[128];
};
constexpr int kCmaxSlots = 128;

// the folded c_max bits: cmax and every partial maximum (non-negative float bits order as
// unsigned integers)
__host__ __device__ inline unsigned long long fold_cmax_bits(const DevScalars& s) {
  unsigned long long m = s.cmax;
  for (int k = 0; k < kCmaxSlots; ++k) m = s.cmax_part[k] > m ? s.cmax_part[k] : m;
  return m;
}

// ------------------------------------------------------------------------------------
// scalar helpers
// ------------------------------------------------------------------------------------

template <typename T> struct Num;
template <> struct Num<float> {
  static __device__ __forceinline__ float div(float a, float b) { return __fdividef(a, b); }
  // a rounded product that the compiler never fuses into a following add
  static __device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ float sqrt(float a) { return sqrtf(a); }
  static __device__ __forceinline__ unsigned long long bits(float v) {
    return (unsigned long long)__float_as_uint(v);
  }
  static __host__ __device__ __forceinline__ double from_bits(unsigned long long b) {
#ifdef __CUDA_ARCH__
    return (double)__uint_as_float((unsigned)b);
#else
    union { unsigned u; float f; } x; x.u = (unsigned)b; return (double)x.f;
#endif
  }
};
template <> struct Num<double> {
  static __device__ __forceinline__ double div(double a, double b) { return a / b; }
  static __device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ double sqrt(double a) { return ::sqrt(a); }
  static __device__ __forceinline__ unsigned long long bits(double v) {
    return (unsigned long long)__double_as_longlong(v);
  }
  static __host__ __device__ __forceinline__ double from_bits(unsigned long long b) {
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)b);
#else
    union { unsigned long long u; double f; } x; x.u = b; return x.f;
#endif
  }
};

// a b + c and b - s a: one fused, singly rounded operation in FP32, two in FP64.  The FP32
// kernels are built without automatic contraction, so every fusion is written here and
// rounds the same in every kernel that inlines the expression (a grid's result does not
// depend on which kernel advanced it); FP64 keeps the oracle's separately rounded steps.
template <typename T>
__device__ __forceinline__ T ffma(T a, T b, T c) {
  if constexpr (sizeof(T) == 4) return __fmaf_rn(a, b, c);
  else return a * b + c;
}
template <typename T>
__device__ __forceinline__ T ffms(T s, T a, T b) {
  if constexpr (sizeof(T) == 4) return __fmaf_rn(-s, a, b);
  else return b - s * a;
}

// Element addressing of a field: a 64-bit element index, or (OFF32, for fields of less
// than 4 GiB each) an unsigned 32-bit byte offset from the field's base pointer, so
// that an access adds a 32-bit offset to a kernel-parameter base instead of doing 64-bit
// index arithmetic per field.  Offsets of neighbours below may be negative: unsigned
// arithmetic modulo 2^32 still yields the right in-range offset.
template <typename T, bool OFF32> struct FieldAddr {
  using I = long long;
  static __device__ __forceinline__ I of(long long e) { return e; }
  static __device__ __forceinline__ const T* at(const T* p, I i) { return p + i; }
  static __device__ __forceinline__ T* at(T* p, I i) { return p + i; }
};
template <typename T> struct FieldAddr<T, true> {
  using I = unsigned;
  static __device__ __forceinline__ I of(long long e) { return (unsigned)(e * (long long)sizeof(T)); }
  static __device__ __forceinline__ const T* at(const T* p, I i) {
    return reinterpret_cast<const T*>(reinterpret_cast<const char*>(p) + i);
  }
  static __device__ __forceinline__ T* at(T* p, I i) {
    return reinterpret_cast<T*>(reinterpret_cast<char*>(p) + i);
  }
};
#ifndef MHD_OFF32
#define MHD_OFF32 1
#endif
// the 32-bit byte offsets fit: every field of the grid spans less than 4 GiB
template <typename T>
__host__ __device__ inline bool field_off32(const GridDesc& g) {
  return MHD_OFF32 && (unsigned long long)g.n[0] * g.n[1] * g.n[2] * sizeof(T) <= 0xFFFFFFFFull;
}
// the x/y fluid march stores by 32-bit offsets too (measured: fluid x/y -3.5% at 512^3;
// the shared-row CT's stores were 1-2.5% slower that way and keep 64-bit indices)
#ifndef MHD_OFF32_XY
#define MHD_OFF32_XY 1
#endif

__device__ __forceinline__ int wrap_index(int i, int n, int bc) {
  if (i >= 0 && i < n) return i;
  if (bc == 0) {
    i %= n;
    return i < 0 ? i + n : i;
  }
  return i < 0 ? 0 : n - 1;
}

// van Leer limiter, Eq. "eq:limiter"; no correction unless both one-sided corrections
// have the same sign (text before Eq. "eq:Delta_F_n").
template <typename T>
__device__ __forceinline__ T vanleer(T a, T b) {
  T ab = a * b;
  return ab > T(0) ? Num<T>::div(T(2) * ab, a + b) : T(0);
}

// Pressure recovery modes of the FP32 sweeps (the context's pressure mode): 0 plain FP32,
// 1 FP64 arithmetic, 2 compensated FP32.  p = (gamma-1)(E - m^2/(2 rho) - B^2/2) cancels at
// low plasma beta, where E is dominated by B^2/2; plain FP32 loses log2(E/p) bits of p.
enum : int { PM_FP32 = 0, PM_FP64 = 1, PM_COMP = 2 };

// Error-free transformations in round-to-nearest FP32: a + b = s + e exactly (Knuth's
// TwoSum, TAOCP vol. 2, Sect. 4.2.2) and a b = p + e exactly (Dekker's product, its error
// term taken with one fused multiply-add).  Written with explicitly rounded operations so
// that no compiler contraction changes them.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bv = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bv)), __fsub_rn(b, bv));
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}
// x^2 + y^2 + z^2 as an unevaluated sum hi + lo (double-float), exact to ~2^-44 relative
__device__ __forceinline__ void sumsq_df(float x, float y, float z, float& hi, float& lo) {
  float p1, e1, p2, e2, p3, e3, s, t1, t2;
  two_prod(x, x, p1, e1);
  two_prod(y, y, p2, e2);
  two_prod(z, z, p3, e3);
  two_sum(p1, p2, s, t1);
  two_sum(s, p3, hi, t2);
  lo = __fadd_rn(__fadd_rn(__fadd_rn(e1, e2), e3), __fadd_rn(t1, t2));
}
// p = (gamma-1)(E - |m|^2/(2 rho) - |B|^2/2) in double-float FP32 arithmetic: the two
// quadratic terms and the two cancelling subtractions keep their rounding errors, so p comes
// out as the FP32 rounding of the exact value for the given FP32 inputs (as FP64 arithmetic
// would give it), at a fraction of GB300's FP64 cost.  gm1 = gamma - 1, ir ~ 1/rho (an
// approximate reciprocal is enough: the remainder below absorbs its error).
__device__ __forceinline__ float pressure_comp(float rho, float ir, float m1, float m2, float m3,
                                               float E, float b0, float b1, float b2, float gm1) {
  float mh, ml, bh, bl;
  sumsq_df(m1, m2, m3, mh, ml);
  sumsq_df(b0, b1, b2, bh, bl);
  // |m|^2 / rho = q + ql: q an approximate quotient, its remainder mh - q rho by one FMA
  // (exact to ~2^-46 of mh for a quotient within a few ulps)
  const float q = __fmul_rn(mh, ir);
  const float r = __fmaf_rn(-q, rho, mh);
  const float ql = __fmul_rn(__fadd_rn(r, ml), ir);
  float x1, f1, x2, f2;
  two_sum(E, -0.5f * q, x1, f1);
  two_sum(x1, -0.5f * bh, x2, f2);
  const float tail = __fadd_rn(__fadd_rn(f1, f2), -0.5f * __fadd_rn(ql, bl));
  return __fmaf_rn(gm1, x2, __fmul_rn(gm1, tail));
}

// Cell flux in local coordinates, Eqs. "eq:flux" and "eq:lr": returns the fluxes of the
// right- and left-moving variables, fr = (c u + F)/2 and fl = (c u - F)/2, with the
// freezing speed c = |v_n| + sqrt(gamma p/rho + B^2/rho) -- scaled by FluxScale<T>::out:
// FP32 returns c u + F and c u - F (twice the fluxes, six fewer multiplications per cell),
// and its callers take half step factors; a power-of-two scale commutes with rounding.
// PM: the pressure recovery mode (PM_FP32, PM_FP64, PM_COMP), FP32 only.
template <typename T> struct FluxScale {
  static constexpr double out = sizeof(T) == 4 ? 2.0 : 1.0;   // cell_flux result / fluxes
  static constexpr double inv = 1.0 / out;                    // factor on dt/h, dt/(2h)
};

template <typename T, int PM>
__device__ __forceinline__ int cell_flux(const T u[5], const T b[3], T gamma, T fr[5], T fl[5]) {
  const T rho = u[0];
  if constexpr (sizeof(T) == 4) {
    // FP32: one reciprocal of rho, the radicand as (gamma p + B^2)/rho, and the doubled
    // relaxed fluxes c u +- F (the same quantities, fewer instructions)
    const T ir = T(1) / rho;
    const T vn = u[1] * ir, vt1 = u[2] * ir, vt2 = u[3] * ir;
    const T b2 = __fmaf_rn(b[2], b[2], __fmaf_rn(b[1], b[1], b[0] * b[0]));
    T p;
    if (PM == PM_COMP) {
      p = pressure_comp(rho, ir, u[1], u[2], u[3], u[4], b[0], b[1], b[2], gamma - T(1));
    } else if (PM == PM_FP64) {
      const double m1 = u[1], m2 = u[2], m3 = u[3];
      const double bb0 = b[0], bb1 = b[1], bb2 = b[2];
      const double ke = 0.5 * __fma_rn(m3, m3, __fma_rn(m2, m2, m1 * m1)) / (double)rho;
      const double bb = __fma_rn(bb2, bb2, __fma_rn(bb1, bb1, bb0 * bb0));
      p = (T)(((double)gamma - 1.0) * __fma_rn(-0.5, bb, (double)u[4] - ke));
    } else {
      const T mv = __fmaf_rn(u[3], vt2, __fmaf_rn(u[2], vt1, u[1] * vn));
      p = (gamma - T(1)) * __fmaf_rn(T(-0.5), b2, __fmaf_rn(T(-0.5), mv, u[4]));
    }
    const T ps = __fmaf_rn(T(0.5), b2, p);
    const T bv = __fmaf_rn(b[2], vt2, __fmaf_rn(b[1], vt1, b[0] * vn));
    T F[5];
    F[0] = u[1];
    F[1] = __fmaf_rn(-b[0], b[0], __fmaf_rn(u[1], vn, ps));
    F[2] = __fmaf_rn(-b[0], b[1], u[2] * vn);
    F[3] = __fmaf_rn(-b[0], b[2], u[3] * vn);
    F[4] = __fmaf_rn(-b[0], bv, (u[4] + ps) * vn);
    const T rad = __fmaf_rn(gamma, p, b2) * ir;
    const int st = (!(rho > T(0)) || rad < T(0)) ? ST_UNPHYSICAL : 0;
    const T c = fabs(vn) + sqrtf(rad);
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      fr[k] = __fmaf_rn(c, u[k], F[k]);
      fl[k] = __fmaf_rn(c, u[k], -F[k]);
    }
    return st;
  } else {
    // FP64: the oracle's expressions, operation for operation
    const T vn = Num<T>::div(u[1], rho), vt1 = Num<T>::div(u[2], rho), vt2 = Num<T>::div(u[3], rho);
    const T b2 = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
    const T v2 = vn * vn + vt1 * vt1 + vt2 * vt2;
    const T p = (gamma - T(1)) * (u[4] - T(0.5) * rho * v2 - T(0.5) * b2);
    const T ps = p + T(0.5) * b2;
    const T bv = b[0] * vn + b[1] * vt1 + b[2] * vt2;
    T F[5];
    F[0] = u[1];
    F[1] = u[1] * vn + ps - b[0] * b[0];
    F[2] = u[2] * vn - b[0] * b[1];
    F[3] = u[3] * vn - b[0] * b[2];
    F[4] = (u[4] + ps) * vn - b[0] * bv;
    const T rad = Num<T>::div(gamma * p, rho) + Num<T>::div(b2, rho);
    const int st = (!(rho > T(0)) || rad < T(0)) ? ST_UNPHYSICAL : 0;
    const T c = fabs(vn) + Num<T>::sqrt(rad);
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      fr[k] = T(0.5) * (c * u[k] + F[k]);
      fl[k] = T(0.5) * (c * u[k] - F[k]);
    }
    return st;
  }
}

// phi(a, b) / 2: the limited correction phi(a/2, b/2) applied to a flux (Eq. "eq:F_n").
// FP32: ab / (a + b) directly; FP64: the oracle's 2ab/(a+b) halved (the same rounded value).
template <typename T>
__device__ __forceinline__ T half_vanleer(T a, T b) {
  if constexpr (sizeof(T) == 4) {
    const T ab = a * b;
    return ab > T(0) ? ab / (a + b) : T(0);
  } else {
    return T(0.5) * vanleer(a, b);
  }
}

// base + phi(a, b)/2 and base - phi(a, b)/2 (the limited corrections of Eq. "eq:F_n"): in
// FP32 the quotient ab/(a+b) is ab times an approximate reciprocal, fused into the sum
template <typename T>
__device__ __forceinline__ T plus_half_vanleer(T base, T a, T b) {
  if constexpr (sizeof(T) == 4) {
    const T ab = a * b;
    const T r = __fdividef(T(1), a + b);
    return ab > T(0) ? __fmaf_rn(ab, r, base) : base;
  } else {
    return base + half_vanleer(a, b);
  }
}
template <typename T>
__device__ __forceinline__ T minus_half_vanleer(T base, T a, T b) {
  if constexpr (sizeof(T) == 4) {
    const T ab = a * b;
    const T r = __fdividef(T(1), a + b);
    return ab > T(0) ? __fmaf_rn(-ab, r, base) : base;
  } else {
    return base - half_vanleer(a, b);
  }
}

// |v|^2 and |B|^2 summed smallest first, so that c_max does not depend on axis order.
template <typename T>
__device__ __forceinline__ T sum3_sorted(T a, T b, T c) {
  T lo = fmin(a, b), hi = fmax(a, b);
  T l2 = fmin(lo, c), m = fmax(lo, c);
  T mid = fmin(hi, m), top = fmax(hi, m);
  return (l2 + mid) + top;
}

// CFL speed of one cell, Eq. "equat_CFL": max(|vx|,|vy|,|vz|) + sqrt(gamma p/rho + B^2/rho).
template <typename T, int PM>
__device__ __forceinline__ T cell_cmax(T rho, T m0, T m1, T m2, T E, T b0, T b1, T b2, T gamma,
                                       int* st) {
  const T v0 = Num<T>::div(m0, rho), v1 = Num<T>::div(m1, rho), v2 = Num<T>::div(m2, rho);
  const T vv = sum3_sorted(v0 * v0, v1 * v1, v2 * v2);
  const T bb = sum3_sorted(b0 * b0, b1 * b1, b2 * b2);
  T p;
  if constexpr (PM == PM_COMP && sizeof(T) == 4) {
    // the three squares of each sum in a fixed order of magnitude, as sum3_sorted, so that
    // c_max does not depend on the axis order
    const float ma = fminf(fminf(fabsf(m0), fabsf(m1)), fabsf(m2));
    const float mc = fmaxf(fmaxf(fabsf(m0), fabsf(m1)), fabsf(m2));
    const float mb = fmaxf(fminf(fabsf(m0), fabsf(m1)), fminf(fmaxf(fabsf(m0), fabsf(m1)), fabsf(m2)));
    const float ba = fminf(fminf(fabsf(b0), fabsf(b1)), fabsf(b2));
    const float bc = fmaxf(fmaxf(fabsf(b0), fabsf(b1)), fabsf(b2));
    const float bm = fmaxf(fminf(fabsf(b0), fabsf(b1)), fminf(fmaxf(fabsf(b0), fabsf(b1)), fabsf(b2)));
    p = pressure_comp(rho, __fdividef(1.f, rho), ma, mb, mc, E, ba, bm, bc, gamma - T(1));
  } else if (PM == PM_FP64) {
    const double rd = rho, mm0 = m0, mm1 = m1, mm2 = m2, c0 = b0, c1 = b1, c2 = b2;
    const double ke = 0.5 * (mm0 * mm0 + mm1 * mm1 + mm2 * mm2) / rd;
    p = (T)(((double)gamma - 1.0) * ((double)E - ke - 0.5 * (c0 * c0 + c1 * c1 + c2 * c2)));
  } else {
    p = (gamma - T(1)) * ffms(T(0.5), bb, ffms(T(0.5) * rho, vv, E));
  }
  const T rad = Num<T>::div(gamma * p, rho) + Num<T>::div(bb, rho);
  if (!(rho > T(0)) || rad < T(0)) *st |= ST_UNPHYSICAL;
  const T vm = fmax(fmax(fabs(v0), fabs(v1)), fabs(v2));
  return vm + Num<T>::sqrt(rad);
}

template <typename T>
__device__ __forceinline__ void block_max_to_global(T v, bool nan_seen, DevScalars* ds) {
  // warp max, then one atomic per warp (c_max >= 0, so float bits order as integers)
  unsigned mask = __activemask();
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(mask, v, o));
  bool anynan = __any_sync(mask, nan_seen);
  if ((threadIdx.x & 31) == 0) {
    if (v > T(0))
      atomicMax(&ds->cmax_part[((blockIdx.x << 2) + (threadIdx.x >> 5)) & (kCmaxSlots - 1)],
                Num<T>::bits(v));
    if (anynan) atomicOr(&ds->status, ST_NONFINITE);
  }
}

__host__ __device__ constexpr int axis_t1(int a) { return (a + 1) % 3; }
__host__ __device__ constexpr int axis_t2(int a) { return (a + 2) % 3; }

// ------------------------------------------------------------------------------------
// auxiliary kernels
// ------------------------------------------------------------------------------------

// CFL speed of cell i of a state, with B averaged from the faces to the cell centre
template <typename T, int PM>
__device__ __forceinline__ T cmax_cell(const GridDesc& g, const FieldSet<T>& in, long long i,
                                       T gamma, int* st) {
  const int z = (int)(i % g.n[2]);
  const long long xy = i / g.n[2];
  const int y = (int)(xy % g.n[1]);
  const int x = (int)(xy / g.n[1]);
  const int c[3] = {x, y, z};
  T bc[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const long long gn = i + (long long)(wrap_index(c[a] + 1, g.n[a], g.bc[a]) - c[a]) * g.s[a];
    bc[a] = T(0.5) * (in.f[5 + a][i] + in.f[5 + a][gn]);
  }
  return cell_cmax<T, PM>(in.f[0][i], in.f[1][i], in.f[2][i], in.f[3][i], in.f[4][i], bc[0],
                           bc[1], bc[2], gamma, st);
}

// c_max of cells [i0, i1) by one block, folded into the partial maxima of ds
template <typename T, int PM>
__device__ __forceinline__ void cmax_range(const GridDesc& g, const FieldSet<T>& in, T gamma,
                                           DevScalars* ds, long long i0, long long i1,
                                           long long stride) {
  T cm = T(0);
  bool nan_seen = false;
  int st = 0;
  for (long long i = i0; i < i1; i += stride) {
    const T v = cmax_cell<T, PM>(g, in, i, gamma, &st);
    if (v != v) nan_seen = true; else cm = fmax(cm, v);
  }
  block_max_to_global(cm, nan_seen, ds);
  if (st) atomicOr(&ds->status, st);
}

// c_max of a state (at initialisation, on request, and at the end of a step whose last
// fluid sweep runs along an axis of one cell)
template <typename T, int PM>
__global__ void cmax_kernel(GridDesc g, FieldSet<T> in, T gamma, DevScalars* ds) {
  const long long N = (long long)g.n[0] * g.n[1] * g.n[2];
  cmax_range<T, PM>(g, in, gamma, ds, blockIdx.x * (long long)blockDim.x + threadIdx.x, N,
                     (long long)gridDim.x * blockDim.x);
}

// dt = cfl h / c_max on the device, clipped to land on t_end (Sect. 4.2 steps 4-5, 8-9)
template <typename T>
__device__ __forceinline__ void dt_update(DevScalars* ds, double cfl_h, double h) {
  const double cm = Num<T>::from_bits(fold_cmax_bits(*ds));
  double dt = cfl_h / cm;
  int clipped = 0, active = 1;
  if (!(cm > 0.0) || !(dt == dt) || dt > 1e300) {
    atomicOr(&ds->status, ST_BAD_DT);
    dt = 0.0;
    active = 0;
  }
  if (active && ds->t_end >= 0.0) {
    if (ds->t >= ds->t_end) {
      dt = 0.0;
      active = 0;
    } else {
      const double rest = 0.5 * (ds->t_end - ds->t);
      if (dt >= rest) { dt = rest; clipped = 1; }
    }
  }
  ds->dt = dt;
  ds->dt_h = (float)(dt / h);
  if (active) {
    ds->t = clipped ? ds->t_end : ds->t + 2.0 * dt;
    ds->dt_last = dt;
    ds->steps_done += 1;
  }
  ds->cmax = 0ull;   // the last sweep of this step accumulates the next c_max
  for (int k = 0; k < kCmaxSlots; ++k) ds->cmax_part[k] = 0ull;
}

template <typename T>
__global__ void dt_kernel(DevScalars* ds, double cfl_h, double h) {
  dt_update<T>(ds, cfl_h, h);
}

// dt/h of the step in flight in the sweep's precision.  FP32 sweeps read the factor that
// dt_update (or mhd_apply) stored, (float)(dt / h), the same rounded value, instead of each
// thread dividing in FP64, which runs at GB300's low FP64 rate (and the z segments would do
// it once per 3 cells)
template <typename T>
__device__ __forceinline__ T step_factor(const DevScalars* ds, double h) {
  if constexpr (sizeof(T) == 4) return ds->dt_h;
  else return ds->dt / h;
}

// Exact float -> double by re-biasing the bits of normal numbers (and zeros) with integer
// operations: GB300 executes the FP64 conversion at its low FP64 rate, which doubled the
// cost of the sums.  Subnormals, infinities and NaN take the ordinary conversion.
__device__ __forceinline__ double widen(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned e = (b >> 23) & 0xffu;
  const bool zero = (b << 1) == 0u;
  if ((e == 0u && !zero) || e == 0xffu) return (double)f;
  const unsigned hi = zero ? (b & 0x80000000u)
                           : (b & 0x80000000u) | ((e + 896u) << 20) | ((b & 0x7fffffu) >> 3);
  const unsigned lo = zero ? 0u : b << 29;
  return __hiloint2double((int)hi, (int)lo);
}
__device__ __forceinline__ double widen(double d) { return d; }

// FP64 conservation sums: per-block partial sums (deterministic two-pass reduction)
template <typename T>
__global__ void sums_partial_kernel(long long N, FieldSet<T> in, double* partial) {
  __shared__ double red[8][32];
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] += widen(in.f[k][i]);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    double v = acc[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[k][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < 8) {
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[threadIdx.x][w];
    partial[blockIdx.x * 8 + threadIdx.x] = v;
  }
}

static __global__ void sums_final_kernel(int nblocks, const double* partial, double* out) {
  if (threadIdx.x < 8) {
    double v = 0.0;
    for (int b = 0; b < nblocks; ++b) v += partial[b * 8 + threadIdx.x];
    out[threadIdx.x] = v;
  }
}

template <typename S, typename D>
__global__ void convert_kernel(long long n, const S* __restrict__ src, D* __restrict__ dst) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = (D)src[i];
}

}  // namespace mhd
