// Device code of the relaxing-TVD ideal-MHD sweeps for sm_103a.
//
// Method: Wong, Wong, Feng & Tang, arXiv:0908.4362, Sect. 3 (numerical scheme) and
// Sect. 4.3 (sweeping operations; Algorithms 1 and 2).  Every sweep is written once in
// local coordinates: normal n = A, transverse t1 = (A+1)%3, t2 = (A+2)%3.
//
// Memory layout: 8 separate field arrays (rho, mx, my, mz, E, Bx, By, Bz), flat index
// (x*ny + y)*nz + z, z contiguous (Sect. 4.1).  B is face centred: Bx[i] on the x-face
// i-1/2, etc. (Eq. "equat_b").  Every kernel is out of place: it reads the current buffer
// of a field and writes the other one, so no tile reads what another tile writes.
//
// Boundaries per axis: periodic (wrap) or outflow (every array index clamped to [0,N-1]).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mhd {

enum : int { ST_UNPHYSICAL = 1, ST_NONFINITE = 2, ST_BAD_DT = 4 };

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
  unsigned long long cmax;   // bits of the running c_max (float or double), atomicMax
  int steps_done;            // steps that advanced t
  int status;                // sticky ST_* bits
};

// ------------------------------------------------------------------------------------
// scalar helpers
// ------------------------------------------------------------------------------------

template <typename T> struct Num;
template <> struct Num<float> {
  static __device__ __forceinline__ float div(float a, float b) { return __fdividef(a, b); }
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

// Cell flux in local coordinates, Eqs. "eq:flux" and "eq:lr": returns the fluxes of the
// right- and left-moving variables, fr = (c u + F)/2 and fl = (c u - F)/2, with the
// freezing speed c = |v_n| + sqrt(gamma p/rho + B^2/rho).
// P64: recover the pressure in double precision (low-beta cancellation in E - B^2/2).
template <typename T, bool P64>
__device__ __forceinline__ int cell_flux(const T u[5], const T b[3], T gamma, T fr[5], T fl[5]) {
  const T rho = u[0];
  const T vn = Num<T>::div(u[1], rho), vt1 = Num<T>::div(u[2], rho), vt2 = Num<T>::div(u[3], rho);
  const T b2 = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
  T p;
  if (P64) {
    const double rd = (double)rho;
    const double m1 = u[1], m2 = u[2], m3 = u[3];
    const double bb0 = b[0], bb1 = b[1], bb2 = b[2];
    const double ke = 0.5 * (m1 * m1 + m2 * m2 + m3 * m3) / rd;
    p = (T)(((double)gamma - 1.0) * ((double)u[4] - ke - 0.5 * (bb0 * bb0 + bb1 * bb1 + bb2 * bb2)));
  } else {
    const T v2 = vn * vn + vt1 * vt1 + vt2 * vt2;
    p = (gamma - T(1)) * (u[4] - T(0.5) * rho * v2 - T(0.5) * b2);
  }
  const T ps = p + T(0.5) * b2;
  const T bv = b[0] * vn + b[1] * vt1 + b[2] * vt2;
  T F[5];
  F[0] = u[1];
  F[1] = u[1] * vn + ps - b[0] * b[0];
  F[2] = u[2] * vn - b[0] * b[1];
  F[3] = u[3] * vn - b[0] * b[2];
  F[4] = (u[4] + ps) * vn - b[0] * bv;
  const T rad = Num<T>::div(gamma * p, rho) + Num<T>::div(b2, rho);
  int st = (!(rho > T(0)) || rad < T(0)) ? ST_UNPHYSICAL : 0;
  const T c = fabs(vn) + Num<T>::sqrt(rad);
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    fr[k] = T(0.5) * (c * u[k] + F[k]);
    fl[k] = T(0.5) * (c * u[k] - F[k]);
  }
  return st;
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
template <typename T, bool P64>
__device__ __forceinline__ T cell_cmax(T rho, T m0, T m1, T m2, T E, T b0, T b1, T b2, T gamma,
                                       int* st) {
  const T v0 = Num<T>::div(m0, rho), v1 = Num<T>::div(m1, rho), v2 = Num<T>::div(m2, rho);
  const T vv = sum3_sorted(v0 * v0, v1 * v1, v2 * v2);
  const T bb = sum3_sorted(b0 * b0, b1 * b1, b2 * b2);
  T p;
  if (P64) {
    const double rd = rho, mm0 = m0, mm1 = m1, mm2 = m2, c0 = b0, c1 = b1, c2 = b2;
    const double ke = 0.5 * (mm0 * mm0 + mm1 * mm1 + mm2 * mm2) / rd;
    p = (T)(((double)gamma - 1.0) * ((double)E - ke - 0.5 * (c0 * c0 + c1 * c1 + c2 * c2)));
  } else {
    p = (gamma - T(1)) * (E - T(0.5) * rho * vv - T(0.5) * bb);
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
    if (v > T(0)) atomicMax(&ds->cmax, Num<T>::bits(v));
    if (anynan) atomicOr(&ds->status, ST_NONFINITE);
  }
}

__host__ __device__ constexpr int axis_t1(int a) { return (a + 1) % 3; }
__host__ __device__ constexpr int axis_t2(int a) { return (a + 2) % 3; }
// tile geometry: pencils of S cells along A, W pencils side by side along the "width" axis
// (z when A != z, for coalescing; y when A == z), one row along the remaining axis.
__host__ __device__ constexpr int axis_w(int a) { return a == 2 ? 1 : 2; }
__host__ __device__ constexpr int axis_o(int a) { return a == 0 ? 1 : 0; }

template <typename T> struct FluidTile { static constexpr int S = 64, W = 8, NT = 256; };
template <> struct FluidTile<double> { static constexpr int S = 32, W = 8, NT = 256; };
template <typename T> struct CtTile { static constexpr int S = 64, W = 8, NT = 256; };
template <> struct CtTile<double> { static constexpr int S = 32, W = 8, NT = 256; };

// ------------------------------------------------------------------------------------
// fluid_A(dt): Algorithm 1.  Stage 1: first-order upwind fluxes of u^t give u^{t+dt/2}
// (Eq. "eq:Delta_u_half"); stage 2: van Leer limited fluxes of u^{t+dt/2} give u^{t+dt}
// (Eq. "eq:Delta_u_full").  B is frozen and averaged to cell centres.  LAST: also reduce
// c_max of the new state for the next step's CFL condition (fused Eq. "equat_CFL").
// ------------------------------------------------------------------------------------
template <typename T, int A, bool LAST, bool P64>
__global__ void __launch_bounds__(FluidTile<T>::NT)
fluid_kernel(GridDesc g, FieldSet<T> in, FieldSet<T> out, T gamma, double h, DevScalars* ds) {
  constexpr int S = FluidTile<T>::S, W = FluidTile<T>::W, NT = FluidTile<T>::NT;
  constexpr int G = 3, E = S + 2 * G, EW = E * W;
  constexpr int T1 = axis_t1(A), T2 = axis_t2(A), WX = axis_w(A), OX = axis_o(A);
  constexpr int DS = (A == 2) ? 1 : W;   // smem stride from cell e to e+1
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* su = reinterpret_cast<T*>(smem_raw);
  T* sb = su + 5 * EW;
  T* sfr = sb + 3 * EW;
  T* sfl = sfr + 5 * EW;
  T* sh = sfl + 5 * EW;

  const double dtd = ds->dt;
  const T dth = (T)(dtd / h);
  const int nA = g.n[A], nW = g.n[WX];
  const int a0 = blockIdx.x * S, w0 = blockIdx.y * W, io = blockIdx.z;
  const int bcA = g.bc[A];
  int st = 0;

  // phase 0: load u and cell-centred B on the extended pencils, stage-1 fluxes
  for (int idx = threadIdx.x; idx < EW; idx += NT) {
    const int e = (A == 2) ? idx % E : idx / W;
    const int w = (A == 2) ? idx / E : idx % W;
    int c[3];
    c[A] = wrap_index(a0 + e - G, nA, bcA);
    c[WX] = min(w0 + w, nW - 1);
    c[OX] = io;
    const long long gi = c[0] * g.s[0] + c[1] * g.s[1] + c[2] * g.s[2];
    T u[5], b[3], fr[5], fl[5];
    u[0] = in.f[0][gi];
    u[1] = in.f[1 + A][gi];
    u[2] = in.f[1 + T1][gi];
    u[3] = in.f[1 + T2][gi];
    u[4] = in.f[4][gi];
    const long long gn = gi + (long long)(wrap_index(a0 + e - G + 1, nA, bcA) - c[A]) * g.s[A];
    const long long g1 = gi + (long long)(wrap_index(c[T1] + 1, g.n[T1], g.bc[T1]) - c[T1]) * g.s[T1];
    const long long g2 = gi + (long long)(wrap_index(c[T2] + 1, g.n[T2], g.bc[T2]) - c[T2]) * g.s[T2];
    b[0] = T(0.5) * (in.f[5 + A][gi] + in.f[5 + A][gn]);
    b[1] = T(0.5) * (in.f[5 + T1][gi] + in.f[5 + T1][g1]);
    b[2] = T(0.5) * (in.f[5 + T2][gi] + in.f[5 + T2][g2]);
    st |= cell_flux<T, P64>(u, b, gamma, fr, fl);
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      su[k * EW + idx] = u[k];
      sfr[k * EW + idx] = fr[k];
      sfl[k * EW + idx] = fl[k];
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) sb[k * EW + idx] = b[k];
  }
  __syncthreads();

  // phase 1: u^{t+dt/2} = u - dt/2h (G1_{e+1/2} - G1_{e-1/2}), G1_{e+1/2} = FR_e - FL_{e+1}
  const T hd = T(0.5) * dth;
  for (int idx = threadIdx.x; idx < EW; idx += NT) {
    const int e = (A == 2) ? idx % E : idx / W;
    if (e < 1 || e >= E - 1) continue;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const T gp = sfr[k * EW + idx] - sfl[k * EW + idx + DS];
      const T gm = sfr[k * EW + idx - DS] - sfl[k * EW + idx];
      sh[k * EW + idx] = su[k * EW + idx] - hd * (gp - gm);
    }
  }
  __syncthreads();

  // phase 2: stage-2 fluxes of u^{t+dt/2} (same frozen B), overwriting stage-1 fluxes
  for (int idx = threadIdx.x; idx < EW; idx += NT) {
    const int e = (A == 2) ? idx % E : idx / W;
    if (e < 1 || e >= E - 1) continue;
    T u[5], b[3], fr[5], fl[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) u[k] = sh[k * EW + idx];
#pragma unroll
    for (int k = 0; k < 3; ++k) b[k] = sb[k * EW + idx];
    st |= cell_flux<T, P64>(u, b, gamma, fr, fl);
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      sfr[k * EW + idx] = fr[k];
      sfl[k * EW + idx] = fl[k];
    }
  }
  __syncthreads();

  // phase 3: limited interface fluxes G2_{e+1/2} for e in [G-1, G+S)
  //   right-moving: FR_e + phi((FR_e - FR_{e-1})/2, (FR_{e+1} - FR_e)/2)    Eq. "eq:F_n"
  //   left-moving (mirror): FL_{e+1} - phi((FL_{e+1} - FL_e)/2, (FL_{e+2} - FL_{e+1})/2)
  for (int idx = threadIdx.x; idx < EW; idx += NT) {
    const int e = (A == 2) ? idx % E : idx / W;
    if (e < G - 1 || e >= G + S) continue;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const T* r = sfr + k * EW + idx;
      const T* l = sfl + k * EW + idx;
      const T frm = r[-DS], fr0 = r[0], frp = r[DS];
      const T fl0 = l[0], fl1 = l[DS], fl2 = l[2 * DS];
      const T right = fr0 + vanleer(T(0.5) * (fr0 - frm), T(0.5) * (frp - fr0));
      const T left = fl1 - vanleer(T(0.5) * (fl1 - fl0), T(0.5) * (fl2 - fl1));
      sh[k * EW + idx] = right - left;
    }
  }
  __syncthreads();

  // phase 4: u^{t+dt} = u^t - dt/h (G2_{e+1/2} - G2_{e-1/2}); store; optional c_max
  T cm = T(0);
  bool nan_seen = false;
  for (int idx = threadIdx.x; idx < EW; idx += NT) {
    const int e = (A == 2) ? idx % E : idx / W;
    const int w = (A == 2) ? idx / E : idx % W;
    const int ia = a0 + e - G;
    if (e < G || e >= G + S || ia >= nA || w0 + w >= nW) continue;
    int c[3];
    c[A] = ia;
    c[WX] = w0 + w;
    c[OX] = io;
    const long long gi = c[0] * g.s[0] + c[1] * g.s[1] + c[2] * g.s[2];
    T un[5];
#pragma unroll
    for (int k = 0; k < 5; ++k)
      un[k] = su[k * EW + idx] - dth * (sh[k * EW + idx] - sh[k * EW + idx - DS]);
    out.f[0][gi] = un[0];
    out.f[1 + A][gi] = un[1];
    out.f[1 + T1][gi] = un[2];
    out.f[1 + T2][gi] = un[3];
    out.f[4][gi] = un[4];
    if (!(un[0] > T(0))) st |= ST_UNPHYSICAL;
    if (LAST) {
      const T b0 = sb[idx], b1 = sb[EW + idx], b2 = sb[2 * EW + idx];
      // global component order for the CFL speed is irrelevant: the sums are sorted
      const T v = cell_cmax<T, P64>(un[0], un[1], un[2], un[3], un[4], b0, b1, b2, gamma, &st);
      if (v != v) nan_seen = true; else cm = fmax(cm, v);
    }
  }
  if (LAST) block_max_to_global(cm, nan_seen, ds);
  if (st) atomicOr(&ds->status, st);
}

// ------------------------------------------------------------------------------------
// CT_A: for t in (t1, t2): face velocity of the post-fluid state across the t-face,
// smoothed 1/4(1,2,1) along A (Eq. "eq:averaging_x"), first-order upwind EMF v B_t by the
// sign of the edge velocity (Eq. "eq:first_flux"), B_t at t+dt/2, limited second-order
// EMF; then B_t -= dt/h d_A EMF (advection) and B_A += dt/h d_t EMF (constraint), both
// from the same EMF (Sect. 3; Algorithm 2).
//
// Tile: S cells along A; EMF rows (pencils along A) are kept for
//   group 0: t = WX, rows w0 .. w0+W (W+1 rows) at io,
//   group 1: t = OX, rows w0 .. w0+W-1 at io,
//   group 2: t = OX, rows w0 .. w0+W-1 at io+1,
// which are all the EMFs the tile's B_t and B_A updates need.
// ------------------------------------------------------------------------------------
template <typename T, int A>
__global__ void __launch_bounds__(CtTile<T>::NT)
ct_kernel(GridDesc g, FieldSet<T> in, FieldSet<T> out, double h, DevScalars* ds) {
  constexpr int S = CtTile<T>::S, W = CtTile<T>::W, NT = CtTile<T>::NT;
  constexpr int G = 4, E = S + 2 * G, R = 3 * W + 1, ER = E * R;
  constexpr int T1 = axis_t1(A), T2 = axis_t2(A), WX = axis_w(A), OX = axis_o(A);
  constexpr int DS = (A == 2) ? 1 : R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sv = reinterpret_cast<T*>(smem_raw);   // vf, later g = vs B_half
  T* ss = sv + ER;                           // vs
  T* sbt = ss + ER;                          // B_t
  T* se = sbt + ER;                          // E1, later E2

  const T dth = (T)(ds->dt / h);
  const int nA = g.n[A], nW = g.n[WX], nO = g.n[OX];
  const int a0 = blockIdx.x * S, w0 = blockIdx.y * W, io = blockIdx.z;
  const int bcA = g.bc[A];
  const int io1 = wrap_index(io + 1, nO, g.bc[OX]);

  // phase 0: face velocity across the t-face and B_t on every EMF row
  for (int idx = threadIdx.x; idx < ER; idx += NT) {
    const int e = (A == 2) ? idx % E : idx / R;
    const int r = (A == 2) ? idx / E : idx % R;
    int c[3], cx[3];
    c[A] = cx[A] = wrap_index(a0 + e - G, nA, bcA);
    int t;
    if (r <= W) {                   // group 0: t = WX
      t = WX;
      c[WX] = wrap_index(w0 + r, nW, g.bc[WX]);
      c[OX] = io;
      cx[WX] = wrap_index(c[WX] - 1, nW, g.bc[WX]);
      cx[OX] = io;
    } else {                        // groups 1, 2: t = OX
      t = OX;
      const int rr = (r - W - 1) % W, grp = (r - W - 1) / W;
      c[WX] = cx[WX] = wrap_index(w0 + rr, nW, g.bc[WX]);
      c[OX] = grp == 0 ? io : io1;
      cx[OX] = wrap_index(c[OX] - 1, nO, g.bc[OX]);
    }
    const long long gi = c[0] * g.s[0] + c[1] * g.s[1] + c[2] * g.s[2];
    const long long gx = cx[0] * g.s[0] + cx[1] * g.s[1] + cx[2] * g.s[2];
    sv[idx] = Num<T>::div(in.f[1 + A][gi] + in.f[1 + A][gx], in.f[0][gi] + in.f[0][gx]);
    sbt[idx] = in.f[5 + t][gi];
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < ER; idx += NT) {
    const int e = (A == 2) ? idx % E : idx / R;
    if (e < 1 || e >= E - 1) continue;
    ss[idx] = T(0.25) * (sv[idx + DS] + T(2) * sv[idx] + sv[idx - DS]);
  }
  __syncthreads();
  // first-order upwind EMF at the A-face e+1/2
  for (int idx = threadIdx.x; idx < ER; idx += NT) {
    const int e = (A == 2) ? idx % E : idx / R;
    if (e < 1 || e >= E - 2) continue;
    const T ve = T(0.5) * (ss[idx] + ss[idx + DS]);
    se[idx] = ve > T(0) ? ss[idx] * sbt[idx] : ss[idx + DS] * sbt[idx + DS];
  }
  __syncthreads();
  // B_t at t + dt/2 and g = vs B_half
  const T hd = T(0.5) * dth;
  for (int idx = threadIdx.x; idx < ER; idx += NT) {
    const int e = (A == 2) ? idx % E : idx / R;
    if (e < 2 || e >= E - 2) continue;
    const T bh = sbt[idx] - hd * (se[idx] - se[idx - DS]);
    sv[idx] = ss[idx] * bh;
  }
  __syncthreads();
  // limited second-order EMF at A-faces e+1/2, e in [G-1, G+S-1]
  for (int idx = threadIdx.x; idx < ER; idx += NT) {
    const int e = (A == 2) ? idx % E : idx / R;
    if (e < G - 1 || e > G + S - 1) continue;
    const T ve = T(0.5) * (ss[idx] + ss[idx + DS]);
    const T gm = sv[idx - DS], g0 = sv[idx], gp = sv[idx + DS], gpp = sv[idx + 2 * DS];
    se[idx] = ve > T(0) ? g0 + vanleer(T(0.5) * (g0 - gm), T(0.5) * (gp - g0))
                        : gp - vanleer(T(0.5) * (gp - g0), T(0.5) * (gpp - gp));
  }
  __syncthreads();
  // outputs: B_t advection for t1, t2 and the constraint on B_A (t1 first, then t2)
  int st = 0;
  for (int idx = threadIdx.x; idx < S * W; idx += NT) {
    const int ei = (A == 2) ? idx % S : idx / W;
    const int w = (A == 2) ? idx / S : idx % W;
    const int ia = a0 + ei;
    if (ia >= nA || w0 + w >= nW) continue;
    const int e = ei + G;
    int c[3];
    c[A] = ia;
    c[WX] = w0 + w;
    c[OX] = io;
    const long long gi = c[0] * g.s[0] + c[1] * g.s[1] + c[2] * g.s[2];
    auto at = [&](int row, int ee) -> T {
      return (A == 2) ? se[row * E + ee] : se[ee * R + row];
    };
    const int rW0 = w, rW1 = w + 1;              // group 0 rows (t = WX)
    const int rO0 = W + 1 + w, rO1 = 2 * W + 1 + w;  // groups 1 and 2 (t = OX)
    const T bw = in.f[5 + WX][gi] - dth * (at(rW0, e) - at(rW0, e - 1));
    const T bo = in.f[5 + OX][gi] - dth * (at(rO0, e) - at(rO0, e - 1));
    const T dW = dth * (at(rW1, e - 1) - at(rW0, e - 1));
    const T dO = dth * (at(rO1, e - 1) - at(rO0, e - 1));
    T ba = in.f[5 + A][gi];
    if (T1 == WX) { ba = ba + dW; ba = ba + dO; }
    else { ba = ba + dO; ba = ba + dW; }
    out.f[5 + WX][gi] = bw;
    out.f[5 + OX][gi] = bo;
    out.f[5 + A][gi] = ba;
    if (!(bw == bw) || !(bo == bo) || !(ba == ba)) st |= ST_NONFINITE;
  }
  if (st) atomicOr(&ds->status, st);
}

// ------------------------------------------------------------------------------------
// auxiliary kernels
// ------------------------------------------------------------------------------------

// c_max of a state (used at initialisation and on request)
template <typename T, bool P64>
__global__ void cmax_kernel(GridDesc g, FieldSet<T> in, T gamma, DevScalars* ds) {
  const long long N = (long long)g.n[0] * g.n[1] * g.n[2];
  T cm = T(0);
  bool nan_seen = false;
  int st = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
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
    const T v = cell_cmax<T, P64>(in.f[0][i], in.f[1][i], in.f[2][i], in.f[3][i], in.f[4][i],
                                  bc[0], bc[1], bc[2], gamma, &st);
    if (v != v) nan_seen = true; else cm = fmax(cm, v);
  }
  block_max_to_global(cm, nan_seen, ds);
  if (st) atomicOr(&ds->status, st);
}

// dt = cfl h / c_max on the device, clipped to land on t_end (Sect. 4.2 steps 4-5, 8-9)
template <typename T>
__global__ void dt_kernel(DevScalars* ds, double cfl_h) {
  const double cm = Num<T>::from_bits(ds->cmax);
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
  if (active) {
    ds->t = clipped ? ds->t_end : ds->t + 2.0 * dt;
    ds->dt_last = dt;
    ds->steps_done += 1;
  }
  ds->cmax = 0ull;   // the last sweep of this step accumulates the next c_max
}

// FP64 conservation sums: per-block partial sums (deterministic two-pass reduction)
template <typename T>
__global__ void sums_partial_kernel(long long N, FieldSet<T> in, double* partial) {
  __shared__ double red[8][32];
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] += (double)in.f[k][i];
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
