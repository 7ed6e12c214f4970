// Sweeps along an axis of one cell (2D grids with nz = 1, 1D grids with ny = nz = 1).
//
// Along such an axis every neighbour of a cell is the cell itself (periodic wrap or
// outflow clamp alike), so:
//  - the fluid sweep (Algorithm 1) computes both interface fluxes of a cell from the same
//    values in the same order: they are equal, their difference is exactly 0 and
//    u^{t+dt} = u^t bit for bit.  The sweep is skipped; when it is the last one of a step,
//    c_max is taken from the unchanged state instead (cmax_kernel);
//  - the constrained transport along A (Algorithm 2) leaves B_t1 and B_t2 unchanged (their
//    EMF differences along A vanish) but still updates B_A from the differences of the EMF
//    across the transverse faces (Eq. "eq:first_flux" with every A-neighbour equal).  With
//    constant inputs along A the smoothed velocity (1,2,1)/4 and the edge average return the
//    face velocity exactly, the half-step B_t equals B_t, the limiter sees zero slopes, and
//    the EMF of a transverse row is the product of its face velocity and its B_t.  ct_flat
//    evaluates just that, per cell, and writes B_A only.
#pragma once

#include "mhd_kernels.cuh"

namespace mhd {

__host__ __device__ __forceinline__ bool axis_is_flat(const GridDesc& g, int a) {
  return g.n[a] == 1;
}

// B_A of cell i after the constrained transport along a flat axis A.  The face velocities
// and the EMF are the expressions of the marching CT with every A-neighbour equal.
template <typename T, int A>
__device__ __forceinline__ T ct_flat_cell(const GridDesc& g, const FieldSet<T>& in, T dth,
                                          long long i) {
  constexpr int T1 = axis_t1(A), T2 = axis_t2(A);
  const int z = (int)(i % g.n[2]);
  const long long xy = i / g.n[2];
  const int y = (int)(xy % g.n[1]);
  const int x = (int)(xy / g.n[1]);
  const int c[3] = {x, y, z};
  const T* __restrict__ pr = in.f[0];
  const T* __restrict__ pm = in.f[1 + A];
  T e[2][2];   // [t][own, upper row]
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int t = q == 0 ? T1 : T2;
    const int ct = c[t];
    const int lo = wrap_index(ct - 1, g.n[t], g.bc[t]), hi = wrap_index(ct + 1, g.n[t], g.bc[t]);
    const long long ilo = i + (long long)(lo - ct) * g.s[t];
    const long long ihi = i + (long long)(hi - ct) * g.s[t];
    // the upper row's lower neighbour: the cell itself, or (clamped at the top) the lower row
    const long long iha = (wrap_index(hi - 1, g.n[t], g.bc[t]) != ct) ? ilo : i;
    const T vo = Num<T>::div(pm[i] + pm[ilo], pr[i] + pr[ilo]);
    const T vn = Num<T>::div(pm[ihi] + pm[iha], pr[ihi] + pr[iha]);
    const T* __restrict__ pb = in.f[5 + t];
    e[q][0] = Num<T>::mul_rn(vo, pb[i]);
    e[q][1] = Num<T>::mul_rn(vn, pb[ihi]);
  }
  T b = ffma(dth, e[0][1] - e[0][0], in.f[5 + A][i]);   // constraint from t1, then t2
  b = ffma(dth, e[1][1] - e[1][0], b);
  return b;
}

// cells [i0, i1) with stride; returns ST_NONFINITE if an output is not finite
template <typename T, int A>
__device__ __forceinline__ int ct_flat_range(const GridDesc& g, const FieldSet<T>& in,
                                             const FieldSet<T>& out, T dth, long long i0,
                                             long long i1, long long stride) {
  int st = 0;
  for (long long i = i0; i < i1; i += stride) {
    const T b = ct_flat_cell<T, A>(g, in, dth, i);
    out.f[5 + A][i] = b;
    if (!(b == b)) st |= ST_NONFINITE;
  }
  return st;
}

template <typename T, int A>
__global__ void ct_flat_kernel(GridDesc g, FieldSet<T> in, FieldSet<T> out, double h,
                               DevScalars* ds) {
  const long long N = (long long)g.n[0] * g.n[1] * g.n[2];
  const T dth = step_factor<T>(ds, h);
  const int st = ct_flat_range<T, A>(g, in, out, dth,
                                     blockIdx.x * (long long)blockDim.x + threadIdx.x, N,
                                     (long long)gridDim.x * blockDim.x);
  if (st) atomicOr(&ds->status, st);
}

}  // namespace mhd
