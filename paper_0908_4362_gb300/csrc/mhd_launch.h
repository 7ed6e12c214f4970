// Host-side launchers of the sweep kernels, one explicit instantiation per precision
// (kernels_f32.cu, kernels_f64.cu).  Internal to the library.
#pragma once

#include <cuda_runtime.h>

namespace mhd {

struct GridDesc;
struct DevScalars;
template <typename T> struct FieldSet;

template <typename T>
struct Launch {
  // one-time kernel attribute setup (dynamic shared memory opt-in); not capturable
  static cudaError_t setup();
  // fluid_axis(dt) with dt read from ds; last: also accumulate c_max of the result.
  // tmaps: NULL, or the tensor maps (TmaMaps, host memory) of the 8 input buffers, for the
  // TMA-staged x/y sweeps (FP32, nz a multiple of 128)
  static cudaError_t fluid(const GridDesc& g, const FieldSet<T>& in, const FieldSet<T>& out,
                           double gamma, double h, DevScalars* ds, int axis, bool last,
                           int pm, cudaStream_t s, const void* tmaps = nullptr);
  // CT along axis for both transverse components (t1 then t2)
  static cudaError_t ct(const GridDesc& g, const FieldSet<T>& in, const FieldSet<T>& out,
                        double h, DevScalars* ds, int axis, cudaStream_t s);
  // CT along axis applied twice in one launch (the middle pair of a step whose axis order
  // ends with that axis); cudaErrorNotSupported where there is no such kernel (a flat axis;
  // x/y outside the shared-row form or with an outflow sweep axis)
  static cudaError_t ct2(const GridDesc& g, const FieldSet<T>& in, const FieldSet<T>& out,
                         double h, DevScalars* ds, int axis, cudaStream_t s);
  // the reverse L along axis (CT, then the fluid sweep) in one launch; cudaErrorNotSupported
  // where there is no such kernel (FP64, an axis other than z, a flat z axis, a pressure mode
  // other than plain FP32)
  static cudaError_t ct_fluid(const GridDesc& g, const FieldSet<T>& in, const FieldSet<T>& out,
                              double gamma, double h, DevScalars* ds, int axis, int pm,
                              cudaStream_t s);
  static cudaError_t cmax(const GridDesc& g, const FieldSet<T>& in, double gamma,
                          DevScalars* ds, int pm, cudaStream_t s);
  static cudaError_t dt(DevScalars* ds, double cfl_h, double h, cudaStream_t s);
  static cudaError_t sums(long long n, const FieldSet<T>& in, double* partial, int nblocks,
                          double* out, cudaStream_t s);
  // dst (T) <- src (dtype 0 float, 1 double), device pointers
  static cudaError_t from(const void* src, int dtype, T* dst, long long n, cudaStream_t s);
  // dst (dtype) <- src (T), device pointers
  static cudaError_t to(const T* src, void* dst, int dtype, long long n, cudaStream_t s);
};

}  // namespace mhd
