// C ABI of the solver (include/mhd.h): context, device state, step sequencing on the
// device, CUDA-graph replay of whole steps.
//
// Step (Sect. 4.2 steps 4-8, Eq. "eq:L_sequence"): a one-thread kernel turns the c_max
// left by the previous step into dt (clipped to t_end) and advances t; then the forward
// sweep applies, for the axis order (a, b, c) of the current phase, fluid_a, CT_a,
// fluid_b, CT_b, fluid_c, CT_c, and the reverse sweep CT_c, fluid_c, CT_b, fluid_b, CT_a,
// fluid_a (reverse L: magnetic updates first, Sect. 4.3); the two CT_c in the middle run as
// one launch where a two-pass kernel exists (z; x and y in the shared-row form, periodic).  The last fluid sweep also reduces the next c_max.  Each sweep is
// out of place; the context tracks which of the two buffers holds each field.  A step's
// launch sequence depends on the phase and on the buffer state it starts from, which
// alternates between two states (a middle CT pair in one launch flips the B buffers once), so
// each phase keeps up to two captured CUDA graphs.
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include "../../include/mhd.h"
#include "mhd_flat.cuh"
#include "mhd_kernels.cuh"
#include "mhd_launch.h"
#include "mhd_tma.cuh"

using mhd::DevScalars;
using mhd::FieldSet;
using mhd::GridDesc;
using mhd::Launch;

#include "mhd_ctx.h"

// kinds: 0..2 fluid along x,y,z; 3..5 CT along x,y,z; 6 dt; 7 other
static cudaEvent_t take_event(mhd_ctx* ctx) {
  if (!ctx->free_events.empty()) {
    cudaEvent_t e = ctx->free_events.back();
    ctx->free_events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

struct ProfScope {
  mhd_ctx* ctx;
  int kind;
  cudaEvent_t a = nullptr, b = nullptr;
  ProfScope(mhd_ctx* c, int k) : ctx(c), kind(k) {
    if (ctx->profile) {
      a = take_event(ctx);
      b = take_event(ctx);
      cudaEventRecord(a, ctx->stream);
    }
  }
  ~ProfScope() {
    if (ctx->profile) {
      cudaEventRecord(b, ctx->stream);
      ctx->pending.push_back({kind, a, b});
    }
  }
};


static mhd_status cuda_fail(mhd_ctx* c, cudaError_t e, const char* what) {
  if (c) {
    c->err = std::string(what) + ": " + cudaGetErrorString(e);
  }
  return MHD_ERR_CUDA;
}

#define CK(call, what)                                           \
  do {                                                           \
    cudaError_t _e = (call);                                     \
    if (_e != cudaSuccess) return cuda_fail(ctx, _e, what);      \
  } while (0)

template <typename T>
static FieldSet<T> fields_of(mhd_ctx* ctx, bool other) {
  FieldSet<T> fs;
  for (int k = 0; k < 8; ++k) fs.f[k] = (T*)ctx->buf[other ? 1 - ctx->cur[k] : ctx->cur[k]][k];
  return fs;
}

static unsigned cur_sig(const mhd_ctx* ctx) {
  unsigned s = 0;
  for (int k = 0; k < 8; ++k) s |= (unsigned)ctx->cur[k] << k;
  return s | 0x100u;
}

template <typename T>
static cudaError_t enqueue_fluid(mhd_ctx* ctx, int axis, bool last) {
  ProfScope ps(ctx, axis);
  FieldSet<T> in = fields_of<T>(ctx, false), out = fields_of<T>(ctx, true);
  mhd::TmaMaps maps;
  if (ctx->tma)
    for (int k = 0; k < 8; ++k) {
      maps.one[k] = ctx->tmap_one[ctx->cur[k]][k];
      maps.gx[k] = ctx->tmap_gx[ctx->cur[k]][k];
      maps.gy[k] = ctx->tmap_gy[ctx->cur[k]][k];
    }
  cudaError_t e = Launch<T>::fluid(ctx->g, in, out, ctx->cfg.gamma, ctx->cfg.h, ctx->ds, axis,
                                   last, ctx->cfg.fp64_pressure, ctx->stream,
                                   ctx->tma ? &maps : nullptr);
  if (!mhd::axis_is_flat(ctx->g, axis))   // along a flat axis the sweep is the identity
    for (int k = 0; k < 5; ++k) ctx->cur[k] ^= 1;
  return e;
}

template <typename T>
static cudaError_t enqueue_ct(mhd_ctx* ctx, int axis) {
  ProfScope ps(ctx, 3 + axis);
  FieldSet<T> in = fields_of<T>(ctx, false), out = fields_of<T>(ctx, true);
  cudaError_t e = Launch<T>::ct(ctx->g, in, out, ctx->cfg.h, ctx->ds, axis, ctx->stream);
  if (mhd::axis_is_flat(ctx->g, axis)) ctx->cur[5 + axis] ^= 1;   // only B_A changes
  else for (int k = 5; k < 8; ++k) ctx->cur[k] ^= 1;
  return e;
}

// the middle CT pair of a step runs as one launch where a two-pass kernel exists
// (MHD_PAIR = 1) or always as two (0)
#ifndef MHD_PAIR
#define MHD_PAIR 1
#endif
static constexpr bool kPair = MHD_PAIR != 0;

// CT along axis twice: one launch where a two-pass kernel exists (the same bits as two
// enqueue_ct), else two launches
template <typename T>
static cudaError_t enqueue_ct2(mhd_ctx* ctx, int axis) {
  if (kPair && !mhd::axis_is_flat(ctx->g, axis)) {
    FieldSet<T> in = fields_of<T>(ctx, false), out = fields_of<T>(ctx, true);
    cudaError_t e;
    {
      ProfScope ps(ctx, 3 + axis);
      e = Launch<T>::ct2(ctx->g, in, out, ctx->cfg.h, ctx->ds, axis, ctx->stream);
    }
    if (e == cudaSuccess) {
      for (int k = 5; k < 8; ++k) ctx->cur[k] ^= 1;
      return e;
    }
    if (e != cudaErrorNotSupported) return e;   // (no kernel launched: nothing to clear)
  }
  cudaError_t e = enqueue_ct<T>(ctx, axis);
  return e != cudaSuccess ? e : enqueue_ct<T>(ctx, axis);
}

// the reverse L along axis (CT, then fluid) in one launch; cudaErrorNotSupported (nothing
// launched) where the library has no such kernel
template <typename T>
static cudaError_t enqueue_ct_fluid(mhd_ctx* ctx, int axis) {
  FieldSet<T> in = fields_of<T>(ctx, false), out = fields_of<T>(ctx, true);
  cudaError_t e;
  {
    ProfScope ps(ctx, 7);
    e = Launch<T>::ct_fluid(ctx->g, in, out, ctx->cfg.gamma, ctx->cfg.h, ctx->ds, axis,
                            ctx->cfg.fp64_pressure, ctx->stream);
  }
  if (e == cudaSuccess)
    for (int k = 0; k < 8; ++k) ctx->cur[k] ^= 1;
  return e;
}

template <typename T>
static cudaError_t enqueue_step_t(mhd_ctx* ctx, int phase) {
  cudaError_t e;
  {
    ProfScope ps(ctx, 6);
    e = Launch<T>::dt(ctx->ds, ctx->cfg.cfl * ctx->cfg.h, ctx->cfg.h, ctx->stream);
  }
  if (e != cudaSuccess) return e;
  const int* o = kOrder[phase];
  // the two CT operators of the middle axis meet (forward L ends with CT, reverse L starts
  // with it): they run as one launch where a two-pass kernel exists (the same bits, one pass
  // over memory less)
  for (int k = 0; k < 3; ++k) {
    if ((e = enqueue_fluid<T>(ctx, o[k], false)) != cudaSuccess) return e;
    if (k == 2) {
      if ((e = enqueue_ct2<T>(ctx, o[k])) != cudaSuccess) return e;
    } else if ((e = enqueue_ct<T>(ctx, o[k])) != cudaSuccess) {
      return e;
    }
  }
  for (int k = 2; k >= 0; --k) {
    if (k != 2)
      if ((e = enqueue_ct<T>(ctx, o[k])) != cudaSuccess) return e;
    if ((e = enqueue_fluid<T>(ctx, o[k], k == 0)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

static cudaError_t enqueue_step(mhd_ctx* ctx, int phase) {
  return ctx->esz == 4 ? enqueue_step_t<float>(ctx, phase) : enqueue_step_t<double>(ctx, phase);
}

// one step through the per-phase graph (captured on first use for this buffer state)
static mhd_status launch_step(mhd_ctx* ctx) {
  const int ph = ctx->phase;
  if (ctx->profile) {
    CK(enqueue_step(ctx, ph), "profiled step");
    ctx->phase = (ph + 1) % 3;
    return MHD_OK;
  }
  const unsigned sig = cur_sig(ctx);
  mhd_ctx::StepGraph* sg = nullptr;
  for (auto& c : ctx->graph[ph])
    if (c.exec && c.sig_in == sig) sg = &c;
  if (!sg) {
    sg = &ctx->graph[ph][ctx->graph_next[ph]];
    ctx->graph_next[ph] ^= 1;
    if (sg->exec) {
      cudaGraphExecDestroy(sg->exec);
      sg->exec = nullptr;
    }
    const int cur0[8] = {ctx->cur[0], ctx->cur[1], ctx->cur[2], ctx->cur[3],
                         ctx->cur[4], ctx->cur[5], ctx->cur[6], ctx->cur[7]};
    cudaGraph_t gr = nullptr;
    CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    cudaError_t e = enqueue_step(ctx, ph);
    cudaError_t e2 = cudaStreamEndCapture(ctx->stream, &gr);
    const unsigned sig_out = cur_sig(ctx);
    for (int k = 0; k < 8; ++k) ctx->cur[k] = cur0[k];   // applied below, with the launch
    if (e != cudaSuccess) { if (gr) cudaGraphDestroy(gr); return cuda_fail(ctx, e, "capture step"); }
    if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "end capture");
    e = cudaGraphInstantiate(&sg->exec, gr, 0);
    cudaGraphDestroy(gr);
    if (e != cudaSuccess) { sg->exec = nullptr; return cuda_fail(ctx, e, "instantiate"); }
    sg->sig_in = sig;
    sg->sig_out = sig_out;
  }
  CK(cudaGraphLaunch(sg->exec, ctx->stream), "graph launch");
  for (int k = 0; k < 8; ++k) ctx->cur[k] = (int)((sg->sig_out >> k) & 1u);
  ctx->phase = (ph + 1) % 3;
  return MHD_OK;
}

static mhd_status status_from(int st) {
  if (st & mhd::ST_TIMEOUT) return MHD_ERR_TIMEOUT;
  return st ? MHD_ERR_UNPHYSICAL : MHD_OK;
}

// synchronise and pull the device scalars into the host mirror
static mhd_status sync_scalars(mhd_ctx* ctx) {
  CK(cudaMemcpyAsync(ctx->hs, ctx->ds, sizeof(DevScalars), cudaMemcpyDeviceToHost, ctx->stream),
     "read scalars");
  CK(cudaStreamSynchronize(ctx->stream), "synchronize");
  ctx->status |= ctx->hs->status;
  return MHD_OK;
}

static mhd_status push_scalars(mhd_ctx* ctx) {
  CK(cudaMemcpyAsync(ctx->ds, ctx->hs, sizeof(DevScalars), cudaMemcpyHostToDevice, ctx->stream),
     "write scalars");
  CK(cudaStreamSynchronize(ctx->stream), "synchronize");
  return MHD_OK;
}

static mhd_status compute_cmax(mhd_ctx* ctx) {
  // cmax accumulator must be zero: the scalars were just pushed with cmax = 0
  FieldSet<float> f32;
  FieldSet<double> f64;
  cudaError_t e;
  if (ctx->esz == 4) {
    f32 = fields_of<float>(ctx, false);
    e = Launch<float>::cmax(ctx->g, f32, ctx->cfg.gamma, ctx->ds, ctx->cfg.fp64_pressure,
                            ctx->stream);
  } else {
    f64 = fields_of<double>(ctx, false);
    e = Launch<double>::cmax(ctx->g, f64, ctx->cfg.gamma, ctx->ds, 0, ctx->stream);
  }
  CK(e, "cmax");
  return MHD_OK;
}

// Tensor maps of the state buffers for the TMA-staged sweeps: each buffer as a 3D FP32 tensor
// (z, y, x) with boxes of 128 x 1 x 1 elements.  The encoding entry point comes from the
// driver through the runtime (no link-time dependency on the driver library).  Any failure
// leaves ctx->tma false (the sweeps then use the cp.async staging).
static void make_tensor_maps(mhd_ctx* ctx) {
  ctx->tma = false;
  if (!MHD_TMA_MARCH || ctx->esz != 4 || ctx->g.n[2] % 128 != 0) return;
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const cuuint64_t dims[3] = {(cuuint64_t)ctx->g.n[2], (cuuint64_t)ctx->g.n[1],
                              (cuuint64_t)ctx->g.n[0]};
  const cuuint64_t strides[2] = {(cuuint64_t)ctx->g.n[2] * 4,
                                 (cuuint64_t)ctx->g.n[2] * ctx->g.n[1] * 4};
  const cuuint32_t G = mhd::kTmaG;
  const cuuint32_t box_one[3] = {128, 1, 1}, box_gx[3] = {128, 1, G}, box_gy[3] = {128, G, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  auto enc = [&](CUtensorMap* m, void* base, const cuuint32_t* box) {
    return encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  };
  for (int b = 0; b < 2; ++b)
    for (int k = 0; k < 8; ++k)
      if (!enc(&ctx->tmap_one[b][k], ctx->buf[b][k], box_one) ||
          !enc(&ctx->tmap_gx[b][k], ctx->buf[b][k], box_gx) ||
          !enc(&ctx->tmap_gy[b][k], ctx->buf[b][k], box_gy))
        return;
  ctx->tma = true;
}

extern "C" {

const char* mhd_status_str(mhd_status s) {
  switch (s) {
    case MHD_OK: return "ok";
    case MHD_ERR_INVALID: return "invalid argument";
    case MHD_ERR_OOM: return "out of device memory";
    case MHD_ERR_CUDA: return "CUDA error";
    case MHD_ERR_UNPHYSICAL: return "unphysical state (rho <= 0, non-finite, or negative fast-speed radicand)";
    case MHD_ERR_TIMEOUT: return "device wait timed out";
  }
  return "unknown status";
}

const char* mhd_last_error(const mhd_ctx* ctx) { return ctx ? ctx->err.c_str() : "no context"; }

void mhd_destroy(mhd_ctx* ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  for (auto& p : ctx->pending) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
  for (auto e : ctx->free_events) cudaEventDestroy(e);
  for (int p = 0; p < 3; ++p)
    for (auto& c : ctx->graph[p])
      if (c.exec) cudaGraphExecDestroy(c.exec);
  for (int b = 0; b < 2; ++b)
    for (int k = 0; k < 8; ++k)
      if (ctx->buf[b][k]) cudaFree(ctx->buf[b][k]);
  if (ctx->staging) cudaFree(ctx->staging);
  if (ctx->ds) cudaFree(ctx->ds);
  if (ctx->partial) cudaFree(ctx->partial);
  if (ctx->sums_out) cudaFree(ctx->sums_out);
  if (ctx->hs) cudaFreeHost(ctx->hs);
  if (ctx->sums_host) cudaFreeHost(ctx->sums_host);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

static mhd_status validate(const mhd_config* c) {
  if (!c) return MHD_ERR_INVALID;
  if (c->nx < 1 || c->ny < 1 || c->nz < 1) return MHD_ERR_INVALID;
  if (c->ny > 65535 * 8 || c->nz > 65535 * 8 || c->nx > 65535) return MHD_ERR_INVALID;
  if (!(c->h > 0) || !(c->gamma > 1) || !(c->cfl > 0) || !(c->cfl < 1)) return MHD_ERR_INVALID;
  for (int a = 0; a < 3; ++a)
    if (c->bc[a] != MHD_BC_PERIODIC && c->bc[a] != MHD_BC_OUTFLOW) return MHD_ERR_INVALID;
  if (c->prec != MHD_FP32 && c->prec != MHD_FP64) return MHD_ERR_INVALID;
  if (c->fp64_pressure < MHD_PRESSURE_FP32 || c->fp64_pressure > MHD_PRESSURE_COMPENSATED)
    return MHD_ERR_INVALID;
  if (c->prec == MHD_FP64 && c->fp64_pressure) return MHD_ERR_INVALID;
  return MHD_OK;
}

mhd_status mhd_create(const mhd_config* cfg, mhd_ctx** out) {
  if (!out) return MHD_ERR_INVALID;
  *out = nullptr;
  mhd_status v = validate(cfg);
  if (v != MHD_OK) return v;
  mhd_ctx* ctx = new mhd_ctx();
  ctx->cfg = *cfg;
  ctx->esz = cfg->prec == MHD_FP32 ? 4 : 8;
  const int n[3] = {cfg->nx, cfg->ny, cfg->nz};
  for (int a = 0; a < 3; ++a) {
    ctx->g.n[a] = n[a];
    ctx->g.bc[a] = cfg->bc[a];
  }
  ctx->g.s[2] = 1;
  ctx->g.s[1] = n[2];
  ctx->g.s[0] = (long long)n[1] * n[2];
  ctx->N = (long long)n[0] * n[1] * n[2];
  auto fail = [&](mhd_status s) { mhd_destroy(ctx); return s; };
  cudaError_t e;
  static bool attrs_done[2] = {false, false};
  const int pi = cfg->prec == MHD_FP32 ? 0 : 1;
  if (!attrs_done[pi]) {
    e = pi == 0 ? Launch<float>::setup() : Launch<double>::setup();
    if (e != cudaSuccess) { cuda_fail(ctx, e, "kernel setup"); return fail(MHD_ERR_CUDA); }
    attrs_done[pi] = true;
  }
  if (cfg->cuda_stream) {
    ctx->stream = (cudaStream_t)cfg->cuda_stream;
  } else {
    e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { cuda_fail(ctx, e, "stream"); return fail(MHD_ERR_CUDA); }
    ctx->own_stream = true;
  }
  const size_t fb = (size_t)ctx->N * ctx->esz;
  for (int b = 0; b < 2; ++b)
    for (int k = 0; k < 8; ++k) {
      e = cudaMalloc(&ctx->buf[b][k], fb);
      if (e != cudaSuccess) { cuda_fail(ctx, e, "state allocation"); return fail(MHD_ERR_OOM); }
      ctx->dev_bytes += (long long)fb;
    }
  make_tensor_maps(ctx);
  e = cudaMalloc(&ctx->staging, (size_t)ctx->N * sizeof(double));
  if (e != cudaSuccess) { cuda_fail(ctx, e, "staging allocation"); return fail(MHD_ERR_OOM); }
  ctx->dev_bytes += (long long)ctx->N * 8;
  long long nb = (ctx->N + 255) / 256;
  ctx->sum_blocks = (int)(nb < 152 * 8 ? nb : 152 * 8);
  e = cudaMalloc(&ctx->partial, sizeof(double) * 8 * ctx->sum_blocks);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->sums_out, sizeof(double) * 8);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->ds, sizeof(DevScalars));
  if (e != cudaSuccess) { cuda_fail(ctx, e, "scratch allocation"); return fail(MHD_ERR_OOM); }
  ctx->dev_bytes += (long long)sizeof(double) * 8 * (ctx->sum_blocks + 1) + sizeof(DevScalars);
  e = cudaMallocHost(&ctx->hs, sizeof(DevScalars));
  if (e == cudaSuccess) e = cudaMallocHost(&ctx->sums_host, sizeof(double) * 8);
  if (e != cudaSuccess) { cuda_fail(ctx, e, "pinned allocation"); return fail(MHD_ERR_OOM); }
  memset(ctx->hs, 0, sizeof(DevScalars));
  ctx->hs->t_end = -1.0;
  if (push_scalars(ctx) != MHD_OK) return fail(MHD_ERR_CUDA);
  *out = ctx;
  return MHD_OK;
}

static mhd_status reset_after_load(mhd_ctx* ctx, double t0) {
  memset(ctx->hs, 0, sizeof(DevScalars));
  ctx->hs->t = t0;
  ctx->hs->t_end = -1.0;
  ctx->status = 0;
  ctx->phase = 0;
  ctx->step = 0;
  ctx->steps_base = 0;
  mhd_status s = push_scalars(ctx);
  if (s != MHD_OK) return s;
  if ((s = compute_cmax(ctx)) != MHD_OK) return s;
  if ((s = sync_scalars(ctx)) != MHD_OK) return s;
  return status_from(ctx->status);
}

mhd_status mhd_upload(mhd_ctx* ctx, const void* const f[8], int dtype, int on_device, double t0) {
  if (!ctx || !f || (dtype != 0 && dtype != 1)) return MHD_ERR_INVALID;
  for (int k = 0; k < 8; ++k)
    if (!f[k]) return MHD_ERR_INVALID;
  const size_t srcsz = dtype == 0 ? 4 : 8;
  const int want = ctx->esz == 4 ? 0 : 1;
  for (int k = 0; k < 8; ++k) {
    ctx->cur[k] = 0;
    void* dst = ctx->buf[0][k];
    if (dtype == want) {
      CK(cudaMemcpyAsync(dst, f[k], (size_t)ctx->N * srcsz,
                         on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream),
         "upload copy");
      continue;
    }
    const void* src = f[k];
    if (!on_device) {
      CK(cudaMemcpyAsync(ctx->staging, f[k], (size_t)ctx->N * srcsz, cudaMemcpyHostToDevice,
                         ctx->stream), "upload staging copy");
      src = ctx->staging;
    }
    cudaError_t e = ctx->esz == 4 ? Launch<float>::from(src, dtype, (float*)dst, ctx->N, ctx->stream)
                                  : Launch<double>::from(src, dtype, (double*)dst, ctx->N, ctx->stream);
    CK(e, "upload convert");
  }
  return reset_after_load(ctx, t0);
}

mhd_status mhd_init_fields(mhd_ctx* ctx, const double* const f[8], double t0) {
  return mhd_upload(ctx, (const void* const*)f, 1, 0, t0);
}

mhd_status mhd_download(mhd_ctx* ctx, void* const f[8], int dtype, int on_device) {
  if (!ctx || !f || (dtype != 0 && dtype != 1)) return MHD_ERR_INVALID;
  for (int k = 0; k < 8; ++k)
    if (!f[k]) return MHD_ERR_INVALID;
  const size_t dsz = dtype == 0 ? 4 : 8;
  const int have = ctx->esz == 4 ? 0 : 1;
  for (int k = 0; k < 8; ++k) {
    const void* src = ctx->buf[ctx->cur[k]][k];
    if (dtype == have) {
      CK(cudaMemcpyAsync(f[k], src, (size_t)ctx->N * dsz,
                         on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream),
         "download copy");
      continue;
    }
    void* dst = on_device ? f[k] : ctx->staging;
    cudaError_t e = ctx->esz == 4 ? Launch<float>::to((const float*)src, dst, dtype, ctx->N, ctx->stream)
                                  : Launch<double>::to((const double*)src, dst, dtype, ctx->N, ctx->stream);
    CK(e, "download convert");
    if (!on_device)
      CK(cudaMemcpyAsync(f[k], ctx->staging, (size_t)ctx->N * dsz, cudaMemcpyDeviceToHost,
                         ctx->stream), "download staging copy");
  }
  mhd_status s = sync_scalars(ctx);
  if (s != MHD_OK) return s;
  return status_from(ctx->status);
}

mhd_status mhd_read(mhd_ctx* ctx, double* const f[8]) {
  return mhd_download(ctx, (void* const*)f, 1, 0);
}

mhd_status mhd_step(mhd_ctx* ctx, int nsteps, double t_end, int* steps_done, double* t_now) {
  if (!ctx || nsteps < 0) return MHD_ERR_INVALID;
  mhd_status s;
  if (t_end < 0.0) {
    for (int k = 0; k < nsteps; ++k)
      if ((s = launch_step(ctx)) != MHD_OK) return s;
    ctx->step += nsteps;
    ctx->steps_base += nsteps;
    if (steps_done || t_now) {
      if ((s = sync_scalars(ctx)) != MHD_OK) return s;
      if (steps_done) *steps_done = nsteps;
      if (t_now) *t_now = ctx->hs->t;
    }
    return status_from(ctx->status);
  }
  // bounded run to t_end: launch chunks sized from the last dt, watch t between chunks.
  // Steps launched after t reached t_end are exact no-ops on the device (dt = 0), and the
  // phase is re-based on the device's count of steps that advanced t.
  if ((s = sync_scalars(ctx)) != MHD_OK) return s;
  ctx->hs->t_end = t_end;
  CK(cudaMemcpyAsync(&ctx->ds->t_end, &ctx->hs->t_end, sizeof(double), cudaMemcpyHostToDevice,
                     ctx->stream), "t_end");
  const int base = ctx->hs->steps_done;
  const int phase0 = ctx->phase;
  int launched = 0, real = 0;
  while (real < nsteps) {
    if ((s = sync_scalars(ctx)) != MHD_OK) return s;
    real = ctx->hs->steps_done - base;
    if (ctx->hs->t >= t_end || real >= nsteps || ctx->status) break;
    const double dtl = ctx->hs->dt_last;
    int k = 1;
    if (dtl > 0.0) {
      const double est = (t_end - ctx->hs->t) / (2.0 * dtl);
      if (est > 8.0) k = (int)(0.5 * est);
    }
    if (k > nsteps - real) k = nsteps - real;
    if (k > 64) k = 64;
    ctx->phase = (phase0 + real) % 3;
    for (int j = 0; j < k; ++j)
      if ((s = launch_step(ctx)) != MHD_OK) return s;
    launched += k;
  }
  ctx->phase = (phase0 + real) % 3;
  ctx->step += real;
  ctx->hs->t_end = -1.0;
  CK(cudaMemcpyAsync(&ctx->ds->t_end, &ctx->hs->t_end, sizeof(double), cudaMemcpyHostToDevice,
                     ctx->stream), "t_end reset");
  if ((s = sync_scalars(ctx)) != MHD_OK) return s;
  if (steps_done) *steps_done = real;
  if (t_now) *t_now = ctx->hs->t;
  (void)launched;
  return status_from(ctx->status);
}

mhd_status mhd_apply(mhd_ctx* ctx, int op, int axis, double dt) {
  if (!ctx || axis < 0 || axis > 2 || op < 0 || op > 3) return MHD_ERR_INVALID;
  mhd_status s = sync_scalars(ctx);
  if (s != MHD_OK) return s;
  CK(cudaMemcpyAsync(&ctx->ds->dt, &dt, sizeof(double), cudaMemcpyHostToDevice, ctx->stream), "dt");
  const float dt_h = (float)(dt / ctx->cfg.h);    // as dt_update stores it
  CK(cudaMemcpyAsync(&ctx->ds->dt_h, &dt_h, sizeof(float), cudaMemcpyHostToDevice, ctx->stream),
     "dt/h");
  cudaError_t e;
  if (op == 3) {
    e = ctx->esz == 4 ? enqueue_ct_fluid<float>(ctx, axis) : cudaErrorNotSupported;
    if (e == cudaErrorNotSupported) {
      ctx->err = "mhd_apply: no one-launch reverse L for this context and axis";
      return MHD_ERR_INVALID;
    }
  } else if (ctx->esz == 4)
    e = op == 0 ? enqueue_fluid<float>(ctx, axis, false)
                : op == 1 ? enqueue_ct<float>(ctx, axis) : enqueue_ct2<float>(ctx, axis);
  else
    e = op == 0 ? enqueue_fluid<double>(ctx, axis, false)
                : op == 1 ? enqueue_ct<double>(ctx, axis) : enqueue_ct2<double>(ctx, axis);
  CK(e, "apply");
  CK(cudaStreamSynchronize(ctx->stream), "synchronize");
  return MHD_OK;
}

mhd_status mhd_cmax(mhd_ctx* ctx, double* cmax) {
  if (!ctx || !cmax) return MHD_ERR_INVALID;
  mhd_status s = sync_scalars(ctx);
  if (s != MHD_OK) return s;
  // recompute from the current state: the running maximum is replaced by the same value
  CK(cudaMemsetAsync(&ctx->ds->cmax, 0, sizeof(ctx->ds->cmax), ctx->stream), "zero");
  CK(cudaMemsetAsync(ctx->ds->cmax_part, 0, sizeof(ctx->ds->cmax_part), ctx->stream), "zero");
  if ((s = compute_cmax(ctx)) != MHD_OK) return s;
  if ((s = sync_scalars(ctx)) != MHD_OK) return s;
  const unsigned long long bits = mhd::fold_cmax_bits(*ctx->hs);
  *cmax = ctx->esz == 4 ? mhd::Num<float>::from_bits(bits) : mhd::Num<double>::from_bits(bits);
  return status_from(ctx->status);
}

mhd_status mhd_sums(mhd_ctx* ctx, double out[8]) {
  if (!ctx || !out) return MHD_ERR_INVALID;
  cudaError_t e;
  if (ctx->esz == 4)
    e = Launch<float>::sums(ctx->N, fields_of<float>(ctx, false), ctx->partial, ctx->sum_blocks,
                            ctx->sums_out, ctx->stream);
  else
    e = Launch<double>::sums(ctx->N, fields_of<double>(ctx, false), ctx->partial, ctx->sum_blocks,
                             ctx->sums_out, ctx->stream);
  CK(e, "sums");
  CK(cudaMemcpyAsync(ctx->sums_host, ctx->sums_out, 8 * sizeof(double), cudaMemcpyDeviceToHost,
                     ctx->stream), "sums copy");
  mhd_status s = sync_scalars(ctx);
  if (s != MHD_OK) return s;
  for (int k = 0; k < 8; ++k) out[k] = ctx->sums_host[k];
  return status_from(ctx->status);
}

mhd_status mhd_state(mhd_ctx* ctx, double* t, double* dt_last, int* step, int* phase) {
  if (!ctx) return MHD_ERR_INVALID;
  mhd_status s = sync_scalars(ctx);
  if (s != MHD_OK) return s;
  if (t) *t = ctx->hs->t;
  if (dt_last) *dt_last = ctx->hs->dt_last;
  if (step) *step = ctx->step;
  if (phase) *phase = ctx->phase;
  return status_from(ctx->status);
}

mhd_status mhd_set_state(mhd_ctx* ctx, double t, int step, int phase) {
  if (!ctx || phase < 0 || phase > 2 || step < 0) return MHD_ERR_INVALID;
  mhd_status s = sync_scalars(ctx);
  if (s != MHD_OK) return s;
  ctx->hs->t = t;
  CK(cudaMemcpyAsync(&ctx->ds->t, &ctx->hs->t, sizeof(double), cudaMemcpyHostToDevice, ctx->stream), "t");
  CK(cudaStreamSynchronize(ctx->stream), "synchronize");
  ctx->step = step;
  ctx->phase = phase;
  return MHD_OK;
}

mhd_status mhd_sync(mhd_ctx* ctx) {
  if (!ctx) return MHD_ERR_INVALID;
  mhd_status s = sync_scalars(ctx);
  if (s != MHD_OK) return s;
  return status_from(ctx->status);
}

mhd_status mhd_info(const mhd_ctx* ctx, long long* ncells, long long* device_bytes) {
  if (!ctx) return MHD_ERR_INVALID;
  if (ncells) *ncells = ctx->N;
  if (device_bytes) *device_bytes = ctx->dev_bytes;
  return MHD_OK;
}

mhd_status mhd_profile(mhd_ctx* ctx, int enable) {
  if (!ctx) return MHD_ERR_INVALID;
  ctx->profile = enable != 0;
  return MHD_OK;
}

mhd_status mhd_profile_read(mhd_ctx* ctx, double ms[8], long long count[8], int reset) {
  if (!ctx) return MHD_ERR_INVALID;
  CK(cudaStreamSynchronize(ctx->stream), "synchronize");
  for (auto& p : ctx->pending) {
    float v = 0.f;
    CK(cudaEventElapsedTime(&v, p.a, p.b), "event time");
    ctx->prof_ms[p.kind] += v;
    ctx->prof_n[p.kind] += 1;
    ctx->free_events.push_back(p.a);
    ctx->free_events.push_back(p.b);
  }
  ctx->pending.clear();
  for (int k = 0; k < 8; ++k) {
    if (ms) ms[k] = ctx->prof_ms[k];
    if (count) count[k] = ctx->prof_n[k];
    if (reset) { ctx->prof_ms[k] = 0.0; ctx->prof_n[k] = 0; }
  }
  return MHD_OK;
}

mhd_status mhd_stream(const mhd_ctx* ctx, void** stream) {
  if (!ctx || !stream) return MHD_ERR_INVALID;
  *stream = (void*)ctx->stream;
  return MHD_OK;
}

}  // extern "C"
