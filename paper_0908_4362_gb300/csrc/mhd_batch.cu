// Batched persistent form: many grids (solver contexts of any shape) advanced by one
// persistent, graph-captured launch.  The launch keeps as many CTAs resident as the GPU
// holds; each CTA repeatedly takes the next work item (instance, operation, tile) from a
// device queue.  Items are laid out round by round (step, operation) over all instances, so
// that small grids fill the GPU together.  An item of operation k of an instance may start
// only when every item of that instance's earlier operations is complete: each instance
// has a completion counter, incremented with release semantics after an item and awaited
// with acquire semantics (bounded: after kSpinCycles the kernel records MHD_ERR_TIMEOUT,
// raises an abort flag that every CTA checks, and returns instead of hanging).
//
// The operations are those of one method step (Sect. 4.2, Eq. "eq:L_sequence"): dt from
// the previous step's c_max, then the forward and reverse sweeps of the instance's phase.
// Every tile runs the same device bodies as the standalone kernels (FP32), so each grid's
// result is bit-identical to advancing it alone with mhd_step.  Loads inside the
// persistent launch use coherent paths (no read-only cache), because the buffers are
// rewritten by other CTAs during the launch.
#include <algorithm>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/mhd.h"
#include "mhd_ctx.h"
#include "mhd_flat.cuh"
#include "mhd_march.cuh"
#include "mhd_segz.cuh"

namespace mhd {

constexpr int kBatchNT = 128;     // threads per CTA (all bodies use 128)
constexpr int kBatchS = kMarchS;  // march tile length along the sweep (as the single-grid kernels)
constexpr int kBatchK = 3;        // cells per lane of the z segments (or 2, seg_k_for)
constexpr long long kSpinCycles = 4000000000LL;   // ~2 s of SM clock per wait
constexpr int kFlatCells = kBatchNT * 16;   // cells per item of the per-cell operations
constexpr long long kAutoTiles = 1024;      // target items per z sweep when not set
// OP_NOP: a fluid sweep along a flat axis (identity, no items); OP_CMAX: c_max of the state
// (the last fluid sweep of a step along a flat axis); OP_CTFLAT: CT along a flat axis
enum : int { OP_DT = 0, OP_FLUID = 1, OP_CT = 2, OP_NOP = 3, OP_CMAX = 4, OP_CTFLAT = 5 };

constexpr int kBatchRowsR = kBatchNT / 32;   // warps of a shared-row CT tile

struct BatchOp {
  FieldSet<float> in, out;
  GridDesc g;
  int kind, axis, last;
  int rows;            // CT x/y in the shared-row form (ct_rows_xy_tile)
  int segk;            // z segments: cells per lane (2 or 3, seg_k_for)
  int gx;              // march: tiles across the transverse plane (tile = by * gx + bx)
  int wpt;             // z segments: warp segments per tile
  long long nwarps;    // z segments: warp segments of the sweep
  int tiles;
};
struct BatchItem {
  int inst, op, tile, need;
};
struct BatchInst {
  DevScalars* ds;
  float gamma;
  double h, cfl_h;
};
struct BatchArgs {
  const BatchItem* items;
  long long nitems;
  const BatchOp* ops;
  const BatchInst* inst;
  unsigned long long* queue;
  int* done;
  int* abort;
  int* status;
  long long spin_limit;
};

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_relaxed(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

template <int A>
__device__ __forceinline__ void batch_fluid_xy(const BatchOp& op, const BatchInst& in,
                                               unsigned tile, unsigned char* smem) {
  const unsigned bx = tile % op.gx, by = tile / op.gx;
  if (op.last)
    fluid_march_xy_tile<float, A, true, false, kBatchS, kBatchNT>(op.g, op.in, op.out, in.gamma,
                                                                  in.h, in.ds, bx, by, smem);
  else
    fluid_march_xy_tile<float, A, false, false, kBatchS, kBatchNT>(op.g, op.in, op.out, in.gamma,
                                                                   in.h, in.ds, bx, by, smem);
}

template <int A>
__device__ __forceinline__ void batch_ct_xy(const BatchOp& op, const BatchInst& in, unsigned tile,
                                            unsigned char* smem) {
  const unsigned bx = tile % op.gx, by = tile / op.gx;
  if (op.rows)
    ct_rows_xy_tile<float, A, kBatchS, kBatchRowsR>(op.g, op.in, op.out, in.h, in.ds, bx, by,
                                                    smem);
  else
    ct_march_xy_tile<float, A, kBatchS, kBatchNT>(op.g, op.in, op.out, in.h, in.ds, bx, by, smem);
}

// 4 resident CTAs per SM (a 128-register cap, with a few bytes of spill) measured 10%
// faster than 3 on the 64-instance batched workload
#ifndef MHD_BATCH_MINB
#define MHD_BATCH_MINB 4
#endif
__global__ void __launch_bounds__(kBatchNT, MHD_BATCH_MINB) batch_kernel(BatchArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ long long s_id;
  __shared__ int s_go;
  for (;;) {
    if (threadIdx.x == 0) {
      const long long id = (long long)atomicAdd(a.queue, 1ull);
      int go = id < a.nitems ? 1 : 0;
      if (go) {
        const BatchItem it = a.items[id];
        // poll with relaxed loads (cheaper than GPU-scope acquire loads, which must order
        // every later load of the SM), then one acquire load once the count is reached: it
        // reads a value of the counter's release sequence
        if (ld_acquire(a.done + it.inst) < it.need) {
          const long long t0 = clock64();
          while (ld_relaxed(a.done + it.inst) < it.need) {
            if (ld_relaxed(a.abort)) { go = 0; break; }
            if (clock64() - t0 > a.spin_limit) {
              atomicOr(a.status, 1);
              atomicExch(a.abort, 1);
              go = 0;
              break;
            }
            __nanosleep(64);
          }
          if (go) (void)ld_acquire(a.done + it.inst);
        }
      }
      s_id = id;
      s_go = go;
    }
    __syncthreads();
    if (!s_go) break;
    const BatchItem it = a.items[s_id];
    const BatchOp& op = a.ops[it.op];
    const BatchInst& ins = a.inst[it.inst];
    const int warp = threadIdx.x >> 5;
    if (op.kind == OP_DT) {
      if (threadIdx.x == 0) dt_update<float>(ins.ds, ins.cfl_h);
    } else if (op.kind == OP_CMAX || op.kind == OP_CTFLAT) {
      const long long N = (long long)op.g.n[0] * op.g.n[1] * op.g.n[2];
      const long long i0 = (long long)it.tile * kFlatCells;
      const long long i1 = min(i0 + kFlatCells, N);
      if (op.kind == OP_CMAX) {
        cmax_range<float, false>(op.g, op.in, ins.gamma, ins.ds, i0 + threadIdx.x, i1, kBatchNT);
      } else {
        const float dth = (float)(ins.ds->dt / ins.h);
        int st;
        if (op.axis == 0)
          st = ct_flat_range<float, 0>(op.g, op.in, op.out, dth, i0 + threadIdx.x, i1, kBatchNT);
        else if (op.axis == 1)
          st = ct_flat_range<float, 1>(op.g, op.in, op.out, dth, i0 + threadIdx.x, i1, kBatchNT);
        else
          st = ct_flat_range<float, 2>(op.g, op.in, op.out, dth, i0 + threadIdx.x, i1, kBatchNT);
        if (st) atomicOr(&ins.ds->status, st);
      }
    } else if (op.axis < 2) {
      if (op.kind == OP_FLUID) {
        if (op.axis == 0) batch_fluid_xy<0>(op, ins, it.tile, smem_raw);
        else batch_fluid_xy<1>(op, ins, it.tile, smem_raw);
      } else {
        if (op.axis == 0) batch_ct_xy<0>(op, ins, it.tile, smem_raw);
        else batch_ct_xy<1>(op, ins, it.tile, smem_raw);
      }
    } else {
      const long long w0 = (long long)it.tile * op.wpt;
      const long long w1 = min(w0 + op.wpt, op.nwarps);
      for (long long w = w0 + warp; w < w1; w += kBatchNT / 32) {
        if (op.segk == 2) {
          if (op.kind == OP_FLUID) {
            if (op.last)
              fluid_seg_z_warp<float, true, false, 2, false>(op.g, op.in, op.out, ins.gamma, ins.h,
                                                             ins.ds, w);
            else
              fluid_seg_z_warp<float, false, false, 2, false>(op.g, op.in, op.out, ins.gamma,
                                                              ins.h, ins.ds, w);
          } else {
            ct_seg_z_warp<float, 2, false>(op.g, op.in, op.out, ins.h, ins.ds, w);
          }
        } else {
          if (op.kind == OP_FLUID) {
            if (op.last)
              fluid_seg_z_warp<float, true, false, kBatchK, false>(op.g, op.in, op.out, ins.gamma,
                                                                   ins.h, ins.ds, w);
            else
              fluid_seg_z_warp<float, false, false, kBatchK, false>(op.g, op.in, op.out,
                                                                    ins.gamma, ins.h, ins.ds, w);
          } else {
            ct_seg_z_warp<float, kBatchK, false>(op.g, op.in, op.out, ins.h, ins.ds, w);
          }
        }
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(a.done + it.inst, 1);
    }
  }
}

}  // namespace mhd

using mhd::BatchArgs;
using mhd::BatchInst;
using mhd::BatchItem;
using mhd::BatchOp;

struct mhd_batch {
  std::vector<mhd_ctx*> ctx;
  std::vector<unsigned> sig;           // buffer state of each context when its ops were built
  std::vector<BatchOp> ops;            // [instance][phase][13]
  cudaStream_t stream = nullptr;
  int grid = 0;                        // resident CTAs of the persistent launch
  int wpt = 0;                         // z warp segments per tile (0: chosen per sweep)
  size_t smem = 0;
  BatchOp* d_ops = nullptr;
  BatchInst* d_inst = nullptr;
  BatchItem* d_items = nullptr;
  long long items_cap = 0;
  unsigned long long* d_queue = nullptr;
  int* d_done = nullptr;
  int* d_abort = nullptr;              // d_abort[0] abort flag, d_abort[1] status
  int* h_status = nullptr;             // pinned
  cudaEvent_t ev = nullptr;
  // graph per (nsteps, phases of the instances); items uploaded for the same key
  std::map<std::vector<int>, std::pair<cudaGraphExec_t, long long>> graphs;
  std::vector<int> items_key;
  std::string err;
};

static constexpr int kOpsPerStep = 13;

static mhd_status bfail(mhd_batch* b, cudaError_t e, const char* what) {
  if (b) b->err = std::string(what) + ": " + cudaGetErrorString(e);
  return MHD_ERR_CUDA;
}
#define BK(call, what)                                   \
  do {                                                   \
    cudaError_t _e = (call);                             \
    if (_e != cudaSuccess) return bfail(b, _e, what);    \
  } while (0)

static unsigned ctx_sig(const mhd_ctx* c) {
  unsigned s = 0;
  for (int k = 0; k < 8; ++k) s |= (unsigned)c->cur[k] << k;
  return s;
}

// the 13 operations of one step at `phase`, in launch order, with the buffers they read
// and write (mirrors enqueue_step_t in mhd_capi.cu)
static void build_step_ops(const mhd_ctx* c, int phase, int wpt, BatchOp* out) {
  int cur[8];
  for (int k = 0; k < 8; ++k) cur[k] = c->cur[k];
  auto fs = [&](bool other) {
    FieldSet<float> f;
    for (int k = 0; k < 8; ++k) f.f[k] = (float*)c->buf[other ? 1 - cur[k] : cur[k]][k];
    return f;
  };
  auto geometry = [&](BatchOp& op) {
    const GridDesc& g = c->g;
    if (op.axis < 2) {
      const int o = op.axis == 0 ? 1 : 0;
      const long long np = (long long)g.n[2] * g.n[o];
      op.rows = (op.kind == mhd::OP_CT && mhd::ct_use_rows(g, op.axis)) ? 1 : 0;
      op.gx = op.rows ? ((g.n[2] + 30) / 31) * ((g.n[o] + mhd::kBatchRowsR - 2) /
                                                (mhd::kBatchRowsR - 1))
                      : (int)((np + mhd::kBatchNT - 1) / mhd::kBatchNT);
      op.tiles = op.gx * ((g.n[op.axis] + mhd::kBatchS - 1) / mhd::kBatchS);
    } else {
      op.segk = mhd::seg_k_for(g.n[2]);
      const int seg = 32 * op.segk - (op.kind == mhd::OP_FLUID ? 6 : 8);
      op.nwarps = (long long)g.n[0] * g.n[1] * ((g.n[2] + seg - 1) / seg);
      // 0: about kAutoTiles items per z sweep (small grids get short items, large ones
      // up to 128 warp segments each)
      long long w = wpt > 0 ? wpt : (op.nwarps + mhd::kAutoTiles - 1) / mhd::kAutoTiles;
      w = w < 4 ? 4 : (w > 128 && wpt == 0 ? 128 : w);
      op.wpt = (int)w;
      op.tiles = (int)((op.nwarps + w - 1) / w);
    }
  };
  int n = 0;
  auto add = [&](int kind, int axis, bool last) {
    BatchOp op;
    std::memset(&op, 0, sizeof(op));
    op.g = c->g;
    op.kind = kind;
    op.axis = axis;
    op.last = last ? 1 : 0;
    op.in = fs(false);
    op.out = fs(true);
    const long long ncell = (long long)c->g.n[0] * c->g.n[1] * c->g.n[2];
    const int flat_tiles = (int)((ncell + mhd::kFlatCells - 1) / mhd::kFlatCells);
    if (kind == mhd::OP_DT) {
      op.tiles = 1;
    } else if (mhd::axis_is_flat(c->g, axis)) {
      // along a flat axis (mhd_flat.cuh): the fluid sweep is the identity, the CT changes B_A
      if (kind == mhd::OP_FLUID) {
        op.kind = last ? mhd::OP_CMAX : mhd::OP_NOP;
        op.tiles = last ? flat_tiles : 0;
        op.out = op.in;
      } else {
        op.kind = mhd::OP_CTFLAT;
        op.tiles = flat_tiles;
        cur[5 + axis] ^= 1;
      }
    } else {
      geometry(op);
      if (kind == mhd::OP_FLUID) for (int k = 0; k < 5; ++k) cur[k] ^= 1;
      else for (int k = 5; k < 8; ++k) cur[k] ^= 1;
    }
    out[n++] = op;
  };
  add(mhd::OP_DT, 0, false);
  const int* o = kOrder[phase];
  for (int k = 0; k < 3; ++k) {
    add(mhd::OP_FLUID, o[k], false);
    add(mhd::OP_CT, o[k], false);
  }
  for (int k = 2; k >= 0; --k) {
    add(mhd::OP_CT, o[k], false);
    add(mhd::OP_FLUID, o[k], k == 0);
  }
}

extern "C" {

void mhd_batch_destroy(mhd_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (auto& kv : b->graphs)
    if (kv.second.first) cudaGraphExecDestroy(kv.second.first);
  cudaFree(b->d_ops);
  cudaFree(b->d_inst);
  cudaFree(b->d_items);
  cudaFree(b->d_queue);
  cudaFree(b->d_done);
  cudaFree(b->d_abort);
  if (b->h_status) cudaFreeHost(b->h_status);
  if (b->ev) cudaEventDestroy(b->ev);
  if (b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

mhd_status mhd_batch_create(mhd_ctx* const* ctxs, int n, int z_tile_warps, int ctas_per_sm,
                            mhd_batch** out) {
  if (!out || !ctxs || n < 1) return MHD_ERR_INVALID;
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    const mhd_ctx* c = ctxs[i];
    if (!c || c->esz != 4 || c->cfg.fp64_pressure) return MHD_ERR_INVALID;
  }
  mhd_batch* b = new mhd_batch();
  b->wpt = z_tile_warps > 0 ? z_tile_warps : 0;
  b->ctx.assign(ctxs, ctxs + n);
  b->sig.resize(n);
  b->ops.resize((size_t)n * 3 * kOpsPerStep);
  for (int i = 0; i < n; ++i) {
    b->sig[i] = ctx_sig(ctxs[i]);
    for (int p = 0; p < 3; ++p)
      build_step_ops(ctxs[i], p, b->wpt, &b->ops[((size_t)i * 3 + p) * kOpsPerStep]);
  }
  std::vector<BatchInst> inst(n);
  for (int i = 0; i < n; ++i) {
    inst[i].ds = ctxs[i]->ds;
    inst[i].gamma = (float)ctxs[i]->cfg.gamma;
    inst[i].h = ctxs[i]->cfg.h;
    inst[i].cfl_h = ctxs[i]->cfg.cfl * ctxs[i]->cfg.h;
  }
  auto fail = [&](mhd_status s) { mhd_batch_destroy(b); return s; };
  cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_ops, sizeof(BatchOp) * b->ops.size());
  if (e == cudaSuccess) e = cudaMalloc(&b->d_inst, sizeof(BatchInst) * n);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_queue, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_done, sizeof(int) * n);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_abort, sizeof(int) * 2);
  if (e == cudaSuccess) e = cudaMallocHost(&b->h_status, sizeof(int) * 2);
  if (e != cudaSuccess) { bfail(b, e, "batch allocation"); return fail(MHD_ERR_OOM); }
  e = cudaMemcpy(b->d_ops, b->ops.data(), sizeof(BatchOp) * b->ops.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_inst, inst.data(), sizeof(BatchInst) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(b->d_abort, 0, sizeof(int) * 2);
  // shared memory: the largest tile body (the per-element CT march's prefetch ring, 15 values
  // per iteration, or the 16-byte fluid staging)
  b->smem = std::max({sizeof(float) * (size_t)mhd::kMarchRing * 15 * mhd::kBatchNT,
                      mhd::march_tile_smem<float>(), mhd::ct_rows_smem<float>(mhd::kBatchRowsR)});
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(mhd::batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)b->smem);
  int per_sm = 0, dev = 0, sms = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mhd::batch_kernel, mhd::kBatchNT,
                                                      b->smem);
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess || per_sm < 1) { bfail(b, e, "batch setup"); return fail(MHD_ERR_CUDA); }
  if (ctas_per_sm > 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
  b->grid = per_sm * sms;   // every CTA resident: no item waits on a CTA that cannot run
  *out = b;
  return MHD_OK;
}

// Advance every instance by nsteps steps in one persistent launch.
// One persistent launch advancing instance i by nsteps[i] steps (0 leaves it as it is).
static mhd_status batch_step_counts(mhd_batch* b, const int* nsteps) {
  const int n = (int)b->ctx.size();
  int smax = 0;
  std::vector<int> key;
  bool ops_changed = false;
  for (int i = 0; i < n; ++i) {
    mhd_ctx* c = b->ctx[i];
    if (nsteps[i] < 0) return MHD_ERR_INVALID;
    if (ctx_sig(c) != b->sig[i]) {
      // the context's buffers moved since its operations were built (steps run alone,
      // whose middle CT pair flips the B buffers, or mhd_apply): rebuild them; the work
      // list and the captured graphs refer to operations by index and stay valid
      b->sig[i] = ctx_sig(c);
      for (int p = 0; p < 3; ++p)
        build_step_ops(c, p, b->wpt, &b->ops[((size_t)i * 3 + p) * kOpsPerStep]);
      ops_changed = true;
    }
    smax = nsteps[i] > smax ? nsteps[i] : smax;
    key.push_back(nsteps[i]);
    key.push_back(c->phase);
  }
  if (smax < 1) return MHD_ERR_INVALID;
  if (ops_changed) {
    // a launch in flight may still read the operations
    BK(cudaStreamSynchronize(b->stream), "synchronize before updating the operations");
    BK(cudaMemcpy(b->d_ops, b->ops.data(), sizeof(BatchOp) * b->ops.size(),
                  cudaMemcpyHostToDevice), "operations upload");
  }
  auto it = b->graphs.find(key);
  if (it == b->graphs.end()) {
    // the previous launch may still read the current work list: let it finish first
    BK(cudaStreamSynchronize(b->stream), "synchronize before rebuilding the work list");
    // items: round by round (step, operation), all instances of a round together
    std::vector<BatchItem> items;
    std::vector<int> need(n, 0);
    for (int s = 0; s < smax; ++s)
      for (int k = 0; k < kOpsPerStep; ++k)
        for (int i = 0; i < n; ++i) {
          if (s >= nsteps[i]) continue;
          const int p = (b->ctx[i]->phase + s) % 3;
          const int opi = (i * 3 + p) * kOpsPerStep + k;
          const int tiles = b->ops[opi].tiles;
          for (int t = 0; t < tiles; ++t) items.push_back({i, opi, t, need[i]});
          need[i] += tiles;
        }
    const long long nitems = (long long)items.size();
    if (nitems > b->items_cap) {
      cudaFree(b->d_items);
      b->d_items = nullptr;
      BK(cudaMalloc(&b->d_items, sizeof(BatchItem) * nitems), "items allocation");
      b->items_cap = nitems;
    }
    BK(cudaMemcpy(b->d_items, items.data(), sizeof(BatchItem) * nitems, cudaMemcpyHostToDevice),
       "items upload");
    // drop graphs that referenced another item list
    for (auto& kv : b->graphs)
      if (kv.second.first) cudaGraphExecDestroy(kv.second.first);
    b->graphs.clear();
    BatchArgs args;
    args.items = b->d_items;
    args.nitems = nitems;
    args.ops = b->d_ops;
    args.inst = b->d_inst;
    args.queue = b->d_queue;
    args.done = b->d_done;
    args.abort = b->d_abort;
    args.status = b->d_abort + 1;
    args.spin_limit = mhd::kSpinCycles;
    cudaGraph_t gr = nullptr;
    BK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    cudaMemsetAsync(b->d_queue, 0, sizeof(unsigned long long), b->stream);
    cudaMemsetAsync(b->d_done, 0, sizeof(int) * n, b->stream);
    cudaMemsetAsync(b->d_abort, 0, sizeof(int), b->stream);   // abort flag; status is sticky
    mhd::batch_kernel<<<b->grid, mhd::kBatchNT, b->smem, b->stream>>>(args);
    cudaError_t e1 = cudaGetLastError();
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &gr);
    if (e1 != cudaSuccess) { if (gr) cudaGraphDestroy(gr); return bfail(b, e1, "capture"); }
    if (e2 != cudaSuccess) return bfail(b, e2, "end capture");
    cudaGraphExec_t ex = nullptr;
    cudaError_t e3 = cudaGraphInstantiate(&ex, gr, 0);
    cudaGraphDestroy(gr);
    if (e3 != cudaSuccess) return bfail(b, e3, "instantiate");
    it = b->graphs.emplace(key, std::make_pair(ex, nitems)).first;
  }
  // order after each context's pending work, run, and make each context wait for it
  for (int i = 0; i < n; ++i) {
    BK(cudaEventRecord(b->ev, b->ctx[i]->stream), "event");
    BK(cudaStreamWaitEvent(b->stream, b->ev, 0), "wait event");
  }
  BK(cudaGraphLaunch(it->second.first, b->stream), "batch launch");
  BK(cudaEventRecord(b->ev, b->stream), "event");
  for (int i = 0; i < n; ++i) {
    BK(cudaStreamWaitEvent(b->ctx[i]->stream, b->ev, 0), "wait event");
    mhd_ctx* c = b->ctx[i];
    c->phase = (c->phase + nsteps[i]) % 3;
    c->step += nsteps[i];
    c->steps_base += nsteps[i];
  }
  return MHD_OK;
}

mhd_status mhd_batch_step(mhd_batch* b, int nsteps) {
  if (!b || nsteps < 1) return MHD_ERR_INVALID;
  std::vector<int> counts(b->ctx.size(), nsteps);
  return batch_step_counts(b, counts.data());
}

mhd_status mhd_batch_step_each(mhd_batch* b, const int* nsteps) {
  if (!b || !nsteps) return MHD_ERR_INVALID;
  return batch_step_counts(b, nsteps);
}

// Wait for the batch's stream; MHD_ERR_TIMEOUT if a bounded wait gave up.
mhd_status mhd_batch_sync(mhd_batch* b) {
  if (!b) return MHD_ERR_INVALID;
  BK(cudaMemcpyAsync(b->h_status, b->d_abort, sizeof(int) * 2, cudaMemcpyDeviceToHost, b->stream),
     "status");
  BK(cudaStreamSynchronize(b->stream), "synchronize");
  if (!b->h_status[1]) return MHD_OK;
  BK(cudaMemset(b->d_abort + 1, 0, sizeof(int)), "status reset");   // reported once
  return MHD_ERR_TIMEOUT;
}

// Exercise the bounded wait of the persistent kernel: one work item waits for a completion
// count that nothing produces; the wait must give up after spin_cycles and report
// MHD_ERR_TIMEOUT, leaving the device usable.
mhd_status mhd_batch_selftest_timeout(long long spin_cycles) {
  if (spin_cycles < 1 || spin_cycles > mhd::kSpinCycles) return MHD_ERR_INVALID;
  mhd_batch* b = nullptr;
  BatchItem item{0, 0, 0, 1};            // instance 0 waits for one completion: never comes
  BatchItem* d_item = nullptr;
  unsigned long long* d_queue = nullptr;
  int* d_words = nullptr;                 // done[0], abort, status
  int h_words[3] = {0, 0, 0};
  mhd_status st = MHD_OK;
  cudaError_t e = cudaMalloc(&d_item, sizeof(item));
  if (e == cudaSuccess) e = cudaMalloc(&d_queue, sizeof(*d_queue));
  if (e == cudaSuccess) e = cudaMalloc(&d_words, sizeof(int) * 3);
  if (e == cudaSuccess) e = cudaMemcpy(d_item, &item, sizeof(item), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(d_queue, 0, sizeof(*d_queue));
  if (e == cudaSuccess) e = cudaMemset(d_words, 0, sizeof(int) * 3);
  if (e == cudaSuccess) {
    BatchArgs a;
    std::memset(&a, 0, sizeof(a));
    a.items = d_item;
    a.nitems = 1;
    a.queue = d_queue;
    a.done = d_words;
    a.abort = d_words + 1;
    a.status = d_words + 2;
    a.spin_limit = spin_cycles;
    mhd::batch_kernel<<<1, mhd::kBatchNT, 0>>>(a);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(h_words, d_words, sizeof(int) * 3, cudaMemcpyDeviceToHost);
  }
  if (e != cudaSuccess) st = MHD_ERR_CUDA;
  else st = h_words[2] ? MHD_ERR_TIMEOUT : MHD_OK;
  cudaFree(d_item);
  cudaFree(d_queue);
  cudaFree(d_words);
  (void)b;
  return st;
}

mhd_status mhd_batch_info(const mhd_batch* b, int* resident_ctas, long long* items_per_launch,
                          void** stream) {
  if (!b) return MHD_ERR_INVALID;
  if (stream) *stream = (void*)b->stream;
  if (resident_ctas) *resident_ctas = b->grid;
  if (items_per_launch) *items_per_launch = b->graphs.empty() ? 0 : b->graphs.begin()->second.second;
  return MHD_OK;
}

}  // extern "C"
