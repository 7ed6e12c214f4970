// Batched persistent form: many grids (solver contexts of any shape) advanced by one
// persistent, graph-captured launch.  The launch keeps as many CTAs resident as the GPU
// holds; each CTA repeatedly takes the next work item (instance, operation, tile) from a
// device queue.  Items are laid out round by round (step, operation) over all instances, so
// that small grids fill the GPU together.  An item of operation k of an instance may start
// only when every item of that instance's earlier operations is complete: each instance
// has a completion counter, incremented with release semantics after an item and awaited
// with acquire semantics (bounded: after the spin limit the kernel records MHD_ERR_TIMEOUT,
// raises an abort flag that every CTA checks, and returns instead of hanging).
//
// Each context has a launch shape (mhd_batch_shape: tile length of the x/y marches, CT form,
// z segment length and items, or a route through the single-grid kernels); the kernel runs
// at 128 or 256 threads per CTA (mhd_batch.cuh).  Shapes change speed, never bits.
#include <algorithm>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/mhd.h"
#include "mhd_batch.cuh"
#include "mhd_ctx.h"


using mhd::BatchArgs;
using mhd::BatchInst;
using mhd::BatchItem;
using mhd::BatchOp;

// a context's launch shape with its defaults resolved (mhd_batch_shape)
struct BatchShape {
  int s = mhd::kMarchS == 128 || mhd::kMarchS == 256 ? mhd::kMarchS : 192;
  int rows = 1;       // shared-row CT where the grid allows it
  int segk = 0;       // 0: seg_k_for(nz)
  int wpt = 0;        // 0: the batch's z_tile_warps
  int alone = 0;
};

struct mhd_batch {
  std::vector<mhd_ctx*> ctx;
  std::vector<unsigned> sig;           // buffer state of each context when its ops were built
  std::vector<BatchShape> shape;
  std::vector<BatchOp> ops;            // [instance][phase][13]
  const mhd::BatchKernel* kern = nullptr;
  cudaStream_t stream = nullptr;
  int grid = 0;                        // resident CTAs of the persistent launch
  int ctas_per_sm = 0;                 // asked for (0: as many as fit)
  int wpt = 0;                         // z warp segments per tile (0: chosen per sweep)
  long long spin = mhd::kSpinCycles;
  BatchOp* d_ops = nullptr;
  BatchInst* d_inst = nullptr;
  BatchItem* d_items = nullptr;
  long long items_cap = 0;
  unsigned long long* d_queue = nullptr;
  int* d_done = nullptr;
  int* d_abort = nullptr;              // d_abort[0] abort flag, d_abort[1] status
  int* h_status = nullptr;             // pinned
  cudaEvent_t ev = nullptr;
  // graph per (step counts, phases of the instances); items uploaded for the same key
  std::map<std::vector<int>, std::pair<cudaGraphExec_t, long long>> graphs;
  std::vector<char> in_last;           // contexts in a persistent launch since the last sync
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
// and write (mirrors enqueue_step_t in mhd_capi.cu), tiled for NT threads per CTA
static void build_step_ops(const mhd_ctx* c, int phase, int bwpt, const BatchShape& sh, int nt,
                           BatchOp* out) {
  int cur[8];
  for (int k = 0; k < 8; ++k) cur[k] = c->cur[k];
  const int R = nt / 32;                 // EMF rows of a shared-row CT tile
  const int flat_cells = nt * mhd::kFlatPerThread;
  const int wpt = sh.wpt > 0 ? sh.wpt : bwpt;
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
      op.s = sh.s;
      op.rows = (op.kind == mhd::OP_CT && sh.rows && mhd::ct_use_rows(g, op.axis)) ? 1 : 0;
      op.gx = op.rows ? ((g.n[2] + 30) / 31) * ((g.n[o] + R - 2) / (R - 1))
                      : (int)((np + nt - 1) / nt);
      op.tiles = op.gx * ((g.n[op.axis] + op.s - 1) / op.s);
    } else {
      op.segk = sh.segk ? sh.segk : mhd::seg_k_for(g.n[2]);
      const int seg = 32 * op.segk - (op.kind == mhd::OP_FLUID ? 6 : 8);
      op.nwarps = (long long)g.n[0] * g.n[1] * ((g.n[2] + seg - 1) / seg);
      // 0: about kAutoTiles items per z sweep (small grids get short items, large ones
      // up to 128 warp segments each)
      long long w = wpt > 0 ? wpt : (op.nwarps + mhd::kAutoTiles - 1) / mhd::kAutoTiles;
      if (wpt == 0) w = w < 4 ? 4 : (w > 128 ? 128 : w);
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
    const int flat_tiles = (int)((ncell + flat_cells - 1) / flat_cells);
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

static void build_ops(mhd_batch* b, int i) {
  b->sig[i] = ctx_sig(b->ctx[i]);
  for (int p = 0; p < 3; ++p)
    build_step_ops(b->ctx[i], p, b->wpt, b->shape[i], b->kern->nt,
                   &b->ops[((size_t)i * 3 + p) * kOpsPerStep]);
}

static void drop_graphs(mhd_batch* b) {
  for (auto& kv : b->graphs)
    if (kv.second.first) cudaGraphExecDestroy(kv.second.first);
  b->graphs.clear();
}

// the persistent kernel's resident CTAs for the batch's kernel and CTAs-per-SM request
static mhd_status set_grid(mhd_batch* b) {
  int per_sm = 0, dev = 0, sms = 0;
  cudaError_t e = b->kern->prepare(&per_sm);
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return bfail(b, e, "batch kernel setup");
  if (per_sm < 1) {
    b->err = "batch kernel: no resident CTA fits";
    return MHD_ERR_CUDA;
  }
  if (b->ctas_per_sm > 0 && b->ctas_per_sm < per_sm) per_sm = b->ctas_per_sm;
  b->grid = per_sm * sms;   // every CTA resident: no item waits on a CTA that cannot run
  return MHD_OK;
}

extern "C" {

void mhd_batch_destroy(mhd_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  drop_graphs(b);
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
  b->kern = &mhd::batch_kernel_nt128();
  b->wpt = z_tile_warps > 0 ? z_tile_warps : 0;
  b->ctas_per_sm = ctas_per_sm > 0 ? ctas_per_sm : 0;
  b->ctx.assign(ctxs, ctxs + n);
  b->sig.resize(n);
  b->shape.resize(n);
  b->in_last.assign(n, 0);
  b->ops.resize((size_t)n * 3 * kOpsPerStep);
  for (int i = 0; i < n; ++i) build_ops(b, i);
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
  if (e != cudaSuccess) { bfail(b, e, "batch setup"); return fail(MHD_ERR_CUDA); }
  const mhd_status gs = set_grid(b);
  if (gs != MHD_OK) return fail(gs);
  *out = b;
  return MHD_OK;
}

mhd_status mhd_batch_configure(mhd_batch* b, int threads_per_cta, int ctas_per_sm,
                               long long spin_cycles, const mhd_batch_shape* shapes) {
  if (!b) return MHD_ERR_INVALID;
  if (threads_per_cta != 0 && threads_per_cta != 128 && threads_per_cta != 256)
    return MHD_ERR_INVALID;
  if (ctas_per_sm < 0 || spin_cycles < 0 || spin_cycles > mhd::kSpinCycles) return MHD_ERR_INVALID;
  const int n = (int)b->ctx.size();
  std::vector<BatchShape> sh(n);
  for (int i = 0; shapes && i < n; ++i) {
    const mhd_batch_shape& q = shapes[i];
    if ((q.march_len != 0 && !mhd::batch_len_ok(q.march_len)) || q.ct_march < 0 ||
        q.ct_march > 1 || (q.seg_k != 0 && q.seg_k != 2 && q.seg_k != 3) || q.z_warps < 0 ||
        q.z_warps > (1 << 20) || q.alone < 0 || q.alone > 1)
      return MHD_ERR_INVALID;
    if (q.march_len) sh[i].s = q.march_len;
    sh[i].rows = q.ct_march ? 0 : 1;
    sh[i].segk = q.seg_k;
    sh[i].wpt = q.z_warps;
    sh[i].alone = q.alone;
  }
  // the previous launch may still read the operations and the work list
  BK(cudaStreamSynchronize(b->stream), "synchronize before reconfiguring");
  drop_graphs(b);
  if (threads_per_cta) {
    b->kern = threads_per_cta == 256 ? &mhd::batch_kernel_nt256() : &mhd::batch_kernel_nt128();
  }
  b->ctas_per_sm = ctas_per_sm;
  b->spin = spin_cycles > 0 ? spin_cycles : mhd::kSpinCycles;
  b->shape = sh;
  for (int i = 0; i < n; ++i) build_ops(b, i);
  BK(cudaMemcpy(b->d_ops, b->ops.data(), sizeof(BatchOp) * b->ops.size(), cudaMemcpyHostToDevice),
     "operations upload");
  return set_grid(b);
}

// One persistent launch advancing instance i by nsteps[i] steps (0 leaves it as it is);
// contexts routed alone step through mhd_step on their own streams instead.
static mhd_status batch_step_counts(mhd_batch* b, const int* nsteps) {
  const int n = (int)b->ctx.size();
  int smax = 0, pmax = 0;
  std::vector<int> key;
  bool ops_changed = false;
  for (int i = 0; i < n; ++i) {
    if (nsteps[i] < 0) return MHD_ERR_INVALID;
    smax = nsteps[i] > smax ? nsteps[i] : smax;
  }
  if (smax < 1) return MHD_ERR_INVALID;
  for (int i = 0; i < n; ++i) {
    mhd_ctx* c = b->ctx[i];
    const int k = b->shape[i].alone ? 0 : nsteps[i];
    if (k > 0 && ctx_sig(c) != b->sig[i]) {
      // the context's buffers moved since its operations were built (steps run alone,
      // whose middle CT pair flips the B buffers, or mhd_apply): rebuild them; the work
      // list and the captured graphs refer to operations by index and stay valid
      build_ops(b, i);
      ops_changed = true;
    }
    pmax = k > pmax ? k : pmax;
    key.push_back(k);
    key.push_back(k > 0 ? c->phase : 0);
  }
  // contexts routed through the single-grid kernels
  for (int i = 0; i < n; ++i) {
    if (!b->shape[i].alone || nsteps[i] == 0) continue;
    // (a status the context already carries is its own to report, as in the launch)
    const mhd_status st = mhd_step(b->ctx[i], nsteps[i], -1.0, nullptr, nullptr);
    if (st != MHD_OK && st != MHD_ERR_UNPHYSICAL && st != MHD_ERR_TIMEOUT) return st;
  }
  if (pmax < 1) {
    // nothing for the persistent kernel: the batch's stream still orders after the
    // contexts' steps, so that mhd_batch_sync waits for them
    for (int i = 0; i < n; ++i) {
      if (!nsteps[i]) continue;
      BK(cudaEventRecord(b->ev, b->ctx[i]->stream), "event");
      BK(cudaStreamWaitEvent(b->stream, b->ev, 0), "wait event");
    }
    return MHD_OK;
  }
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
    for (int s = 0; s < pmax; ++s)
      for (int k = 0; k < kOpsPerStep; ++k)
        for (int i = 0; i < n; ++i) {
          if (s >= key[2 * i]) continue;
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
    drop_graphs(b);
    BatchArgs args;
    args.items = b->d_items;
    args.nitems = nitems;
    args.ops = b->d_ops;
    args.inst = b->d_inst;
    args.queue = b->d_queue;
    args.done = b->d_done;
    args.abort = b->d_abort;
    args.status = b->d_abort + 1;
    args.spin_limit = b->spin;
    cudaGraph_t gr = nullptr;
    BK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    cudaMemsetAsync(b->d_queue, 0, sizeof(unsigned long long), b->stream);
    cudaMemsetAsync(b->d_done, 0, sizeof(int) * n, b->stream);
    cudaMemsetAsync(b->d_abort, 0, sizeof(int), b->stream);   // abort flag; status is sticky
    cudaError_t e1 = b->kern->launch(b->grid, b->stream, args);
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &gr);
    if (e1 != cudaSuccess) { if (gr) cudaGraphDestroy(gr); return bfail(b, e1, "capture"); }
    if (e2 != cudaSuccess) return bfail(b, e2, "end capture");
    cudaGraphExec_t ex = nullptr;
    cudaError_t e3 = cudaGraphInstantiate(&ex, gr, 0);
    cudaGraphDestroy(gr);
    if (e3 != cudaSuccess) return bfail(b, e3, "instantiate");
    it = b->graphs.emplace(key, std::make_pair(ex, nitems)).first;
  }
  // order after each persistent context's pending work, run, and make each of them wait
  // for the launch
  for (int i = 0; i < n; ++i) {
    if (!key[2 * i]) continue;
    BK(cudaEventRecord(b->ev, b->ctx[i]->stream), "event");
    BK(cudaStreamWaitEvent(b->stream, b->ev, 0), "wait event");
  }
  BK(cudaGraphLaunch(it->second.first, b->stream), "batch launch");
  BK(cudaEventRecord(b->ev, b->stream), "event");
  for (int i = 0; i < n; ++i) {
    if (!key[2 * i]) continue;
    b->in_last[i] = 1;
    BK(cudaStreamWaitEvent(b->ctx[i]->stream, b->ev, 0), "wait event");
    mhd_ctx* c = b->ctx[i];
    c->phase = (c->phase + nsteps[i]) % 3;
    c->step += nsteps[i];
    c->steps_base += nsteps[i];
  }
  // the routed contexts' steps run beside the launch; the batch's stream then waits for
  // them, so that mhd_batch_sync covers them
  for (int i = 0; i < n; ++i) {
    if (!b->shape[i].alone || !nsteps[i]) continue;
    BK(cudaEventRecord(b->ev, b->ctx[i]->stream), "event");
    BK(cudaStreamWaitEvent(b->stream, b->ev, 0), "wait event");
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

// Wait for the batch's stream; MHD_ERR_TIMEOUT if a bounded wait gave up, and then every
// context of the persistent launches since the last sync is marked (its later calls
// report the timeout until it is initialised again).
mhd_status mhd_batch_sync(mhd_batch* b) {
  if (!b) return MHD_ERR_INVALID;
  BK(cudaMemcpyAsync(b->h_status, b->d_abort, sizeof(int) * 2, cudaMemcpyDeviceToHost, b->stream),
     "status");
  BK(cudaStreamSynchronize(b->stream), "synchronize");
  std::vector<char> launched(b->ctx.size(), 0);
  launched.swap(b->in_last);
  if (!b->h_status[1]) return MHD_OK;
  BK(cudaMemset(b->d_abort + 1, 0, sizeof(int)), "status reset");   // reported once
  for (size_t i = 0; i < b->ctx.size(); ++i)
    if (launched[i]) b->ctx[i]->status |= mhd::ST_TIMEOUT;
  return MHD_ERR_TIMEOUT;
}

// Exercise the bounded wait of the persistent kernel: one work item waits for a completion
// count that nothing produces; the wait must give up after spin_cycles and report
// MHD_ERR_TIMEOUT, leaving the device usable.
mhd_status mhd_batch_selftest_timeout(long long spin_cycles) {
  if (spin_cycles < 1 || spin_cycles > mhd::kSpinCycles) return MHD_ERR_INVALID;
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
  int per_sm = 0;
  const mhd::BatchKernel& k = mhd::batch_kernel_nt128();
  if (e == cudaSuccess) e = k.prepare(&per_sm);
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
    e = k.launch(1, nullptr, a);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(h_words, d_words, sizeof(int) * 3, cudaMemcpyDeviceToHost);
  }
  if (e != cudaSuccess) st = MHD_ERR_CUDA;
  else st = h_words[2] ? MHD_ERR_TIMEOUT : MHD_OK;
  cudaFree(d_item);
  cudaFree(d_queue);
  cudaFree(d_words);
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
