"""Served form: continuous batching of MHD solves on one GPU.

Requests (a grid, an initial state, a number of steps) arrive over time.  The scheduler
admits them in arrival order while their device memory fits a budget, keeps every admitted
state resident in HBM, and advances all active requests together: each iteration is one
persistent batched launch (mhd_batch_step_each) in which request i advances by its own
step count s_i; grids large enough to fill the GPU by themselves run their s_i steps as
plain graph launches on their own streams, concurrently with that launch.  The counts share
the cell updates of an iteration (sized so that it takes about `iter_ms` at the measured
throughput) among the active requests, with weights that grow with each request's waiting
time: a small grid takes many steps per iteration and finishes soon, a large one a few, and
long-waiting requests get more.  Counts of 3 or more are multiples of 3, so that the
axis-order phase of every request is the same from one iteration to the next and the
launch's work list and graph are reused.  Requests that finish leave the batch and are read
back while the next iteration runs, freeing memory for the next arrivals, which join at the
next iteration.  Each request's result is the same bits as running it alone (the batched
launch runs the same arithmetic per grid).

The scheduling logic talks to the GPU through a small backend interface (`GpuBackend`),
so that it can be exercised with a fake backend on a machine without a GPU.
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np

from . import inputs as I


def device_bytes(ncells: int) -> int:
    """Device memory of one FP32 context: two buffers per field, the FP64 staging array
    and the scalar block."""
    return int(ncells) * (2 * 8 * 4 + 8) + 4096


@dataclasses.dataclass
class Job:
    req: I.Request
    need: int
    handle: object = None
    remaining: int = 0
    admitted: float = 0.0
    done: float = -1.0
    result: object = None


class GpuBackend:
    """The CUDA library behind the scheduler (FP32 contexts and batches)."""

    def __init__(self, z_tile_warps: int = 0, ctas_per_sm: int = 0):
        from . import mhd
        self.mhd = mhd
        self.z_tile_warps, self.ctas_per_sm = z_tile_warps, ctas_per_sm

    def create(self, prob: I.Problem, fields32: list):
        s = self.mhd.Solver(prob.n, prob.bc, prob.h, prob.gamma, prob.cfl, prec=self.mhd.FP32)
        s.upload(fields32)
        return s

    def batch(self, handles):
        return self.mhd.Batch(handles, self.z_tile_warps, self.ctas_per_sm)

    def step(self, handle, n: int):
        handle.step(n)

    def read(self, handle) -> np.ndarray:
        """The 8 FP32 fields, (8, N), downloaded into a reused page-locked buffer: the
        returned array is valid until the next read."""
        import torch
        n = 8 * handle.ncells
        if getattr(self, "_pin", None) is None or self._pin.numel() < n:
            self._pin = torch.empty(n, dtype=torch.float32, pin_memory=True)
        views = [self._pin[k * handle.ncells:(k + 1) * handle.ncells] for k in range(8)]
        handle.download(views)
        return self._pin[:n].numpy().reshape(8, handle.ncells)

    def sync(self, batch):
        st = batch.sync()
        if st != self.mhd.MHD_OK:
            raise self.mhd.MhdError(st, "batched launch failed")

    def wait(self, handle):
        handle.sync()

    def close(self, handle):
        handle.close()


class ICCache:
    """Initial states by (kind, edge), kept as FP32 host arrays (requests of the same kind
    and edge start from the same state); `pinned` keeps them in page-locked memory (torch)
    so that uploads run at full link speed."""

    def __init__(self, pinned: bool = False):
        self.cache = {}
        self.pinned = pinned

    def get(self, req: I.Request):
        key = (req.kind, req.edge)
        if key not in self.cache:
            prob = req.problem()
            f32 = [np.ascontiguousarray(prob.fields[k], dtype=np.float32) for k in range(8)]
            if self.pinned:
                import torch
                f32 = [torch.from_numpy(a).pin_memory() for a in f32]
            self.cache[key] = (dataclasses.replace(prob, fields=None), f32)
        return self.cache[key]


class Server:
    """Continuous-batching scheduler.

    budget_bytes   device memory the admitted requests may hold together
    iter_ms        target duration of one iteration (sets the step counts)
    rate0          initial estimate of the throughput (cell updates per second); updated
                   from every iteration's measured time
    max_steps      cap on one request's steps per iteration (bounds the dependent chain of
                   a small grid inside one launch)
    age_tau        seconds of waiting that double a request's weight (see counts)
    plain_min_cells  grids at least this large run their steps as plain graph launches on
                   their own streams, concurrently with the batched launch of the smaller
                   ones (a large grid fills the GPU by itself; batching pays off for grids
                   whose launches cannot)
    """

    def __init__(self, backend, budget_bytes: float = 120e9, iter_ms: float = 25.0,
                 rate0: float = 3e9, max_steps: int = 240, plain_min_cells: int = 1 << 21,
                 age_tau: float = 0.5, ics: ICCache | None = None, clock=time.perf_counter,
                 keep_results=False):
        self.be = backend
        self.age_tau = float(age_tau)
        self.plain_min_cells = int(plain_min_cells)
        self.budget = int(budget_bytes)
        self.iter_s = iter_ms / 1e3
        self.rate = float(rate0)
        self.max_steps = int(max_steps)
        self.ics = ics or ICCache()
        self.clock = clock
        self.keep_results = keep_results
        self.peak_bytes = 0
        self.iterations = 0
        self.batch_rebuilds = 0
        self.times = {"admit": 0.0, "rebuild": 0.0, "launch": 0.0, "wait": 0.0, "retire": 0.0}

    def counts(self, active, now: float = 0.0) -> list:
        """Steps per active request for the next iteration: the iteration's cell updates
        (iter_ms x throughput) shared with weights (1 + age / age_tau)^2, so that a request
        gains share the longer it has waited (new small requests still finish within a few
        iterations, and large ones are not starved by a stream of small arrivals)."""
        w = [(1.0 + max(0.0, now - j.req.arrival) / self.age_tau) ** 2 for j in active]
        total = sum(w) or 1.0
        out = []
        for j, wj in zip(active, w):
            share = self.iter_s * self.rate * wj / total              # cell updates
            s = int(share // j.req.ncells)
            s = max(1, min(s, self.max_steps))
            if s >= 3:
                s -= s % 3
            out.append(min(s, j.remaining))
        return out

    def run(self, trace) -> list:
        """Serve the requests of `trace` (arrival times in seconds from now); returns the
        jobs with their admission and completion times.

        Each iteration launches the active set, then, while the GPU works, admits the
        requests that arrived (creating and uploading their states) and reads back the
        requests that finished in the previous iteration; then it waits for the launch.  A
        request admitted during an iteration joins the next one; a request is complete
        when its result has been read back."""
        pending = collections.deque(sorted(trace, key=lambda r: r.arrival))
        jobs: list = []
        active: list = []
        to_retire: list = []
        self._used = 0
        batch, batch_ids = None, None
        tm = self.times
        t0 = self.clock()
        while pending or active or to_retire:
            counts = []
            big = [j for j in active if j.req.ncells >= self.plain_min_cells]
            small = [j for j in active if j.req.ncells < self.plain_min_cells]
            if active:
                c0 = self.clock()
                ids = tuple(id(j) for j in small)
                if ids != batch_ids:
                    if batch is not None:
                        batch.close()
                    batch = self.be.batch([j.handle for j in small]) if small else None
                    batch_ids = ids
                    self.batch_rebuilds += 1
                c1 = self.clock()
                counts = self.counts(active, c1 - t0)
                cnt = dict(zip(map(id, active), counts))
                if batch is not None:
                    batch.step_each([cnt[id(j)] for j in small])
                for j in big:
                    self.be.step(j.handle, cnt[id(j)])
                c2 = self.clock()
                tm["rebuild"] += c1 - c0
                tm["launch"] += c2 - c1
            # admission, in arrival order, while the budget allows (overlaps the launch)
            a0 = self.clock()
            newly = self._admit(pending, jobs, t0)
            tm["admit"] += self.clock() - a0
            # read back what finished in the previous iteration (overlaps the launch)
            if to_retire:
                r0 = self.clock()
                for j in to_retire:
                    res = self.be.read(j.handle)
                    j.done = self.clock() - t0
                    if self.keep_results:
                        j.result = (self.keep_results(res) if callable(self.keep_results)
                                    else np.array(res))
                    self.be.close(j.handle)
                    j.handle = None
                    self._used -= j.need
                to_retire = []
                tm["retire"] += self.clock() - r0
            if not active:
                if not newly and pending:
                    wait = pending[0].arrival - (self.clock() - t0)
                    if wait > 0:
                        time.sleep(min(wait, 0.05))
                active = newly
                continue
            w0 = self.clock()
            if batch is not None:
                self.be.sync(batch)
            for j in big:
                self.be.wait(j.handle)
            w1 = self.clock()
            tm["wait"] += w1 - w0
            self.iterations += 1
            work = 0
            for j, s in zip(active, counts):
                j.remaining -= s
                work += s * j.req.ncells
            dt = w1 - c0
            if dt > 0 and work > 0:
                self.rate = 0.7 * self.rate + 0.3 * (work / dt)
            # finished requests leave the batch now (it never outlives its contexts) and are
            # read back during the next iteration
            finished = [j for j in active if j.remaining == 0]
            if finished:
                if batch is not None and any(j.remaining == 0 for j in small):
                    batch.close()
                    batch, batch_ids = None, None
                to_retire = finished
            active = [j for j in active if j.remaining > 0] + newly
        if batch is not None:
            batch.close()
        return jobs

    def _admit(self, pending, jobs, t0) -> list:
        out = []
        now = self.clock() - t0
        while pending and pending[0].arrival <= now:
            r = pending[0]
            need = device_bytes(r.ncells)
            if need > self.budget:
                pending.popleft()
                jobs.append(Job(r, need, done=float("nan")))   # can never fit: rejected
                continue
            if self._used + need > self.budget:
                break
            pending.popleft()
            prob, f32 = self.ics.get(r)
            job = Job(r, need, self.be.create(prob, f32), r.steps, self.clock() - t0)
            self._used += need
            self.peak_bytes = max(self.peak_bytes, self._used)
            out.append(job)
            jobs.append(job)
        return out


def serve_sequential(backend, trace, ics: ICCache | None = None, clock=time.perf_counter,
                     keep_results=False) -> list:
    """The baseline: one request at a time in arrival order, each alone on the GPU with
    plain (graph-replayed) steps."""
    ics = ics or ICCache()
    jobs = []
    t0 = clock()
    for r in sorted(trace, key=lambda r: r.arrival):
        wait = r.arrival - (clock() - t0)
        if wait > 0:
            time.sleep(wait)
        prob, f32 = ics.get(r)
        job = Job(r, device_bytes(r.ncells), backend.create(prob, f32), r.steps, clock() - t0)
        backend.step(job.handle, r.steps)
        res = backend.read(job.handle)
        job.done = clock() - t0
        if keep_results:
            job.result = keep_results(res) if callable(keep_results) else np.array(res)
        backend.close(job.handle)
        job.handle = None
        job.remaining = 0
        jobs.append(job)
    return jobs


def summarize(jobs) -> dict:
    ok = [j for j in jobs if j.done == j.done and j.done >= 0]
    lat = np.array([j.done - j.req.arrival for j in ok])
    work = sum(j.req.ncells * j.req.steps for j in ok)
    makespan = max((j.done for j in ok), default=0.0)
    return {"requests": len(jobs), "completed": len(ok),
            "rejected": sum(1 for j in jobs if j.done != j.done),
            "p50_s": float(np.percentile(lat, 50)) if lat.size else None,
            "p99_s": float(np.percentile(lat, 99)) if lat.size else None,
            "mean_s": float(lat.mean()) if lat.size else None,
            "makespan_s": makespan, "cell_updates": int(work),
            "cell_updates_per_s": work / makespan if makespan > 0 else None}
