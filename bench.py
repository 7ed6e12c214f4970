#!/usr/bin/env python
"""Benchmark of the hot path: the relaxing-TVD MHD step on a 512^3 magnetised blast wave
(periodic unit cube, gamma 5/3, rho 1, p 10 inside r < 0.1 else 0.1, B = (1,1,0)/sqrt(2)),
FP32 sweeps with FP64 conservation sums every 10 steps.

One "step" is one full method step (dt from the CFL condition, forward and reverse
dimensionally split sweeps, 6 fluid + 6 constrained-transport operators), advancing
every cell once: the metric counts cell-updates per second.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference] [--n 512]

N > 1 (under torchrun): independent replicas, one grid per GPU (the path needs no data
exchange between grids); value = cells x steps summed over ranks / max time over ranks.
--impl reference: the FP64 CPU oracle on the host cores, timed on a bounded sample of the
same workload (rank 0 only).
Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "cell-updates/s (512³ FP32) & %HBM roofline vs FP64; batched p50/p99 latency"
UNIT = "cell-updates/s"
SUMS_EVERY = 10
FALLBACK_HBM_GBS = 6800.0
# algorithmic bytes per cell for one launch of each kernel kind (FP32): the fields the
# operator must read and write once.  fluid: reads 8 fields, writes 5; CT: reads rho, m_n
# and the 3 B components, writes 3.  The method step (6 L-ops x 8 fields read + written)
# is 384 B per cell.
ALG_BYTES = {"fluid": 13 * 4, "ct": 8 * 4}
STEP_ALG_BYTES = 384
# DRAM bytes per cell of one fluid-sweep launch (average over the 4 x/y and 2 z launches of
# a step) from ncu captures on a 256^3 grid (the ncu summaries under profiles/), keyed by the
# hash of the kernel sources they were taken on; another hash reports null.
NCU_TRAFFIC_PER_CELL = {"6493be2955de5ac4": 50.74, "b10257c0c22a2f1c": 50.74,
                        "e5f6604cfb2b726c": 50.74}
# thread instructions per cell of one launch of each sweep kernel (ncu
# smsp__thread_inst_executed.sum / cells, 256^3; one launch in six of each axis's fluid sweeps
# also reduces c_max, and one CT launch in five of each axis is a two-pass middle pair: both
# weighted in), keyed like the traffic: the sweeps are bound by
# instruction issue, and this gives the issue rate they reach beside the HBM roofline
NCU_INSTR_PER_CELL = {"6493be2955de5ac4": {"fluid_x": 313.3, "fluid_y": 313.3, "fluid_z": 364.9,
                                           "ct_x": 178.4, "ct_y": 178.4, "ct_z": 263.8},
                      "b10257c0c22a2f1c": {"fluid_x": 313.3, "fluid_y": 313.3, "fluid_z": 364.9,
                                           "ct_x": 197.3, "ct_y": 197.3, "ct_z": 189.2},
                      "e5f6604cfb2b726c": {"fluid_x": 313.3, "fluid_y": 313.3, "fluid_z": 364.9,
                                           "ct_x": 197.3, "ct_y": 197.3, "ct_z": 190.4}}


KERNEL_SOURCES = ("mhd_kernels.cuh", "mhd_march.cuh", "mhd_segz.cuh", "mhd_flat.cuh",
                  "mhd_tma.cuh", "mhd_launch_impl.cuh")


def issue_object(dom: str, prof: dict, ipc: dict | None, cells: int, sms: int,
                 mhz: float) -> dict | None:
    """Instruction-issue rate of the `dom` sweeps: ncu thread instructions per cell of each
    kernel kind (`ipc`, None when the counts are not of these kernel sources) x cells x
    launches, over their total live time (`prof`: kind -> (ms, launches)), against the SMs'
    issue peak (4 schedulers x 32 lanes per SM per clock)."""
    if ipc is None:
        return None
    ks = [k for k in ipc if k.startswith(dom + "_") and prof.get(k, (0, 0))[1]]
    tms = sum(prof[k][0] for k in ks)
    if not ks or tms <= 0:
        return None
    ins = sum(ipc[k] * cells * prof[k][1] for k in ks)
    peak = sms * 4 * 32 * mhz * 1e6 / 1e12
    achieved = ins / (tms / 1e3) / 1e12
    return {"kernel": f"{dom} sweep (all axes)", "unit": "T thread-instructions/s",
            "achieved": achieved, "peak": peak, "frac": achieved / peak,
            "instr_per_cell": {k: ipc[k] for k in ks},
            "peak_note": f"{sms} SMs x 4 schedulers x 32 lanes x {mhz:.0f} MHz (median SM "
                         f"clock of the timed region); instruction counts from ncu on the "
                         f"same kernel sources"}


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_0908_4362_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    with open(os.path.join(ROOT, "paper_0908_4362_gb300", "build.py"), "rb") as fh:
        h.update(fh.read())          # the compiler flags are part of the kernels
    return h.hexdigest()[:16]


def workload_config(n: int) -> dict:
    return {"workload": f"3D magnetised blast wave {n}^3, periodic unit cube, gamma 5/3, "
                        f"p 10 in r<0.1 else 0.1, B=(1,1,0)/sqrt(2), FP32 sweeps, FP64 "
                        f"conservation sums every {SUMS_EVERY} steps",
            "grid": [n, n, n], "cells": n ** 3, "cfl": 0.7,
            "l2": "inputs larger than L2 (8 FP32 fields x 2 buffers, no flush needed)"}


def measured_peaks() -> tuple:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev_id: str | None):
        self.dev_id = dev_id
        self.proc = None
        self.lines: list = []
        self.thread = None

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "200"]
        if self.dev_id:
            cmd += ["-i", self.dev_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict | None:
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons, power = [], [], set(), []
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for name, val in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                                  "sw_power_cap"), parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


def start_clocks(local: int) -> "ClockSampler":
    """A running nvidia-smi sampler of the rank's GPU (stop() returns the clock record)."""
    import torch
    dev_uuid = None
    try:
        dev_uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    c = ClockSampler(dev_uuid)
    c.start()
    time.sleep(0.3)
    return c


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(value: float, world: int) -> float:
    """Max of a host float over ranks (timing reduction only; no data-path collective)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, world: int) -> float:
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ------------------------------------------------------------------------------------
# CPU baseline: the oracle, as it stands, on the host cores
# ------------------------------------------------------------------------------------

def oracle_sample(n: int, edge: int, steps: int) -> dict:
    """Time the FP64 oracle (OpenMP, all host cores) for `steps` steps on an edge^3 cut of
    the n^3 blast workload centred on the blast (periodic cut)."""
    import numpy as np

    import oracle
    from paper_0908_4362_gb300 import inputs as I
    edge = min(edge, n)
    # the cut keeps the full workload's cell width and blast radius
    h = 1.0 / n
    c = (np.arange(edge) - edge / 2 + 0.5) * h
    r2 = c[:, None, None] ** 2 + c[None, :, None] ** 2 + c[None, None, :] ** 2
    p = np.where(r2 < 0.01, 10.0, 0.1)
    z = np.zeros((edge,) * 3)
    f = I.conserved(np.ones((edge,) * 3), [z, z, z], p,
                    [np.full(z.shape, 1 / 2 ** 0.5), np.full(z.shape, 1 / 2 ** 0.5), z],
                    5.0 / 3.0, (0, 0, 0))
    o = oracle.Oracle((edge,) * 3, (0, 0, 0), h, 5.0 / 3.0, 0.7, f)
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    cells = edge ** 3 * steps
    return {"value": cells / dt, "unit": UNIT, "seconds": dt,
            "cores": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)),
            "kind": "oracle",
            "sample": f"{steps} step(s) of an {edge}^3 cut (cell width 1/{n}) of the {n}^3 "
                      f"blast workload, FP64 oracle, OpenMP over pencils"}


def oracle_single_core(n: int, edge: int) -> dict:
    """The same oracle sample on one host core: a child process with OMP_NUM_THREADS=1
    (the OpenMP runtime of this process has already fixed its thread count)."""
    code = ("import json, bench; r = bench.oracle_sample(%d, %d, 1); "
            "print(json.dumps({'value': r['value'], 'sample': r['sample']}))" % (n, edge))
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=600)
    if r.returncode != 0:
        return {"error": r.stderr.strip().splitlines()[-1] if r.stderr.strip() else "failed"}
    out = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": out["value"], "unit": UNIT, "cores": 1, "sample": out["sample"]}


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    edge = args.ref_edge
    oracle_sample(args.n, edge, 1)          # build + warm caches
    for _ in range(max(0, args.warmup - 1)):
        oracle_sample(args.n, edge, 1)
    t0 = time.perf_counter()
    res = None
    tot = 0.0
    for _ in range(args.steps):
        res = oracle_sample(args.n, edge, 1)
        tot += res["seconds"]
    value = edge ** 3 * args.steps / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args.n),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": res["cores"],
                             "kind": "oracle", "sample": res["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "wall_s": time.perf_counter() - t0}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------

def run_ours(args, world, rank, local):
    import numpy as np
    import torch

    from paper_0908_4362_gb300 import build, mhd
    from paper_0908_4362_gb300 import inputs as I

    build.build()
    torch.cuda.set_device(local)
    n = args.n
    prob = I.blast3d(n)
    N = prob.ncells
    # pinned FP32 host copies of the initial state (the e2e inputs)
    host = [torch.from_numpy(prob.fields[k].astype(np.float32)).pin_memory() for k in range(8)]
    del prob.fields
    solver = mhd.Solver((n, n, n), (0, 0, 0), 1.0 / n, 5.0 / 3.0, 0.7, prec=mhd.FP32)
    solver.upload(host)
    solver.step(args.warmup, sync=True)
    solver.sums()

    # ---- timed region: device-resident state, steps as the product runs them (one CUDA
    # graph per step), CUDA events on the context stream around the whole region ----
    stream = torch.cuda.ExternalStream(solver.stream_handle())
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dev_uuid = None
    try:
        dev_uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    clocks = ClockSampler(dev_uuid)
    torch.cuda.synchronize()
    solver.sync()
    barrier(world)
    clocks.start()
    time.sleep(0.3)
    ev0.record(stream)
    sums_calls = 0
    for k in range(args.steps):
        solver.step(1)
        if (k + 1) % SUMS_EVERY == 0:
            solver.sums()
            sums_calls += 1
    ev1.record(stream)
    ev1.synchronize()
    solver.sync()
    barrier(world)
    clk = clocks.stop()
    ms_total = ev0.elapsed_time(ev1)
    # ---- per-kernel times: the same steps launched kernel by kernel, an event pair around
    # each launch (a second region after the timed one) ----
    psteps = min(args.steps, 30)
    solver.profile(True)
    solver.profile_read(reset=True)
    ep0, ep1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ep0.record(stream)
    solver.step(psteps)
    ep1.record(stream)
    ep1.synchronize()
    solver.sync()
    prof = solver.profile_read(reset=True)
    solver.profile(False)
    prof_step_ms = ep0.elapsed_time(ep1) / psteps
    max_ms = max_over_ranks(ms_total, world)
    total_cells = sum_over_ranks(float(N) * args.steps, world)
    value = total_cells / (max_ms / 1e3)

    # roofline of the dominant kernel kind (by total time), algorithmic bytes / duration
    kinds = {}
    for name, (ms, cnt) in prof.items():
        base = name.split("_")[0]
        if base in ALG_BYTES and cnt:
            kms, kc = kinds.get(base, (0.0, 0))
            kinds[base] = (kms + ms, kc + cnt)
    dom = max(kinds, key=lambda k: kinds[k][0])
    dom_ms, dom_cnt = kinds[dom]
    avg_ms = dom_ms / dom_cnt
    achieved = ALG_BYTES[dom] * N / (avg_ms / 1e3) / 1e9
    peak, peak_src = measured_peaks()
    src_hash = kernel_source_hash()
    tpc = NCU_TRAFFIC_PER_CELL.get(src_hash)
    traffic = tpc * N if tpc is not None else None
    launches = sum(c for _, c in prof.values()) * args.steps // psteps + 2 * sums_calls

    # ---- e2e: through the C ABI with pinned host buffers, copies inside the region ----
    e2e = None
    if not args.no_e2e:
        out = [torch.empty(N, dtype=torch.float32).pin_memory() for _ in range(8)]
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        solver.upload(host)
        solver.step(args.steps)
        solver.download(out)
        e2e_s = time.perf_counter() - t0
        e2e_s = max_over_ranks(e2e_s, world)
        nb = 8 * N * 4
        e2e = {"value": total_cells / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": nb / args.steps, "d2h_bytes_per_step": nb / args.steps,
               "note": f"one job per rank: upload of the 8 FP32 fields from pinned host memory, "
                       f"{args.steps} steps, download of the 8 fields to pinned host memory"}
    solver.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = oracle_sample(n, args.cpu_edge, 1)
        cpu.pop("seconds", None)
        cpu["single_core"] = oracle_single_core(n, min(64, args.cpu_edge))

    issue = issue_object(dom, prof, NCU_INSTR_PER_CELL.get(src_hash), N,
                         torch.cuda.get_device_properties(local).multi_processor_count,
                         (clk or {}).get("sm_mhz") or 2070.0)

    if rank == 0:
        step_ms = max_ms / args.steps
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic", "config": workload_config(n),
                "roofline": {"bound": "hbm", "kernel": f"{dom} sweep (all axes)",
                             "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "peak_source": peak_src,
                             "traffic": traffic, "alg_bytes_per_cell": ALG_BYTES[dom],
                             "avg_launch_ms": avg_ms, "kernel_source": src_hash},
                "step_roofline": {"alg_bytes_per_cell": STEP_ALG_BYTES,
                                  "achieved": STEP_ALG_BYTES * N / (step_ms / 1e3) / 1e9,
                                  "frac": STEP_ALG_BYTES * N / (step_ms / 1e3) / 1e9 / peak},
                "issue": issue,
                "kernels_ms": {k: v[0] / max(v[1], 1) for k, v in prof.items() if v[1]},
                "kernels_timing": {"steps": psteps, "ms_per_step": prof_step_ms,
                                   "how": "kernel-by-kernel launches with an event pair "
                                          "around each, after the timed region (which "
                                          "replays one CUDA graph per step)"},
                "gpu_launches": launches, "e2e": e2e, "cpu_baseline": cpu, "clocks": clk}
        print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------
# Batched workload: 64 uneven grids, one persistent launch per call vs plain launches
# ------------------------------------------------------------------------------------

def run_batched(args, world, rank, local):
    import numpy as np
    import torch

    from paper_0908_4362_gb300 import autotune, build, mhd
    from paper_0908_4362_gb300 import inputs as I

    build.build()
    torch.cuda.set_device(local)
    count = args.instances
    problems = [I.batched_instance(i) for i in range(count)]
    cells = sum(p.ncells for p in problems)
    per_call = 3                               # steps per persistent launch (work list reused)
    k = max(per_call, (args.steps + per_call - 1) // per_call * per_call)
    tune = autotune.tune_batch(problems, nsteps=per_call)

    def timed(stream_handle, fn):
        st = torch.cuda.ExternalStream(stream_handle)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        fn()
        e1.record(st)
        e1.synchronize()
        return e0.elapsed_time(e1)

    # persistent batched form, at the tuned shapes and at the defaults
    sb = [mhd.Solver.from_problem(p, prec=mhd.FP32) for p in problems]
    batch = mhd.Batch(sb)
    nwarm = max(1, args.warmup // per_call)

    def run_batch():
        for _ in range(nwarm):
            batch.step(per_call)
        assert batch.sync() == mhd.MHD_OK
        ms = timed(batch.stream_handle(),
                   lambda: [batch.step(per_call) for _ in range(k // per_call)])
        assert batch.sync() == mhd.MHD_OK
        return ms

    clocks = start_clocks(local)
    ms_d = run_batch()
    autotune.apply(batch, tune, problems)
    ms_b = run_batch()
    ctas, items = batch.info()
    # one-at-a-time plain launches on one stream
    shared = torch.cuda.Stream()
    sp = [mhd.Solver(p.n, p.bc, p.h, p.gamma, p.cfl, prec=mhd.FP32, stream=shared.cuda_stream)
          for p in problems]
    for s_, p in zip(sp, problems):
        s_.init_fields(p.fields)
    for s_ in sp:
        s_.step(2 * nwarm * per_call)
    torch.cuda.synchronize()
    ms_p = timed(shared.cuda_stream, lambda: [s_.step(k) for s_ in sp])
    clk = clocks.stop()
    # every instance: tuned batch (after default and tuned launches) against plain steps
    for s_ in sp:
        s_.step(k)
    identical = all(np.array_equal(a.read(), b.read()) for a, b in zip(sb, sp))
    batch.close()
    for s_ in sb + sp:
        s_.close()
    large = run_batched_large(args, local, timed)
    if rank == 0:
        line = {"metric": "cell-updates/s (batched: 64 uneven grids, one persistent launch)",
                "value": cells * k / (ms_b / 1e3), "unit": UNIT, "n_gpus": world, "steps": k,
                "warmup": args.warmup, "ms_per_step": ms_b / k, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": f"{count} seeded 3D instances, edges log-uniform in "
                                       f"[48,192] per axis, random B direction, beta "
                                       f"log-uniform in [0.1,10], Gaussian pressure pulse",
                           "cells": cells, "steps_per_launch": per_call},
                "untuned": {"value": cells * k / (ms_d / 1e3), "ms_per_step": ms_d / k,
                            "how": "the same persistent launch at the default shapes"},
                "plain": {"value": cells * k / (ms_p / 1e3), "ms_per_step": ms_p / k,
                          "how": "mhd_step per instance, one after another on one stream"},
                "speedup_vs_plain": ms_p / ms_b, "results_identical": identical,
                "autotune": tune, "resident_ctas": ctas, "items_per_launch": items,
                "large_instances": large, "clocks": clk}
        print(json.dumps(line), flush=True)
    return 0


def run_batched_large(args, local, timed):
    """Large grids through the batched API, tuned (the autotuner may route them through the
    single-grid kernels), against plain single-grid steps: 4 blasts of 256^3."""
    import numpy as np
    import torch

    from paper_0908_4362_gb300 import autotune, mhd
    from paper_0908_4362_gb300 import inputs as I

    problems = [I.blast3d(256, offset=(0.01 * i, 0.0, 0.0)) for i in range(4)]
    cells = sum(p.ncells for p in problems)
    per_call = 3
    k = 6
    tune = autotune.tune_batch(problems, nsteps=per_call)
    sb = [mhd.Solver.from_problem(p, prec=mhd.FP32) for p in problems]
    batch = mhd.Batch(sb)
    autotune.apply(batch, tune, problems)
    batch.step(per_call)
    assert batch.sync() == mhd.MHD_OK
    ms_b = timed(batch.stream_handle(), lambda: [batch.step(per_call) for _ in range(k // per_call)])
    assert batch.sync() == mhd.MHD_OK
    shared = torch.cuda.Stream()
    sp = [mhd.Solver(p.n, p.bc, p.h, p.gamma, p.cfl, prec=mhd.FP32, stream=shared.cuda_stream)
          for p in problems]
    for s_, p in zip(sp, problems):
        s_.init_fields(p.fields)
    for s_ in sp:
        s_.step(per_call)
    torch.cuda.synchronize()
    ms_p = timed(shared.cuda_stream, lambda: [s_.step(k) for s_ in sp])
    identical = all(np.array_equal(a.read(), b.read()) for a, b in zip(sb, sp))
    batch.close()
    for s_ in sb + sp:
        s_.close()
    return {"workload": "4 magnetised blasts of 256^3 (offsets 0.01 i along x), FP32",
            "batched_tuned": cells * k / (ms_b / 1e3), "single_grid": cells * k / (ms_p / 1e3),
            "ratio": ms_p / ms_b, "results_identical": identical, "autotune": tune}


def run_serving(args, world, rank, local):
    """Served form: Poisson arrivals of OT-2D / blast-3D solves through the continuous-
    batching scheduler, against the same requests served one at a time with plain
    launches.  Three passes: saturation (a prefix of the trace, all requests at time 0:
    capacity of each form), then the whole trace with Poisson arrivals at `load` x the
    served capacity, through both forms (p50/p99 time to result)."""
    import numpy as np
    import torch

    from paper_0908_4362_gb300 import build, serve
    from paper_0908_4362_gb300 import inputs as I

    build.build()
    torch.cuda.set_device(local)
    # results are compared by SHA-1, computed on worker threads from a copy (hashlib releases
    # the interpreter lock), so that hashing does not hold up the serving loop
    import concurrent.futures as cf
    pool = cf.ThreadPoolExecutor(max_workers=8)

    def digest(a):
        buf = np.array(a, copy=True)
        return pool.submit(lambda: hashlib.sha1(buf).hexdigest())
    be = serve.GpuBackend()
    ics = serve.ICCache(pinned=True)
    base = I.serving_trace(args.requests, 0.0, seed=7 + rank)
    t_ic = time.perf_counter()
    for r in base:
        ics.get(r)
    t_ic = time.perf_counter() - t_ic
    mean_work = sum(r.ncells * r.steps for r in base) / len(base)
    budget = args.budget_gb * 1e9
    # warm-up of both forms
    warm = [dataclasses.replace(r, steps=6) for r in base[:8]]
    serve.Server(be, budget, ics=ics).run(warm)
    serve.serve_sequential(be, warm[:2], ics=ics)
    clocks = start_clocks(local)
    # saturation: capacity of each form on the same requests
    calib = [dataclasses.replace(r, arrival=0.0) for r in base[:args.calib]]
    sat_srv = serve.Server(be, budget, ics=ics)
    sat = serve.summarize(sat_srv.run(calib))
    sat_seq = serve.summarize(serve.serve_sequential(be, calib, ics=ics))
    capacity = sat["cell_updates_per_s"] / mean_work           # requests per second
    rate = args.load * capacity
    trace = I.serving_trace(args.requests, rate, seed=7 + rank)
    srv = serve.Server(be, budget, ics=ics, keep_results=digest)
    jobs = srv.run(trace)
    seq = serve.serve_sequential(be, trace, ics=ics, keep_results=digest)
    clk = clocks.stop()
    same = sum(a.result.result() == b.result.result()
               for a, b in zip(sorted(jobs, key=lambda j: j.req.rid),
                               sorted(seq, key=lambda j: j.req.rid)))
    pool.shutdown()
    s, q = serve.summarize(jobs), serve.summarize(seq)
    value = sum_over_ranks(s["cell_updates"], world) / max_over_ranks(s["makespan_s"], world)
    if rank == 0:
        line = {"metric": "cell-updates/s (served: Poisson arrivals of OT-2D and blast-3D solves)",
                "value": value, "unit": UNIT, "n_gpus": world, "steps": None,
                "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": f"{args.requests} requests, Poisson arrivals (seed 7) at "
                                       f"{args.load:g} x measured served capacity; 50% "
                                       f"Orszag-Tang 2D edge logU[128,1024], 50% blast 3D edge "
                                       f"logU[32,256] (edges rounded to 16), steps U{{50..500}}",
                           "budget_gb": args.budget_gb, "iter_ms": srv.iter_s * 1e3,
                           "timing": "host wall clock from the first arrival to the last "
                                     "result read back (uploads and downloads included)"},
                "served": s, "sequential": q,
                "saturation": {"requests": len(calib),
                               "served_cell_updates_per_s": sat["cell_updates_per_s"],
                               "sequential_cell_updates_per_s": sat_seq["cell_updates_per_s"],
                               "speedup": sat["cell_updates_per_s"] / sat_seq["cell_updates_per_s"],
                               "capacity_req_per_s": capacity,
                               "host_seconds": {k: round(v, 3) for k, v in sat_srv.times.items()}},
                "rate_req_per_s": rate, "peak_resident_gb": srv.peak_bytes / 1e9,
                "iterations": srv.iterations, "batch_rebuilds": srv.batch_rebuilds,
                "host_seconds": {k: round(v, 3) for k, v in srv.times.items()},
                "results_identical_alone_vs_mix": f"{same}/{len(jobs)}",
                "initial_states_s": t_ic, "clocks": clk}
        print(json.dumps(line), flush=True)
    return 0


def run_vis(args, world, rank, local):
    """Headless visualization kernels (Sect. 8): frame times of a colour slice of the 512^2
    Orszag-Tang density and of volume ray casts of the blast pressure at 128^3 and 512^3."""
    import torch

    from paper_0908_4362_gb300 import build, mhd
    from paper_0908_4362_gb300 import inputs as I

    build.build()
    torch.cuda.set_device(local)

    def frames(s, fn, reps=20):
        st = torch.cuda.ExternalStream(s.stream_handle())
        for _ in range(3):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        for _ in range(reps):
            fn()
        e1.record(st)
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    res = {}
    clocks = start_clocks(local)
    with mhd.Solver.from_problem(I.orszag_tang(512), prec=mhd.FP32) as s:
        s.step(30, sync=True)
        lo, hi = s.vis_range("rho")
        res["slice_ot512_ms"] = frames(s, lambda: s.vis_slice("rho", 2, 0, lo, hi))
    for n in (128, 512):
        with mhd.Solver.from_problem(I.blast3d(n), prec=mhd.FP32) as s:
            s.step(10, sync=True)
            lo, hi = s.vis_range("p")
            for axis in (0, 2):
                res[f"volume_blast{n}_axis{axis}_ms"] = frames(
                    s, lambda: s.vis_volume("p", axis, lo, hi, 0.02), reps=5)
    clk = clocks.stop()
    if rank == 0:
        line = {"metric": "frames/s (headless visualization kernels)",
                "value": 1e3 / res["slice_ot512_ms"], "unit": "frames/s", "n_gpus": world,
                "steps": None, "warmup": 3, "ms_per_step": res["slice_ot512_ms"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic",
                "config": {"workload": "colour slice of the 512^2 Orszag-Tang density "
                                       "(RGBA8); volume ray casts of the 3D blast pressure",
                           "timing": "CUDA events on the context stream, each call includes "
                                     "its stream synchronisation"},
                "frame_ms": res,
                "note": "the paper's OpenGL frame rates are unavailable on this box (no "
                        "graphics stack); these are the CUDA kernels producing the same images",
                "clocks": clk}
        print(json.dumps(line), flush=True)
    return 0


def _rel_l1_fields(a, b):
    """Per-field relative L1 difference of two (8, N) states; the momentum and B components
    share the L1 norm of their vector (a component can vanish identically)."""
    import numpy as np
    den = np.abs(b).sum(axis=1)
    den[1:4] = den[1:4].sum()
    den[5:8] = den[5:8].sum()
    return [float(np.abs(a[k] - b[k]).sum() / max(den[k], 1e-300)) for k in range(8)]


def run_precision(args, world, rank, local):
    """The precision variants on the 256^3 blast: FP32 sweeps with the pressure recovered in
    plain FP32, in FP64, and in compensated FP32 (error-free sums and products), and the FP64
    parity path (built without FMA contraction; bit-identical to the FP64 oracle in the
    parity tests).  Each FP32 variant's state after the same 13 steps is compared with the
    FP64 path's (relative L1 per field).  The pressure-recovery variants differ from plain
    FP32 mainly where the thermal energy is a small part of E (low beta, high Mach number);
    the parity tests check that case."""
    import numpy as np
    import torch

    from paper_0908_4362_gb300 import build, mhd
    from paper_0908_4362_gb300 import inputs as I

    build.build()
    torch.cuda.set_device(local)
    n = 256
    prob = I.blast3d(n)
    res = {}
    ref = None
    clocks = start_clocks(local)
    for name, prec, pm in (("fp64", mhd.FP64, mhd.PRESSURE_FP32),
                           ("fp32", mhd.FP32, mhd.PRESSURE_FP32),
                           ("fp32_fp64_pressure", mhd.FP32, mhd.PRESSURE_FP64),
                           ("fp32_compensated_pressure", mhd.FP32, mhd.PRESSURE_COMPENSATED)):
        with mhd.Solver(prob.n, prob.bc, prob.h, prob.gamma, prob.cfl, prec=prec,
                        pressure=pm) as s:
            s.init_fields(prob.fields)
            s.step(3, sync=True)
            st = torch.cuda.ExternalStream(s.stream_handle())
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            k = 10
            torch.cuda.synchronize()
            e0.record(st)
            s.step(k)
            e1.record(st)
            e1.synchronize()
            ms = e0.elapsed_time(e1) / k
            res[name] = {"ms_per_step": ms, "cell_updates_per_s": prob.ncells / (ms / 1e3)}
            state = s.read()
            if ref is None:
                ref = state
            else:
                err = _rel_l1_fields(state, ref)
                res[name]["rel_l1_vs_fp64_per_field"] = err
                res[name]["max_rel_l1_vs_fp64"] = max(err)
            del state
    clk = clocks.stop()
    if rank == 0:
        line = {"metric": "cell-updates/s by precision (256^3 blast)",
                "value": res["fp64"]["cell_updates_per_s"], "unit": UNIT, "n_gpus": world,
                "steps": 10, "warmup": 3, "ms_per_step": res["fp64"]["ms_per_step"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic",
                "config": {"workload": "3D magnetised blast 256^3, periodic",
                           "error": "state after 13 steps vs the FP64 path's (each variant "
                                    "takes its own dt from its own c_max)"},
                "variants": res, "clocks": clk}
        print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--cpu-edge", type=int, default=256)
    ap.add_argument("--ref-edge", type=int, default=64)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--workload", default="blast", choices=["blast", "batched", "serving", "vis",
                                                      "precision"])
    ap.add_argument("--instances", type=int, default=64)
    ap.add_argument("--requests", type=int, default=500)
    ap.add_argument("--calib", type=int, default=40)
    ap.add_argument("--load", type=float, default=0.8)
    ap.add_argument("--budget-gb", type=float, default=120.0)
    args = ap.parse_args(argv)
    args.warmup = max(args.warmup, 3)
    world, rank, local = dist_setup()
    try:
        if args.impl == "reference":
            return run_reference(args, world, rank)
        if args.workload == "batched":
            return run_batched(args, world, rank, local)
        if args.workload == "serving":
            return run_serving(args, world, rank, local)
        if args.workload == "vis":
            return run_vis(args, world, rank, local)
        if args.workload == "precision":
            return run_precision(args, world, rank, local)
        return run_ours(args, world, rank, local)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
