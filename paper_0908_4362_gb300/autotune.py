"""Autotuner of the batched persistent launch: times candidate launch shapes (warp segments
per z work item, resident CTAs per SM) on throwaway copies of the workload and caches the
fastest per (GPU, grid shapes, steps per launch).  Launch shapes never change results, only
speed, so the tuned and untuned runs give the same bits."""
from __future__ import annotations

import hashlib
import json
import os
import time

from . import build as _build
from . import mhd

CACHE = os.path.join(_build.BUILD, "autotune.json")
# z_tile_warps 0 = chosen per sweep by the library (about 1024 items per z sweep)
CANDIDATES = [(w, c) for w in (0, 32, 64, 128, 256) for c in (0, 2)]


def _key(shapes, nsteps: int) -> str:
    import torch
    name = torch.cuda.get_device_name(0) if torch.cuda.is_available() else "cpu"
    h = hashlib.sha256(repr((name, sorted(tuple(s) for s in shapes), nsteps)).encode())
    return h.hexdigest()[:24]


def _load() -> dict:
    try:
        with open(CACHE) as fh:
            return json.load(fh)
    except Exception:
        return {}


def tune_batch(problems, nsteps: int = 3, repeats: int = 2, use_cache: bool = True) -> dict:
    """Return {"z_tile_warps": w, "ctas_per_sm": c, "ms": {...}} for these problems."""
    key = _key([p.n for p in problems], nsteps)
    cache = _load()
    if use_cache and key in cache:
        return cache[key]
    solvers = [mhd.Solver.from_problem(p, prec=mhd.FP32) for p in problems]
    timings = {}
    try:
        for w, c in CANDIDATES:
            with mhd.Batch(solvers, z_tile_warps=w, ctas_per_sm=c) as b:
                b.step(nsteps)                       # builds the work list and graph
                if b.sync() != mhd.MHD_OK:
                    continue
                best = float("inf")
                for _ in range(repeats):
                    t0 = time.perf_counter()
                    b.step(nsteps)
                    b.sync()
                    best = min(best, time.perf_counter() - t0)
                timings[f"{w},{c}"] = best * 1e3
    finally:
        for s in solvers:
            s.close()
    w, c = (int(v) for v in min(timings, key=timings.get).split(","))
    res = {"z_tile_warps": w, "ctas_per_sm": c, "ms": timings}
    cache[key] = res
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    with open(CACHE, "w") as fh:
        json.dump(cache, fh, indent=1)
    return res
