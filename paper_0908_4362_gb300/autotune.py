"""Autotuner of the batched persistent launch.

It picks the threads per CTA of the persistent kernel (128 or 256; the EMF rows of a
shared-row CT tile are its warps) and, per shape class of the batch's grids, the tile shapes
of mhd_batch_shape: the marching tile length of the x/y sweeps (128, 192 or 256 cells), the
CT form (shared EMF rows or one pipeline per pencil), the cells per lane of the z warp
segments (2 or 3), the warp segments per z work item, and for large grids the route through
the single-grid kernels instead of the persistent launch.  Each candidate is timed on the
workload itself (the whole batch, nsteps steps, best of `repeats`), by coordinate descent:
the batch-wide knob first, then each class, largest first, one knob at a time with the
others at their best so far.  The choice is cached per (GPU, grid shapes, steps per launch)
in _build/autotune.json.  Launch shapes never change results, only speed, so the tuned and
untuned runs give the same bits."""
from __future__ import annotations

import hashlib
import json
import math
import os
import time

from . import build as _build
from . import mhd

CACHE = os.path.join(_build.BUILD, "autotune.json")
VERSION = 3

# per-class knobs and their candidates, in tuning order ("alone" only for classes of at
# least ALONE_MIN_CELLS cells per grid on average: smaller grids leave most of the GPU idle
# alone)
KNOBS = (("alone", (0, 1)), ("march_len", (192, 128, 256)), ("ct_march", (0, 1)),
         ("seg_k", (0, 2, 3)), ("z_warps", (0, 32, 128)))
DEFAULTS = {"alone": 0, "march_len": 192, "ct_march": 0, "seg_k": 0, "z_warps": 0}
ALONE_MIN_CELLS = 1 << 19
THREADS = (128, 256)
MIN_GAIN = 0.01          # a candidate replaces the best so far when at least 1% faster


def shape_class(n) -> str:
    """Class of a grid shape: its cell count in octave pairs (2^17-2^19, 2^19-2^21, ...)."""
    cells = n[0] * n[1] * n[2]
    k = max(0, int(math.log2(max(cells, 1))) - 1) // 2
    return f"2^{2 * k + 1}-2^{2 * k + 3}"


def _key(shapes, nsteps: int) -> str:
    import torch
    name = torch.cuda.get_device_name(0) if torch.cuda.is_available() else "cpu"
    h = hashlib.sha256(repr((VERSION, name, sorted(tuple(s) for s in shapes), nsteps)).encode())
    return h.hexdigest()[:24]


def _load() -> dict:
    try:
        with open(CACHE) as fh:
            return json.load(fh)
    except Exception:
        return {}


def instance_shapes(problems, classes: dict) -> list:
    """Per-instance mhd_batch_shape dicts from per-class choices."""
    return [dict(classes.get(shape_class(p.n), {})) for p in problems]


def apply(batch, res: dict, problems) -> None:
    """Configure a mhd.Batch over `problems` with a tune_batch result."""
    batch.configure(threads_per_cta=res["threads_per_cta"], ctas_per_sm=res["ctas_per_sm"],
                    shapes=instance_shapes(problems, res["classes"]))


def tune_batch(problems, nsteps: int = 3, repeats: int = 3, use_cache: bool = True,
               log=None) -> dict:
    """Return {"threads_per_cta", "ctas_per_sm", "classes": {class: shape dict},
    "ms": {candidate: best ms}, "default_ms", "tuned_ms"} for these problems."""
    key = _key([p.n for p in problems], nsteps)
    cache = _load()
    if use_cache and key in cache:
        return cache[key]
    cls_of = [shape_class(p.n) for p in problems]
    cells = {}
    for p, c in zip(problems, cls_of):
        cells[c] = cells.get(c, 0) + p.ncells
    order = sorted(cells, key=cells.get, reverse=True)
    solvers = [mhd.Solver.from_problem(p, prec=mhd.FP32) for p in problems]
    timings = {}
    try:
        with mhd.Batch(solvers) as b:
            def run(nt, classes, label):
                shapes = [dict(classes.get(c, {})) for c in cls_of]
                b.configure(threads_per_cta=nt, shapes=shapes)
                b.step(nsteps)                       # builds the work list and graph
                if b.sync() != mhd.MHD_OK:
                    raise RuntimeError("batched step failed while tuning")
                best = float("inf")
                for _ in range(repeats):
                    t0 = time.perf_counter()
                    b.step(nsteps)
                    b.sync()
                    best = min(best, time.perf_counter() - t0)
                timings[label] = best * 1e3
                if log:
                    log(f"{label}: {best * 1e3:.2f} ms")
                return best

            nt = THREADS[0]
            best = float("inf")
            for t in THREADS:
                v = run(t, {}, f"threads={t}")
                if v < best:
                    nt, best = t, v
            default = timings[f"threads={THREADS[0]}"]
            classes = {c: {} for c in order}
            for c in order:
                for knob, cands in KNOBS:
                    if knob == "alone" and cells[c] // cls_of.count(c) < ALONE_MIN_CELLS:
                        continue
                    if classes[c].get("alone"):
                        break                        # single-grid kernels: no tile shapes
                    cur = classes[c].get(knob, DEFAULTS[knob])
                    for v in cands:
                        if v == cur:
                            continue
                        trial = {k: dict(s) for k, s in classes.items()}
                        trial[c][knob] = v
                        t = run(nt, trial, f"threads={nt} {c} {knob}={v}")
                        if t < best * (1.0 - MIN_GAIN):
                            classes, best = trial, t
    finally:
        for s in solvers:
            s.close()
    res = {"threads_per_cta": nt, "ctas_per_sm": 0,
           "classes": {c: classes[c] for c in order},
           "class_cells": {c: cells[c] for c in order},
           "ms": timings, "default_ms": default, "tuned_ms": best * 1e3, "nsteps": nsteps}
    cache[key] = res
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    with open(CACHE, "w") as fh:
        json.dump(cache, fh, indent=1)
    return res
