"""Build the CUDA library (sm_103a) in-tree: paper_0908_4362_gb300/_build/libmhd_gb300.so.

Each translation unit compiles in parallel with one -gencode for sm_103a, then nvcc links
them into one shared library exporting the C ABI of include/mhd.h."""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libmhd_gb300.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")

# (source, extra flags)
# FP32 kernels: fast division, square root and flush-to-zero, but no automatic FMA
# contraction: the fusions are written out (ffma/ffms, __fmaf_rn), so an inlined sweep body
# rounds the same in the single-grid kernels and in the persistent batched kernel
FP32_FLAGS = ["--ftz=true", "--prec-div=false", "--prec-sqrt=false", "--fmad=false"]
UNITS = [
    ("kernels_f32.cu", FP32_FLAGS),
    # FP64 is the parity path: no FMA contraction, so that its rounding matches the
    # oracle's operation for operation
    ("kernels_f64.cu", ["--fmad=false"]),
    ("mhd_capi.cu", []),
    ("mhd_noalloc.cu", []),
    # the batched persistent kernel runs the FP32 sweep bodies: same flags as their TU
    # (one unit per threads-per-CTA instantiation, compiled in parallel)
    ("mhd_batch.cu", FP32_FLAGS),
    ("mhd_batch_nt128.cu", FP32_FLAGS),
    ("mhd_batch_nt256.cu", FP32_FLAGS),
    ("mhd_vis.cu", []),
]


def _sources_mtime() -> float:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(ROOT, "include", "mhd.h"))
    files.append(os.path.abspath(__file__))
    return max(os.path.getmtime(f) for f in files if os.path.isfile(f))


# extra preprocessor definitions for every unit (tuning knobs of the kernels, e.g.
# "-DMHD_CT_CHUNK=4"); empty by default
DEFS = os.environ.get("MHD_NVCC_DEFS", "").split()


def _compile(src: str, extra: list, verbose: bool) -> str:
    obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
    cmd = [NVCC, "-c", "-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC",
           "-I", os.path.join(ROOT, "include"), *DEFS, *extra, os.path.join(CSRC, src), "-o", obj]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
    if verbose:
        sys.stderr.write(r.stderr)
    return obj


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _sources_mtime():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(lambda u: _compile(u[0], u[1], verbose), UNITS))
    tmp = LIB + f".{os.getpid()}.tmp"
    r = subprocess.run([NVCC, "-shared", *ARCH, "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
