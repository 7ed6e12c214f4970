"""mhd_sums_noalloc: the FP64 field sums without any device allocation.

Callers that cannot allocate device memory (a process whose HBM is handed out by another
allocator under a fixed budget, or a thread that must not trigger the device-wide
synchronisation of cudaMalloc/cudaFree) use this entry point; its scratch is a fixed array
in the library's device image.  The test calls it through the C ABI on device copies of a
solver state, twice in a row on two different states, and compares with mhd_sums, the
entry point that uses the context's own scratch.  It needs no state from other tests, so
it passes alone in a fresh process and after the rest of the suite (this file is
collected last)."""
import ctypes as C

import numpy as np
import pytest

from paper_0908_4362_gb300 import inputs as I

pytestmark = pytest.mark.gpu

MAX_CELLS = 268435456    # MHD_SUMS_NOALLOC_MAX_CELLS in include/mhd.h


def _api():
    from paper_0908_4362_gb300 import build, mhd
    build.build()
    lib = mhd.load_library()
    fn = lib.mhd_sums_noalloc
    fn.argtypes = [C.POINTER(C.c_void_p), C.c_int, C.c_longlong, C.POINTER(C.c_double), C.c_void_p]
    fn.restype = C.c_int
    return mhd, fn


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_sums_noalloc_matches_context_sums(prec):
    import torch
    mhd, fn = _api()
    p = mhd.FP32 if prec == "fp32" else mhd.FP64
    dt = torch.float32 if p == mhd.FP32 else torch.float64
    # 48^3 = 110592 cells: two partial rows of the built-in scratch, one of them ragged
    prob = I.blast3d(48, offset=(0.3, 0.1, -0.2))
    with mhd.Solver.from_problem(prob, prec=p) as s:
        for _ in range(2):                       # two calls in a row, two different states
            s.step(3, sync=True)
            ref = s.sums()
            bufs = [torch.empty(prob.ncells, dtype=dt, device="cuda") for _ in range(8)]
            s.download(bufs)
            torch.cuda.synchronize()
            out = np.full(8, np.nan)
            ptrs = (C.c_void_p * 8)(*[b.data_ptr() for b in bufs])
            st = fn(ptrs, 0 if p == mhd.FP32 else 1, prob.ncells,
                    out.ctypes.data_as(C.POINTER(C.c_double)), None)
            assert st == mhd.MHD_OK
            l1 = np.array([float(b.double().abs().sum()) for b in bufs])
            # the two reductions differ only in their summation order
            assert np.all(np.abs(out - ref) <= 1e-12 * l1), (out, ref)


def test_sums_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    mhd, fn = _api()
    buf = torch.zeros(8, dtype=torch.float32, device="cuda")
    ptrs = (C.c_void_p * 8)(*([buf.data_ptr()] * 8))
    out = np.zeros(8)
    # rejected before any launch, so the short buffers are never read
    st = fn(ptrs, 0, MAX_CELLS + 1, out.ctypes.data_as(C.POINTER(C.c_double)), None)
    assert st == mhd.MHD_ERR_INVALID
