"""Parity at the benchmarked size: the 512^3 blast workload in the launch configuration
bench.py times (FP32, graph-replayed steps).  One step is compared with a full FP64
oracle step element by element; ten steps are checked by properties that hold at any
size (conservation of the periodic sums, discrete div B)."""
import os

import numpy as np
import pytest

import oracle
from paper_0908_4362_gb300 import inputs as I

pytestmark = pytest.mark.gpu

N = int(os.environ.get("MHD_FULLSIZE_N", "512"))


@pytest.fixture(scope="module")
def mhd():
    from paper_0908_4362_gb300 import build, mhd as m
    build.build()
    m.load_library()
    return m


def test_one_step_full_grid_vs_oracle(mhd):
    prob = I.blast3d(N)
    with mhd.Solver.from_problem(prob, prec=mhd.FP32) as s:
        s.step(1, sync=True)
        got = np.empty((8, prob.ncells), dtype=np.float32)
        s.download([got[k] for k in range(8)])
    ref = oracle.Oracle.from_problem(prob, copy=False)
    ref.step(1)
    absref = np.abs(ref.f).sum(axis=1)
    for k in range(8):
        # vector components share the L1 norm of their vector (momentum, B)
        den = absref[1:4].sum() if 1 <= k <= 3 else absref[5:8].sum() if k >= 5 else absref[k]
        num = np.abs(got[k].astype(np.float64) - ref.f[k]).sum()
        assert num / den <= 2e-5, (k, num / den)


def test_ten_steps_conserve_and_keep_divb(mhd):
    prob = I.blast3d(N)
    with mhd.Solver.from_problem(prob, prec=mhd.FP32) as s:
        s0 = s.sums()
        s.step(10, sync=True)
        s1 = s.sums()
        f = np.empty((8, prob.ncells), dtype=np.float32)
        s.download([f[k] for k in range(8)])
    # scales: sum of rho, E, |B| and, for momentum (zero at rest), the mass times the
    # largest signal speed
    absf = np.abs(f.astype(np.float64)).sum(axis=1)
    scale = np.array([absf[0], 0, 0, 0, absf[4], 0, 0, 0])
    scale[1:4] = absf[0] * 5.0
    scale[5:8] = absf[5:8].sum()
    drift = np.abs(s1 - s0) / scale
    assert np.all(drift <= 2e-6), drift
    b = [f[5 + a].reshape(N, N, N).astype(np.float64) for a in range(3)]
    div = sum(np.roll(b[a], -1, axis=a) - b[a] for a in range(3))
    assert np.abs(div).max() / np.abs(np.stack(b)).max() <= 1e-5
