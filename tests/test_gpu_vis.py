"""Visualization kernels (Sect. 8, headless) against the FP64 visualization oracle: the
1D curve, colour slices along every axis (RGBA8: each channel within half a level of the
oracle's colour plus the state's rounding), volume ray casts along every axis, and the
value range."""
import numpy as np
import pytest

from oracle import vis
from paper_0908_4362_gb300 import inputs as I

pytestmark = pytest.mark.gpu

QS = ["rho", "p", "E", "vmag", "bmag"]


@pytest.fixture(scope="module")
def mhd():
    from paper_0908_4362_gb300 import build, mhd as m
    build.build()
    return m


def _solver(mhd, prob, prec):
    p = mhd.FP64 if prec == "fp64" else mhd.FP32
    return mhd.Solver.from_problem(prob, prec=p)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_curve_brio_wu(mhd, prec):
    prob = I.brio_wu(200)
    with _solver(mhd, prob, prec) as s:
        s.step(5, sync=True)
        f = s.read()
        for qi, q in enumerate(QS):
            got = s.vis_curve(q).cpu().numpy()
            ref = vis.curve(f, prob.n, prob.bc, prob.gamma, prob.h, qi)
            np.testing.assert_allclose(got, ref, rtol=2e-6, atol=1e-6)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_slice_every_axis(mhd, prec, axis):
    prob = I.random_smooth((23, 17, 29), seed=21, bc=(0, 1, 0))
    with _solver(mhd, prob, prec) as s:
        s.step(2, sync=True)
        f = s.read()
        for qi, q in enumerate(QS):
            lo, hi = s.vis_range(q)
            qq = vis.quantity(f, prob.n, prob.bc, prob.gamma, qi)
            assert abs(lo - qq.min()) <= 1e-5 * abs(qq).max() + 1e-30
            assert abs(hi - qq.max()) <= 1e-5 * abs(qq).max() + 1e-30
            vmin, vmax = float(qq.min()), float(qq.max())
            index = prob.n[axis] // 3
            img = s.vis_slice(q, axis, index, vmin, vmax).cpu().numpy()
            ref = vis.slice_rgb(f, prob.n, prob.bc, prob.gamma, qi, axis, index, vmin, vmax)
            assert img.shape == ref.shape[:2] + (4,)
            assert np.all(img[..., 3] == 255)
            dev = np.abs(img[..., :3].astype(np.float64) - 255.0 * ref)
            assert dev.max() <= 0.5 + 0.01, (q, dev.max())


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_volume_every_axis(mhd, prec, axis):
    prob = I.blast3d(24, offset=(0.3, -0.2, 0.1))
    with _solver(mhd, prob, prec) as s:
        s.step(4, sync=True)
        f = s.read()
        for qi, q in enumerate(["rho", "p"]):
            qq = vis.quantity(f, prob.n, prob.bc, prob.gamma, qi)
            vmin, vmax = float(qq.min()), float(qq.max())
            got = s.vis_volume(q, axis, vmin, vmax, opacity=0.08).cpu().numpy()
            ref = vis.volume(f, prob.n, prob.bc, prob.gamma, qi, axis, vmin, vmax, 0.08)
            tol = 1e-6 if prec == "fp64" else 2e-5      # the image itself is FP32
            np.testing.assert_allclose(got, ref, rtol=0, atol=tol)


def test_orszag_tang_frame(mhd):
    """A 2D frame of the Orszag-Tang density (the paper's 2D visualization example)."""
    prob = I.orszag_tang(128)
    with _solver(mhd, prob, "fp32") as s:
        s.step(20, sync=True)
        f = s.read()
        img = s.vis_slice("rho", 2, 0).cpu().numpy()
        qq = vis.quantity(f, prob.n, prob.bc, prob.gamma, vis.RHO)
        ref = vis.slice_rgb(f, prob.n, prob.bc, prob.gamma, vis.RHO, 2, 0, float(qq.min()),
                            float(qq.max()))
        assert img.shape == (128, 128, 4)
        assert np.abs(img[..., :3] - 255.0 * ref).max() <= 0.51


def test_invalid_arguments(mhd):
    prob = I.random_smooth((8, 8, 8), seed=3)
    with _solver(mhd, prob, "fp32") as s:
        with pytest.raises(mhd.MhdError):
            s.vis_slice("rho", 3, 0, 0.0, 1.0)
        with pytest.raises(mhd.MhdError):
            s.vis_slice("rho", 0, 8, 0.0, 1.0)
        with pytest.raises(mhd.MhdError):
            s.vis_volume("rho", 0, 1.0, 1.0)
        with pytest.raises(mhd.MhdError):
            s.vis_curve("rho")                      # not a 1D grid
        import ctypes
        import torch
        buf = torch.empty(8 * 8 * 4, dtype=torch.uint8, device="cuda")
        ptr = ctypes.c_void_p(buf.data_ptr())
        assert s.lib.mhd_vis_slice(s.ctx, 0, 3, 0, 0.0, 1.0, ptr) == mhd.MHD_ERR_INVALID
        assert s.lib.mhd_vis_slice(s.ctx, 9, 0, 0, 0.0, 1.0, ptr) == mhd.MHD_ERR_INVALID
        assert s.lib.mhd_vis_slice(s.ctx, 0, 0, 0, 0.0, 1.0, None) == mhd.MHD_ERR_INVALID
