"""Pins of the FP64 oracle against exact solutions, conservation, div B, symmetry and
the paper's printed inputs.  CPU only."""
import math

import numpy as np
import pytest

import oracle
import pins
import riemann_exact
from paper_0908_4362_gb300 import inputs as I


@pytest.mark.parametrize("name", sorted(pins.ALL_PINS))
def test_pin(name):
    ok, detail = pins.ALL_PINS[name]()
    assert ok, f"{name}: {detail}"


def _golden(fname):
    rows = {}
    with open(f"{pins.__file__.rsplit('/', 1)[0]}/golden/{fname}") as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, *vals = line.split()
            rows[key] = [float(v) for v in vals]
    return rows


def test_exact_riemann_solver_star_state():
    """The exact solver reproduces the textbook star state of Sod's problem."""
    g = _golden("sod_star_state.txt")
    p, u = riemann_exact.star_state((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 1.4)
    assert abs(p - g["p_star"][0]) < 1e-5 and abs(u - g["u_star"][0]) < 1e-5
    x = np.array([0.5 + u * 0.2 - 1e-3, 0.5 + u * 0.2 + 1e-3])
    w = riemann_exact.sample((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 1.4, x, 0.2)
    assert abs(w[0, 0] - g["rho_star_left"][0]) < 1e-5
    assert abs(w[0, 1] - g["rho_star_right"][0]) < 1e-5


def test_inputs_match_paper_states():
    """The preset generators sample the initial states printed in Sect. 5."""
    g = _golden("paper_initial_states.txt")
    bw = I.brio_wu(16)
    f = bw.fields
    gam = g["bw_gamma"][0]
    left, right = 0, 15
    for side, c in (("bw_left", left), ("bw_right", right)):
        rho, p, bx, by, bz = g[side]
        assert f[0, c] == rho and f[5, c] == bx and f[6, c] == by and f[7, c] == bz
        assert abs((gam - 1) * (f[4, c] - 0.5 * (by * by + bz * bz + bx * bx)) - p) < 1e-14
    ot = I.orszag_tang(8, "paper")
    rho, p, b0sq4pi = g["ot_paper"]
    assert abs(ot.fields[0, 0] - rho) < 1e-14 * rho
    # Bx on the face (x_{-1/2}, y_0) = -B0 sin(2 pi y_0), y_0 = h/2
    y0 = 0.5 / 8
    assert abs(ot.fields[5, 0] + math.sqrt(b0sq4pi) * math.sin(2 * math.pi * y0)) < 1e-15
    assert abs((5 / 3 - 1) * (ot.fields[4, 0] - 0.5 * ot.fields[0, 0]
               * ((ot.fields[1, 0] ** 2 + ot.fields[2, 0] ** 2) / ot.fields[0, 0] ** 2)
               - 0.5 * (0.5 * (ot.fields[5, 0] + ot.fields[5, 8])) ** 2
               - 0.5 * (0.5 * (ot.fields[6, 0] + ot.fields[6, 1])) ** 2) - p) < 1e-14
    bl = I.blast3d(20, b_dir=(1, 1, 1))
    p_in, p_out, r, bcomp = g["blast_paper"]
    assert abs(bl.fields[5, 0] - bcomp) < 1e-15


def test_oracle_thread_invariance():
    """Pencils are independent, so the OpenMP and serial builds agree bit for bit."""
    pr = I.random_smooth((10, 12, 9), seed=11)
    a = oracle.Oracle.from_problem(pr, openmp=True)
    b = oracle.Oracle.from_problem(pr, openmp=False)
    a.step(2)
    b.step(2)
    assert np.array_equal(a.f, b.f)


def test_t_end_clip_lands_exactly():
    pr = I.brio_wu(64)
    o = oracle.Oracle.from_problem(pr)
    n = o.run_to(0.05)
    assert o.t == 0.05 and n > 0
    assert o.step(5, t_end=0.05) == 0     # no step once t_end is reached


def test_degenerate_axis_fluid_is_noop():
    """A periodic axis of length 1 gives identical interface fluxes: the fluid sweep along
    it changes nothing, bit for bit."""
    pr = I.random_smooth((6, 1, 5), seed=2)
    o = oracle.Oracle.from_problem(pr)
    o.fluid(1, 1e-3)
    assert np.array_equal(o.f[:5], pr.fields[:5])


def test_unphysical_flagged():
    pr = I.random_smooth((5, 4, 3), seed=4)
    f = pr.fields.copy()
    f[4, 7] = -10.0        # pressure so negative that the fast-speed radicand is < 0
    o = oracle.Oracle(pr.n, pr.bc, pr.h, pr.gamma, pr.cfl, f)
    o.fluid(0, 1e-4)
    assert o.status & oracle.UNPHYSICAL
