"""Pins of the visualization oracle (oracle/vis.py) against closed forms: the colour ramp
at and between its stops, the compositing recurrence on columns whose result is known,
and the derived quantities of uniform states."""
import numpy as np
import pytest

from oracle import vis
from paper_0908_4362_gb300 import inputs as I


def test_ramp_stops_and_midpoints():
    s = np.array([0.0, 0.25, 0.5, 0.75, 1.0])
    np.testing.assert_array_equal(vis.colour(s), vis.STOPS)
    mid = vis.colour(np.array([0.125, 0.625]))
    np.testing.assert_allclose(mid[0], [0.0, 0.0, 0.75])          # halfway dark blue -> blue
    np.testing.assert_allclose(mid[1], [0.5, 1.0, 0.5])           # halfway cyan -> yellow


def test_normalise_clamps_and_nan():
    s = vis.normalise(np.array([-1.0, 0.0, 2.5, 5.0, 9.0, np.nan]), 0.0, 5.0)
    np.testing.assert_array_equal(s, [0.0, 0.0, 0.5, 1.0, 1.0, 0.0])


def _column_state(values):
    """A 1 x 1 x k grid whose density column is `values` (other fields uniform)."""
    k = len(values)
    f = np.zeros((8, k))
    f[0] = values
    f[4] = 1.0
    return f, (1, 1, k)


def test_volume_opaque_first_cell_hides_the_rest():
    f, n = _column_state([10.0, 3.0, 7.0])
    img = vis.volume(f, n, (0, 0, 0), 5 / 3, vis.RHO, 2, 0.0, 10.0, opacity=1.0)
    np.testing.assert_allclose(img[0, 0], [1.0, 0.0, 0.0, 1.0])  # s = 1: red, alpha 1


def test_volume_two_layers_closed_form():
    f, n = _column_state([5.0, 10.0])        # s = 0.5 (cyan), then 1.0 (red)
    op = 0.6
    img = vis.volume(f, n, (0, 0, 0), 5 / 3, vis.RHO, 2, 0.0, 10.0, opacity=op)
    a1, a2 = 0.3, 0.6
    expect_c = a1 * np.array([0, 1, 1]) + (1 - a1) * a2 * np.array([1, 0, 0])
    np.testing.assert_allclose(img[0, 0, :3], expect_c)
    np.testing.assert_allclose(img[0, 0, 3], a1 + (1 - a1) * a2)


def test_volume_transparent_column_is_black():
    f, n = _column_state([0.0, 0.0, 0.0])
    img = vis.volume(f, n, (0, 0, 0), 5 / 3, vis.RHO, 2, 0.0, 1.0, opacity=1.0)
    np.testing.assert_array_equal(img[0, 0], [0.0, 0.0, 0.0, 0.0])


def test_quantities_of_uniform_state():
    rho, v, p, B = 2.0, (0.3, -0.4, 1.2), 0.7, (0.5, -1.0, 2.0)
    n = (3, 4, 5)
    f = I.conserved(np.full(n, rho), [np.full(n, c) for c in v], np.full(n, p),
                    [np.full(n, c) for c in B], 5 / 3, (0, 1, 0))
    np.testing.assert_allclose(vis.quantity(f, n, (0, 1, 0), 5 / 3, vis.P), p, rtol=1e-13)
    np.testing.assert_allclose(vis.quantity(f, n, (0, 1, 0), 5 / 3, vis.VMAG),
                               np.sqrt(sum(c * c for c in v)), rtol=1e-13)
    np.testing.assert_allclose(vis.quantity(f, n, (0, 1, 0), 5 / 3, vis.BMAG),
                               np.sqrt(sum(c * c for c in B)), rtol=1e-13)


def test_slice_layout_rows_are_the_higher_axis():
    n = (3, 4, 5)
    f = np.zeros((8, 60))
    rho = np.arange(60, dtype=float).reshape(n) + 1.0
    f[0] = rho.reshape(-1)
    f[4] = 1.0
    img = vis.slice_rgb(f, n, (0, 0, 0), 5 / 3, vis.RHO, 1, 2, 1.0, 60.0)   # plane y = 2
    assert img.shape == (5, 3, 3)                     # rows z, columns x
    expect = vis.colour(vis.normalise(rho[2, 2, 4], 1.0, 60.0))
    np.testing.assert_allclose(img[4, 2], expect)


def test_curve_of_brio_wu():
    prob = I.brio_wu(16)
    c = vis.curve(prob.fields, prob.n, prob.bc, prob.gamma, prob.h, vis.RHO)
    np.testing.assert_allclose(c[:, 0], (np.arange(16) + 0.5) / 16)
    np.testing.assert_array_equal(c[:, 1], np.where(np.arange(16) < 8, 1.0, 0.125))
