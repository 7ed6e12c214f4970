"""FP64 CPU oracle of the visualization products (Sect. 8), numpy.

TEST INFRASTRUCTURE ONLY: imported by the test suite alone; it shares no code with the
CUDA library.

The paper renders 1D results as a vertex per cell (x position, selected value), 2D results
as a pixel per cell coloured by a transfer function, and 3D results by volume rendering.
It gives neither the transfer function nor the compositing rule, so the definitions here are
this project's readings, written out plainly:

- the selected value q of a cell: rho, p = (gamma-1)(E - |m|^2/(2 rho) - |B_c|^2/2), E,
  |v| = |m|/rho or |B_c|, where B_c averages each face component with the upper face along
  its own axis (wrapped for periodic axes, clamped for outflow ones), as for the CFL speed
  (Eq. "equat_CFL");
- s = (q - vmin)/(vmax - vmin), clamped to [0, 1] (NaN to 0);
- colour(s): linear interpolation between five stops at s = 0, 1/4, 1/2, 3/4, 1;
- volume rendering: one ray per cell column along the chosen axis, cells in increasing
  index order (front to back), opacity a = clamp(opacity s, 0, 1), and the emission-
  absorption recurrence C <- C + (1 - A) a colour, A <- A + (1 - A) a.
"""
from __future__ import annotations

import numpy as np

RHO, P, E, VMAG, BMAG = 0, 1, 2, 3, 4

STOPS = np.array([[0.0, 0.0, 0.5], [0.0, 0.0, 1.0], [0.0, 1.0, 1.0], [1.0, 1.0, 0.0],
                  [1.0, 0.0, 0.0]])


def quantity(fields: np.ndarray, n, bc, gamma: float, q: int) -> np.ndarray:
    """q per cell, shaped (nx, ny, nz), from the 8 conserved arrays."""
    f = np.asarray(fields, dtype=np.float64).reshape((8,) + tuple(n))
    rho, E_ = f[0], f[4]
    if q == RHO:
        return rho.copy()
    if q == E:
        return E_.copy()
    mm = f[1] ** 2 + f[2] ** 2 + f[3] ** 2
    if q == VMAG:
        return np.sqrt(mm) / rho
    bb = np.zeros_like(rho)
    for a in range(3):
        b = f[5 + a]
        if bc[a] == 0:
            up = np.roll(b, -1, axis=a)
        else:
            idx = np.minimum(np.arange(n[a]) + 1, n[a] - 1)
            up = np.take(b, idx, axis=a)
        bb += (0.5 * (b + up)) ** 2
    if q == BMAG:
        return np.sqrt(bb)
    if q == P:
        return (gamma - 1.0) * (E_ - 0.5 * mm / rho - 0.5 * bb)
    raise ValueError(q)


def normalise(q: np.ndarray, vmin: float, vmax: float) -> np.ndarray:
    s = (q - vmin) / (vmax - vmin)
    s = np.where(np.isnan(s), 0.0, s)
    return np.clip(s, 0.0, 1.0)


def colour(s: np.ndarray) -> np.ndarray:
    """RGB in [0, 1] for s in [0, 1] (any shape; a trailing axis of 3 is appended)."""
    x = np.asarray(s, dtype=np.float64) * 4.0
    k = np.minimum(np.floor(x).astype(int), 3)
    w = (x - k)[..., None]
    return STOPS[k] + w * (STOPS[k + 1] - STOPS[k])


def image_axes(axis: int) -> tuple:
    """The two grid axes (u, v) of an image normal to ``axis``, u < v."""
    return tuple(a for a in range(3) if a != axis)


def curve(fields, n, bc, gamma, h, q) -> np.ndarray:
    """(x, q) pairs of a 1D grid, shape (len, 2)."""
    axis = int(np.argmax(n)) if max(n) > 1 else 0
    vals = quantity(fields, n, bc, gamma, q).reshape(-1)
    x = (np.arange(n[axis]) + 0.5) * h
    return np.stack([x, vals], axis=1)


def slice_rgb(fields, n, bc, gamma, q, axis, index, vmin, vmax) -> np.ndarray:
    """Colour (float RGB in [0, 1]) of the plane normal to ``axis`` at ``index``, shaped
    (height = n[v], width = n[u], 3)."""
    vals = np.take(quantity(fields, n, bc, gamma, q), index, axis=axis)   # (n[u], n[v])
    return colour(normalise(vals, vmin, vmax)).transpose(1, 0, 2)


def volume(fields, n, bc, gamma, q, axis, vmin, vmax, opacity) -> np.ndarray:
    """Emission-absorption ray cast along ``axis``: RGBA float image (n[v], n[u], 4)."""
    s = normalise(quantity(fields, n, bc, gamma, q), vmin, vmax)
    s = np.moveaxis(s, axis, 0)                                  # (n[axis], n[u], n[v])
    C = np.zeros(s.shape[1:] + (3,))
    A = np.zeros(s.shape[1:])
    for k in range(s.shape[0]):
        a = np.clip(opacity * s[k], 0.0, 1.0)
        wgt = (1.0 - A) * a
        C += wgt[..., None] * colour(s[k])
        A += wgt
    out = np.concatenate([C, A[..., None]], axis=-1)
    return out.transpose(1, 0, 2)
