"""Seeded synthetic initial conditions shaped like the paper's test problems.

This module serves both the CUDA path (benchmarks, batch and serving workloads) and the
FP64 oracle's tests.  It holds none of the scheme's arithmetic: it only samples the
initial states of Sect. 5 (Brio-Wu, Orszag-Tang, 3D blast), the batched and served
workload mixes, and a few smooth problems with known exact solutions (linear and
circularly polarised waves), then converts primitive variables to the 8 conserved
arrays with the equation of state's definition of E (Sect. 3: p = (gamma-1)(E - rho v^2/2
- B^2/2)).  B is sampled directly on the cell faces (Eq. "equat_b"); the B^2 in E uses the
cell-centred average of the two faces, as the scheme does.

Layout: fields is an (8, nx*ny*nz) float64 array, order (rho, mx, my, mz, E, Bx, By, Bz),
flat index (x*ny + y)*nz + z.  Cell centres sit at (i + 1/2) h, faces at i h.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Sequence

import numpy as np

PERIODIC, OUTFLOW = 0, 1
FIELDS = ("rho", "mx", "my", "mz", "E", "Bx", "By", "Bz")


@dataclasses.dataclass
class Problem:
    name: str
    n: tuple            # (nx, ny, nz)
    bc: tuple           # per axis, PERIODIC or OUTFLOW
    h: float
    gamma: float
    cfl: float
    fields: np.ndarray  # (8, N) float64
    t_end: float = -1.0

    @property
    def ncells(self) -> int:
        return int(self.n[0] * self.n[1] * self.n[2])

    def copy(self) -> "Problem":
        return dataclasses.replace(self, fields=self.fields.copy())


def _face_avg(b: np.ndarray, axis: int, bc: int) -> np.ndarray:
    """Average of the two faces of each cell along ``axis`` (the upper face clamped for
    outflow boundaries, wrapped for periodic ones)."""
    if bc == PERIODIC:
        up = np.roll(b, -1, axis=axis)
    else:
        idx = np.minimum(np.arange(b.shape[axis]) + 1, b.shape[axis] - 1)
        up = np.take(b, idx, axis=axis)
    return 0.5 * (b + up)


def conserved(rho, v, p, B, gamma, bc) -> np.ndarray:
    """Pack primitive cell values and face-centred B (each shaped (nx,ny,nz)) into the
    8 conserved arrays."""
    rho = np.asarray(rho, dtype=np.float64)
    shape = rho.shape
    v = [np.broadcast_to(np.asarray(c, dtype=np.float64), shape) for c in v]
    B = [np.broadcast_to(np.asarray(c, dtype=np.float64), shape).copy() for c in B]
    p = np.broadcast_to(np.asarray(p, dtype=np.float64), shape)
    bcen = [_face_avg(B[a], a, bc[a]) for a in range(3)]
    ke = 0.5 * rho * (v[0] ** 2 + v[1] ** 2 + v[2] ** 2)
    me = 0.5 * (bcen[0] ** 2 + bcen[1] ** 2 + bcen[2] ** 2)
    E = p / (gamma - 1.0) + ke + me
    out = np.empty((8,) + shape, dtype=np.float64)
    out[0] = rho
    for a in range(3):
        out[1 + a] = rho * v[a]
        out[5 + a] = B[a]
    out[4] = E
    return out.reshape(8, -1)


def _centres(n: int, h: float) -> np.ndarray:
    return (np.arange(n) + 0.5) * h


def _faces(n: int, h: float) -> np.ndarray:
    return np.arange(n) * h


def _rot(vec: Sequence, axis: int) -> list:
    """Place the components (n, t1, t2) of a 1D problem on axis ``axis``: the problem's x
    goes to ``axis``, y to (axis+1)%3, z to (axis+2)%3."""
    out = [None, None, None]
    for k in range(3):
        out[(axis + k) % 3] = vec[k]
    return out


def _shape1d(n: int, axis: int) -> tuple:
    s = [1, 1, 1]
    s[axis] = n
    return tuple(s)


def _line(x: np.ndarray, axis: int) -> np.ndarray:
    return x.reshape(_shape1d(x.size, axis))


# ------------------------------------------------------------------------------------
# Paper test problems (Sect. 5)
# ------------------------------------------------------------------------------------

def brio_wu(n: int = 512, axis: int = 0, gamma: float = 2.0, cfl: float = 0.8,
            t_end: float = 0.1) -> Problem:
    """Brio-Wu shock tube (Sect. 5.1.1) on [0,1] along ``axis``; outflow along the tube,
    periodic across it."""
    h = 1.0 / n
    xc = _centres(n, h)
    left = xc < 0.5
    rho = np.where(left, 1.0, 0.125)
    p = np.where(left, 1.0, 0.1)
    bt1 = np.where(left, 1.0, -1.0)     # transverse faces sit at the cell centre along x
    shape = _shape1d(n, axis)
    z = np.zeros(shape)
    B = _rot([np.full(shape, 0.75), _line(bt1, axis), z], axis)
    v = _rot([z, z, z], axis)
    bc = _rot([OUTFLOW, PERIODIC, PERIODIC], axis)
    f = conserved(_line(rho, axis), v, _line(p, axis), B, gamma, bc)
    return Problem(f"brio_wu_{n}_axis{axis}", shape, tuple(bc), h, gamma, cfl, f, t_end)


def dai_woodward(n: int = 512, axis: int = 0, cfl: float = 0.7, t_end: float = 0.2) -> Problem:
    """MHD shock tube of Sect. 5.1.2.  The printed left/right B_x "2 sqrt(4 pi)" is read as
    2/sqrt(4 pi), the value that its neighbouring entries and the source problem use."""
    gamma = 5.0 / 3.0
    h = 1.0 / n
    xc = _centres(n, h)
    left = xc < 0.5
    s = math.sqrt(4.0 * math.pi)
    rho = np.where(left, 1.08, 1.0)
    p = np.where(left, 0.95, 1.0)
    vx = np.where(left, 1.2, 0.0)
    vy = np.where(left, 0.01, 0.0)
    vz = np.where(left, 0.5, 0.0)
    by = np.where(left, 3.6 / s, 4.0 / s)
    bz = np.full(n, 2.0 / s)
    shape = _shape1d(n, axis)
    B = _rot([np.full(shape, 2.0 / s), _line(by, axis), _line(bz, axis)], axis)
    v = _rot([_line(vx, axis), _line(vy, axis), _line(vz, axis)], axis)
    bc = _rot([OUTFLOW, PERIODIC, PERIODIC], axis)
    f = conserved(_line(rho, axis), v, _line(p, axis), B, gamma, bc)
    return Problem(f"dai_woodward_{n}_axis{axis}", shape, tuple(bc), h, gamma, cfl, f, t_end)


def orszag_tang(n: int = 512, variant: str = "config", cfl: float = 0.7,
                t_end: float = 0.5, ny: int | None = None) -> Problem:
    """Orszag-Tang vortex on the periodic unit square (Sect. 5.2.1), nz = 1.

    variant "config": rho = 25/9, p = 5/3, B0 = 1/sqrt(4 pi) (the benchmarked workload);
    variant "paper": rho = 25/(36 pi), p = 5/(12 pi), B0 = 1/sqrt(4 pi) (as printed).
    v = (-sin 2 pi y, sin 2 pi x, 0), B = B0 (-sin 2 pi y, sin 4 pi x, 0).
    """
    ny = n if ny is None else ny
    gamma = 5.0 / 3.0
    h = 1.0 / n
    if variant == "config":
        rho0, p0 = 25.0 / 9.0, 5.0 / 3.0
    elif variant == "paper":
        rho0, p0 = 25.0 / (36.0 * math.pi), 5.0 / (12.0 * math.pi)
    else:
        raise ValueError(variant)
    b0 = 1.0 / math.sqrt(4.0 * math.pi)
    xc, yc = _centres(n, h), _centres(ny, h)
    X, Y = np.meshgrid(xc, yc, indexing="ij")
    X, Y = X[:, :, None], Y[:, :, None]
    vx = -np.sin(2 * np.pi * Y) * np.ones_like(X)
    vy = np.sin(2 * np.pi * X) * np.ones_like(Y)
    # Bx on x-faces (x_{i-1/2}, y_j) depends on y only; By on y-faces (x_i, y_{j-1/2}) on x
    # only, so the discrete divergence is exactly zero.
    bx = -b0 * np.sin(2 * np.pi * Y) * np.ones_like(X)
    by = b0 * np.sin(4 * np.pi * X) * np.ones_like(Y)
    shape = (n, ny, 1)
    rho = np.full(shape, rho0)
    f = conserved(rho, [vx, vy, np.zeros(shape)], np.full(shape, p0),
                  [bx, by, np.zeros(shape)], gamma, (PERIODIC,) * 3)
    return Problem(f"orszag_tang_{variant}_{n}x{ny}", shape, (PERIODIC,) * 3, h, gamma, cfl,
                   f, t_end)


def blast2d(n: int = 512, cfl: float = 0.7, t_end: float = 0.2) -> Problem:
    """2D magnetised blast wave of Sect. 5.2.2 on the periodic unit square, nz = 1: rho = 1,
    v = 0, B = (1, 1, 0)/sqrt(2), gamma = 5/3, p = 10 inside r < 0.1 about (0.5, 0.5)
    (cell centres) and 0.1 outside.  The problem's list also prints "p = 5/(12 pi)" on the
    line with rho and gamma; that value contradicts the inside/outside pressures printed
    just above it and is read as left over from the Orszag-Tang list."""
    gamma = 5.0 / 3.0
    h = 1.0 / n
    xc = _centres(n, h)
    r2 = (xc - 0.5)[:, None, None] ** 2 + (xc - 0.5)[None, :, None] ** 2
    shape = (n, n, 1)
    p = np.where(r2 < 0.01, 10.0, 0.1) * np.ones(shape)
    z = np.zeros(shape)
    b = 1.0 / math.sqrt(2.0)
    f = conserved(np.ones(shape), [z, z, z], p, [np.full(shape, b), np.full(shape, b), z],
                  gamma, (PERIODIC,) * 3)
    return Problem(f"blast2d_{n}", shape, (PERIODIC,) * 3, h, gamma, cfl, f, t_end)


def rotor(n: int = 512, variant: int = 1, cfl: float = 0.7, offset=(0.0, 0.0)) -> Problem:
    """MHD rotor of Sect. 5.2.3 on the unit square, nz = 1, outflow in x and y.

    A dense disk (rho = 10, r < r0 = 0.1 about (0.5, 0.5)) rotates rigidly at angular
    speed v0/r0; between r0 and r1 = 0.115 rho = 1 + 9f and the rotation fades with
    f = (r1 - r)/(r1 - r0); outside rho = 1 and v = 0; p and B = (B0, 0, 0) are uniform.
    variant 1: v0 = 2, p = 1, gamma = 1.4, B0 = 5/sqrt(4 pi), t_max = 0.15;
    variant 2: v0 = 1, p = 0.5, gamma = 5/3, B0 = 2.5/sqrt(4 pi), t_max = 0.295.
    Readings: the taper's v_y is printed as -f v0 (x - 0.5)/r, whose sign would reverse the
    rotation across r0 (the disk's v_y is +v0 (x - 0.5)/r0); it is read as +f v0 (x-0.5)/r.
    The boundary type is not stated; outflow (zero gradient) is used.  `offset` moves the
    disk's centre (box units; the paper's is 0, 0)."""
    if variant == 1:
        v0, p0, gamma, b0, t_end = 2.0, 1.0, 1.4, 5.0 / math.sqrt(4 * math.pi), 0.15
    elif variant == 2:
        v0, p0, gamma, b0, t_end = 1.0, 0.5, 5.0 / 3.0, 2.5 / math.sqrt(4 * math.pi), 0.295
    else:
        raise ValueError(variant)
    r0, r1 = 0.1, 0.115
    h = 1.0 / n
    xc = _centres(n, h)
    X = (xc - 0.5 - offset[0])[:, None, None] * np.ones((1, n, 1))
    Y = (xc - 0.5 - offset[1])[None, :, None] * np.ones((n, 1, 1))
    r = np.sqrt(X * X + Y * Y)
    f = (r1 - r) / (r1 - r0)
    inner, taper = r < r0, (r >= r0) & (r < r1)
    rho = np.where(inner, 10.0, np.where(taper, 1.0 + 9.0 * f, 1.0))
    rs = np.where(r > 0, r, 1.0)
    vx = np.where(inner, -v0 * Y / r0, np.where(taper, -f * v0 * Y / rs, 0.0))
    vy = np.where(inner, v0 * X / r0, np.where(taper, f * v0 * X / rs, 0.0))
    shape = (n, n, 1)
    z = np.zeros(shape)
    bc = (OUTFLOW, OUTFLOW, PERIODIC)
    fl = conserved(rho, [vx, vy, z], np.full(shape, p0), [np.full(shape, b0), z, z], gamma, bc)
    return Problem(f"rotor{variant}_{n}", shape, bc, h, gamma, cfl, fl, t_end)


def blast3d(n: int = 512, b_dir=(1.0, 1.0, 0.0), b_mag: float = 1.0, p_in: float = 10.0,
            p_out: float = 0.1, radius: float = 0.1, cfl: float = 0.7,
            shape: tuple | None = None, offset=(0.0, 0.0, 0.0)) -> Problem:
    """Magnetised blast wave in the periodic unit cube (Sect. 5.3): rho = 1, v = 0,
    p = p_in inside |x - c| < radius (cell centres), else p_out, uniform B along b_dir.
    With offset = 0 the blast is mirror symmetric about the grid's middle faces.
    The benchmarked workload uses B = (1,1,0)/sqrt(2); the paper's run uses (1,1,1)/sqrt(3)."""
    shape = (n, n, n) if shape is None else tuple(shape)
    h = 1.0 / max(shape)
    gamma = 5.0 / 3.0
    d = np.asarray(b_dir, dtype=np.float64)
    d = d / np.linalg.norm(d) * b_mag
    c = [_centres(m, h) for m in shape]
    # offset (in cells) moves the blast off the mirror planes of the grid
    centre = [(0.5 * m + offset[a]) * h for a, m in enumerate(shape)]
    r2 = ((c[0] - centre[0]) ** 2)[:, None, None] + ((c[1] - centre[1]) ** 2)[None, :, None] \
        + ((c[2] - centre[2]) ** 2)[None, None, :]
    p = np.where(r2 < radius * radius, p_in, p_out)
    rho = np.ones(shape)
    z = np.zeros(shape)
    B = [np.full(shape, d[0]), np.full(shape, d[1]), np.full(shape, d[2])]
    f = conserved(rho, [z, z, z], p, B, gamma, (PERIODIC,) * 3)
    return Problem(f"blast3d_{shape[0]}x{shape[1]}x{shape[2]}", shape, (PERIODIC,) * 3, h,
                   gamma, cfl, f)


# ------------------------------------------------------------------------------------
# Smooth problems with exact solutions (used to pin the oracle)
# ------------------------------------------------------------------------------------

def sod(n: int, axis: int = 0, gamma: float = 1.4, cfl: float = 0.7, t_end: float = 0.2,
        x0: float = 0.5) -> Problem:
    """Sod's shock tube with B = 0 (pure gas dynamics)."""
    h = 1.0 / n
    xc = _centres(n, h)
    left = xc < x0
    rho = np.where(left, 1.0, 0.125)
    p = np.where(left, 1.0, 0.1)
    shape = _shape1d(n, axis)
    z = np.zeros(shape)
    bc = _rot([OUTFLOW, PERIODIC, PERIODIC], axis)
    f = conserved(_line(rho, axis), [z, z, z], _line(p, axis), [z, z, z], gamma, bc)
    return Problem(f"sod_{n}_axis{axis}", shape, tuple(bc), h, gamma, cfl, f, t_end)


def alfven_circular(n: int, axis: int = 0, amp: float = 0.1, rho0: float = 1.0,
                    p0: float = 0.1, bn: float = 1.0, cfl: float = 0.7,
                    gamma: float = 5.0 / 3.0) -> Problem:
    """Circularly polarised Alfven wave travelling along +axis on the periodic unit
    interval: B_t = amp (cos 2 pi x, sin 2 pi x), v_t = -B_t/sqrt(rho), v_n = 0.  |B| and the
    total pressure are uniform, so it is an exact nonlinear solution; the phase speed is
    bn/sqrt(rho0), the period 1/that."""
    h = 1.0 / n
    xc = _centres(n, h)
    bt1 = amp * np.cos(2 * np.pi * xc)
    bt2 = amp * np.sin(2 * np.pi * xc)
    s = math.sqrt(rho0)
    shape = _shape1d(n, axis)
    B = _rot([np.full(shape, bn), _line(bt1, axis), _line(bt2, axis)], axis)
    v = _rot([np.zeros(shape), _line(-bt1 / s, axis), _line(-bt2 / s, axis)], axis)
    f = conserved(np.full(shape, rho0), v, np.full(shape, p0), B, gamma, (PERIODIC,) * 3)
    prob = Problem(f"alfven_{n}_axis{axis}", shape, (PERIODIC,) * 3, h, gamma, cfl, f,
                   t_end=s / bn)
    return prob


def entropy_wave(n: int, axis: int = 0, amp: float = 0.2, v0: float = 1.0, p0: float = 1.0,
                 b=(0.5, 0.3, -0.2), cfl: float = 0.7, gamma: float = 5.0 / 3.0) -> Problem:
    """Density wave rho = 1 + amp sin 2 pi x advected at uniform v_n = v0 with uniform p and
    B: an exact solution (a contact) that returns to itself after t = 1/v0."""
    h = 1.0 / n
    xc = _centres(n, h)
    rho = 1.0 + amp * np.sin(2 * np.pi * xc)
    shape = _shape1d(n, axis)
    one = np.ones(shape)
    B = _rot([b[0] * one, b[1] * one, b[2] * one], axis)
    v = _rot([v0 * one, 0 * one, 0 * one], axis)
    f = conserved(_line(rho, axis), v, p0 * one, B, gamma, (PERIODIC,) * 3)
    return Problem(f"entropy_{n}_axis{axis}", shape, (PERIODIC,) * 3, h, gamma, cfl, f,
                   t_end=1.0 / abs(v0))


def fast_wave_eigen(rho0=1.0, p0=0.6, bn=1.0, bt=1.5, gamma=5.0 / 3.0):
    """Right-going fast magnetosonic eigenvector of the 1D equations linearised about a
    uniform state at rest with B = (bn, bt, 0), derived from the primitive equations
    rho_t + rho0 vx_x = 0, rho0 vx_t + p_x + bt By_x = 0, rho0 vy_t - bn By_x = 0,
    By_t + bt vx_x - bn vy_x = 0, p_t + gamma p0 vx_x = 0.
    Returns (speed, drho, dvx, dvy, dBy, dp) normalised to dvx = 1."""
    a2 = gamma * p0 / rho0
    bx2 = bn * bn / rho0
    b2 = (bn * bn + bt * bt) / rho0
    lam2 = 0.5 * ((a2 + b2) + math.sqrt((a2 + b2) ** 2 - 4.0 * a2 * bx2))
    lam = math.sqrt(lam2)
    dvx = 1.0
    drho = rho0 * dvx / lam
    dp = gamma * p0 * dvx / lam
    dby = bt * lam * dvx / (lam2 - bx2)
    dvy = -bn * dby / (rho0 * lam)
    return lam, drho, dvx, dvy, dby, dp


def fast_wave(n: int, axis: int = 0, amp: float = 1e-6, cfl: float = 0.7, v0: float = 0.0,
              **kw) -> Problem:
    """Small-amplitude fast magnetosonic wave on a background moving at v0 along the axis
    (a Galilean shift of the eigenvector); returns to itself after t = 1/(v0 + speed)."""
    rho0, p0, bn, bt = kw.get("rho0", 1.0), kw.get("p0", 0.6), kw.get("bn", 1.0), kw.get("bt", 1.5)
    gamma = kw.get("gamma", 5.0 / 3.0)
    lam, drho, dvx, dvy, dby, dp = fast_wave_eigen(rho0, p0, bn, bt, gamma)
    h = 1.0 / n
    s = amp * np.sin(2 * np.pi * _centres(n, h))
    shape = _shape1d(n, axis)
    B = _rot([np.full(shape, bn), _line(bt + dby * s, axis), np.zeros(shape)], axis)
    v = _rot([_line(v0 + dvx * s, axis), _line(dvy * s, axis), np.zeros(shape)], axis)
    f = conserved(_line(rho0 + drho * s, axis), v, _line(p0 + dp * s, axis), B, gamma,
                  (PERIODIC,) * 3)
    return Problem(f"fast_{n}_axis{axis}", shape, (PERIODIC,) * 3, h, gamma, cfl, f,
                   t_end=1.0 / (v0 + lam))


def passive_field_2d(n: int, amp: float = 1e-3, drho: float = 0.5, v=(1.0, 1.0),
                     cfl: float = 0.7, gamma: float = 5.0 / 3.0) -> Problem:
    """A weak face field B = amp (sin 2 pi y, cos 2 pi x, 0) carried by a uniform flow v
    across a density wave rho = 1 + drho sin 2 pi (x + y), uniform p, on the periodic unit
    square.  The field is too weak to push the flow (forces ~ amp^2), so the exact solution
    is the initial state translated by v t; with v = (1, 1) it returns after t = 1."""
    h = 1.0 / n
    xc, xf = _centres(n, h), _centres(n, h)
    X, Y = np.meshgrid(xc, xf, indexing="ij")
    X, Y = X[:, :, None], Y[:, :, None]
    shape = (n, n, 1)
    rho = 1.0 + drho * np.sin(2 * np.pi * (X + Y))
    bx = amp * np.sin(2 * np.pi * Y) * np.ones_like(X)   # x-face (x_{i-1/2}, y_j)
    by = amp * np.cos(2 * np.pi * X) * np.ones_like(Y)   # y-face (x_i, y_{j-1/2})
    one = np.ones(shape)
    f = conserved(rho, [v[0] * one, v[1] * one, 0 * one], one, [bx, by, 0 * one], gamma,
                  (PERIODIC,) * 3)
    return Problem(f"passive2d_{n}", shape, (PERIODIC,) * 3, h, gamma, cfl, f, t_end=1.0)


def random_smooth(shape, seed: int = 0, bc=(PERIODIC,) * 3, gamma: float = 5.0 / 3.0,
                  cfl: float = 0.6, amp: float = 0.3, vamp: float = 0.5,
                  bmag: float = 0.8) -> Problem:
    """Seeded smooth state on an arbitrary (possibly ragged) grid: a few random Fourier
    modes per field.  Each face component of B depends only on the two transverse
    coordinates, so the discrete divergence is exactly zero."""
    rng = np.random.default_rng(seed)
    shape = tuple(int(s) for s in shape)
    h = 1.0 / max(shape)
    xs = [(_centres(m, h) / (m * h))[tuple(slice(None) if k == a else None for k in range(3))]
          for a, m in enumerate(shape)]

    def modes(dep, scale):
        out = np.zeros(shape)
        for _ in range(3):
            ph = rng.uniform(0, 2 * np.pi, 3)
            k = rng.integers(1, 3, 3)
            term = np.ones(shape)
            for a in dep:
                term = term * np.cos(2 * np.pi * k[a] * xs[a] + ph[a])
            out = out + rng.uniform(-1, 1) * term
        return scale * out

    rho = 1.0 + amp * np.tanh(modes((0, 1, 2), 1.0))
    p = 1.0 + amp * np.tanh(modes((0, 1, 2), 1.0))
    v = [modes((0, 1, 2), vamp) for _ in range(3)]
    b0 = rng.normal(size=3)
    b0 = 0.5 * bmag * b0 / np.linalg.norm(b0)
    B = [b0[a] + modes(tuple(k for k in range(3) if k != a), 0.5 * bmag) for a in range(3)]
    f = conserved(rho, v, p, B, gamma, bc)
    return Problem(f"random_{shape[0]}x{shape[1]}x{shape[2]}_s{seed}", shape, tuple(bc), h,
                   gamma, cfl, f)


# ------------------------------------------------------------------------------------
# Batched and served workloads
# ------------------------------------------------------------------------------------

def batched_instance(i: int, base_seed: int = 2009, lo: int = 48, hi: int = 192,
                     p0: float = 1.0, sigma: float = 0.1, cfl: float = 0.7) -> Problem:
    """Instance i of the batched workload: edges log-uniform in [lo, hi] per axis, rho = 1,
    p0 = 1, B direction uniform on the sphere, plasma beta log-uniform in [0.1, 10]
    (|B| = sqrt(2 p0 / beta)), Gaussian pressure pulse p = p0 (1 + A exp(-r^2/(2 sigma^2)))
    with A uniform in [1, 10], centred mid-box, periodic.  Seed = base_seed + i."""
    rng = np.random.default_rng(base_seed + i)
    n = tuple(int(round(math.exp(rng.uniform(math.log(lo), math.log(hi))))) for _ in range(3))
    d = rng.normal(size=3)
    d /= np.linalg.norm(d)
    beta = math.exp(rng.uniform(math.log(0.1), math.log(10.0)))
    bmag = math.sqrt(2.0 * p0 / beta)
    A = rng.uniform(1.0, 10.0)
    h = 1.0 / max(n)
    c = [_centres(m, h) for m in n]
    ctr = [0.5 * m * h for m in n]
    r2 = ((c[0] - ctr[0]) ** 2)[:, None, None] + ((c[1] - ctr[1]) ** 2)[None, :, None] \
        + ((c[2] - ctr[2]) ** 2)[None, None, :]
    p = p0 * (1.0 + A * np.exp(-r2 / (2.0 * sigma * sigma)))
    gamma = 5.0 / 3.0
    z = np.zeros(n)
    B = [np.full(n, bmag * d[a]) for a in range(3)]
    f = conserved(np.ones(n), [z, z, z], p, B, gamma, (PERIODIC,) * 3)
    return Problem(f"batch{i}_{n[0]}x{n[1]}x{n[2]}", n, (PERIODIC,) * 3, h, gamma, cfl, f)


def batched_shapes(count: int = 64, base_seed: int = 2009, lo: int = 48, hi: int = 192):
    """Grid shapes of the batched workload without building the fields."""
    out = []
    for i in range(count):
        rng = np.random.default_rng(base_seed + i)
        out.append(tuple(int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
                         for _ in range(3)))
    return out


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float      # seconds after the start of the trace
    kind: str           # "ot2d" or "blast3d"
    edge: int
    steps: int

    def problem(self) -> Problem:
        if self.kind == "ot2d":
            return orszag_tang(self.edge, "config")
        return blast3d(self.edge)

    @property
    def ncells(self) -> int:
        return self.edge * self.edge * (1 if self.kind == "ot2d" else self.edge)


def serving_trace(count: int, rate: float, seed: int = 7, ot_range=(128, 1024),
                  blast_range=(32, 256), steps_range=(50, 500), quantum: int = 16) -> list:
    """Poisson arrivals at ``rate`` per second: half Orszag-Tang 2D (square edge
    log-uniform in ot_range), half 3D blast (cubic edge log-uniform in blast_range), each
    running a step count uniform in steps_range.  Edges are rounded to multiples of
    ``quantum`` (so that requests share initial states).  The requests do not depend on
    the rate, only their arrival times do (rate 0 or inf: all arrive at time 0)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(count):
        gap = rng.standard_exponential()            # drawn for every rate: same requests
        t += gap / rate if 0 < rate < math.inf else 0.0
        if rng.uniform() < 0.5:
            kind, lo, hi = "ot2d", ot_range[0], ot_range[1]
        else:
            kind, lo, hi = "blast3d", blast_range[0], blast_range[1]
        edge = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        edge = max(quantum, int(round(edge / quantum)) * quantum)
        steps = int(rng.integers(steps_range[0], steps_range[1] + 1))
        out.append(Request(i, t, kind, edge, steps))
    return out
