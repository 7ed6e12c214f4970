"""Exact solution of the Riemann problem of 1D gas dynamics (B = 0), written from the
textbook method (two-wave pressure function, Newton iteration for p*, self-similar
sampling of shocks and rarefaction fans).  Used to pin the oracle's fluid update: with
B = 0 the MHD fluid sweep must converge to this solution."""
from __future__ import annotations

import numpy as np


def _fk(p, rho, pk, a, g):
    """Pressure function of one side and its derivative."""
    if p > pk:
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        q = np.sqrt(A / (p + B))
        return (p - pk) * q, q * (1.0 - 0.5 * (p - pk) / (p + B))
    r = p / pk
    f = 2.0 * a / (g - 1.0) * (r ** ((g - 1.0) / (2.0 * g)) - 1.0)
    df = 1.0 / (rho * a) * r ** (-(g + 1.0) / (2.0 * g))
    return f, df


def star_state(left, right, g):
    rl, ul, pl = left
    rr, ur, pr = right
    al, ar = np.sqrt(g * pl / rl), np.sqrt(g * pr / rr)
    # two-rarefaction initial guess
    z = (g - 1.0) / (2.0 * g)
    p = ((al + ar - 0.5 * (g - 1.0) * (ur - ul)) / (al / pl ** z + ar / pr ** z)) ** (1.0 / z)
    for _ in range(100):
        fl, dfl = _fk(p, rl, pl, al, g)
        fr, dfr = _fk(p, rr, pr, ar, g)
        dp = (fl + fr + ur - ul) / (dfl + dfr)
        pn = max(p - dp, 1e-12)
        if abs(pn - p) < 1e-15 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _fk(p, rl, pl, al, g)
    fr, _ = _fk(p, rr, pr, ar, g)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def sample(left, right, g, x, t, x0=0.5):
    """Primitive (rho, u, p) at positions x and time t > 0."""
    rl, ul, pl = left
    rr, ur, pr = right
    al, ar = np.sqrt(g * pl / rl), np.sqrt(g * pr / rr)
    ps, us = star_state(left, right, g)
    gm, gp = (g - 1.0) / (g + 1.0), g + 1.0
    out = np.empty((3, x.size))
    for k, xi in enumerate(x):
        s = (xi - x0) / t
        if s <= us:
            if ps > pl:
                sl = ul - al * np.sqrt(gp / (2 * g) * ps / pl + (g - 1) / (2 * g))
                if s <= sl:
                    w = (rl, ul, pl)
                else:
                    w = (rl * (ps / pl + gm) / (gm * ps / pl + 1.0), us, ps)
            else:
                shl = ul - al
                asl = al * (ps / pl) ** ((g - 1) / (2 * g))
                stl = us - asl
                if s <= shl:
                    w = (rl, ul, pl)
                elif s <= stl:
                    c = 2.0 / gp + (g - 1) / (gp * al) * (ul - s)
                    w = (rl * c ** (2 / (g - 1)), 2 / gp * (al + 0.5 * (g - 1) * ul + s),
                         pl * c ** (2 * g / (g - 1)))
                else:
                    w = (rl * (ps / pl) ** (1.0 / g), us, ps)
        else:
            if ps > pr:
                sr = ur + ar * np.sqrt(gp / (2 * g) * ps / pr + (g - 1) / (2 * g))
                if s >= sr:
                    w = (rr, ur, pr)
                else:
                    w = (rr * (ps / pr + gm) / (gm * ps / pr + 1.0), us, ps)
            else:
                shr = ur + ar
                asr = ar * (ps / pr) ** ((g - 1) / (2 * g))
                str_ = us + asr
                if s >= shr:
                    w = (rr, ur, pr)
                elif s >= str_:
                    c = 2.0 / gp - (g - 1) / (gp * ar) * (ur - s)
                    w = (rr * c ** (2 / (g - 1)), 2 / gp * (-ar + 0.5 * (g - 1) * ur + s),
                         pr * c ** (2 * g / (g - 1)))
                else:
                    w = (rr * (ps / pr) ** (1.0 / g), us, ps)
        out[:, k] = w
    return out
