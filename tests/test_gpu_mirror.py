"""Reflection equivariance of the CUDA sweeps, through the C ABI: a generic state reflected
about the face planes normal to one axis and advanced by whole steps equals the reflection
of the advanced state, bit for bit, in FP32 and FP64.

Ideal MHD is invariant under the reflection, and every operation of the sweeps is either
odd or even in the reflected quantities, with sums of mirrored neighbours taken in an
order that the reflection does not change (the (1,2,1) smoothing adds its outer
neighbours first).  A rounding that is not sign-symmetric, or a sum taken from one side,
shows up as a difference of an ulp or more.  With that property, the edge velocity of the
constrained transport on the mirror faces of a symmetric problem is exactly 0 in FP32 as
in FP64, so both take the upwind rule of Eq. "eq:first_flux" there (the symmetric blast
parity cases).  A generic state has no exact ties, so the rule is not exercised here.

Shapes: x/y constrained transport with shared EMF rows (nz >= 48) and per pencil, z
segments of 2 and 3 cells per lane, a ragged tail of the marching tiles along x, and a z
extent of 128 (TMA-staged x/y fluid sweeps)."""
import numpy as np
import pytest

from paper_0908_4362_gb300 import inputs as I
from pins import mirror_fields

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mhd():
    from paper_0908_4362_gb300 import build, mhd as m
    build.build()
    m.load_library()
    return m


SHAPES = [(24, 20, 56), (210, 6, 22), (12, 14, 40), (20, 6, 128)]


@pytest.mark.parametrize("shape", SHAPES, ids=["x".join(map(str, s)) for s in SHAPES])
@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_reflection_equivariance(mhd, shape, axis, prec):
    p = mhd.FP32 if prec == "fp32" else mhd.FP64
    # periodic along the mirror axis; one other axis outflow
    bc = tuple(0 if a == axis else (1 if a == (axis + 1) % 3 else 0) for a in range(3))
    prob = I.random_smooth(shape, seed=40 + axis, bc=bc)
    dtype = np.float32 if p == mhd.FP32 else np.float64
    f0 = prob.fields.astype(dtype)
    m0 = mirror_fields(f0, shape, axis)
    out = []
    for start in (f0, m0):
        with mhd.Solver(shape, bc, prob.h, prob.gamma, prob.cfl, prec=p) as s:
            s.upload([start[k] for k in range(8)])
            s.step(3, sync=True)
            got = np.empty((8, prob.ncells), dtype=dtype)
            s.download([got[k] for k in range(8)])
            out.append((got, s.state()[0]))
    (a, ta), (b, tb) = out
    assert ta == tb
    diff = np.abs(mirror_fields(a, shape, axis).astype(np.float64) - b).max()
    assert np.array_equal(mirror_fields(a, shape, axis), b), diff
