"""The batched persistent form (mhd_batch_*): many uneven grids advanced by one persistent
launch give, for every grid, the same bits as advancing it alone with mhd_step; and the
bounded device wait of the persistent kernel gives up with MHD_ERR_TIMEOUT."""
import numpy as np
import pytest

import oracle
from paper_0908_4362_gb300 import inputs as I
from parity import FP32_TOL, rel_l1

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mhd():
    from paper_0908_4362_gb300 import build, mhd as m
    build.build()
    m.load_library()
    return m


def _problems():
    # small uneven instances of the batched workload, one with mixed boundaries, one 2D,
    # and two whose x/y march blocks span several z rows or start inside a periodic z row
    probs = [I.batched_instance(i, lo=12, hi=40) for i in range(5)]
    probs.append(I.random_smooth((21, 9, 30), seed=21, bc=(1, 0, 1)))
    probs.append(I.orszag_tang(40, ny=28))
    probs.append(I.random_smooth((20, 18, 36), seed=22, bc=(0, 1, 0)))
    probs.append(I.random_smooth((6, 5, 132), seed=23))
    return probs


@pytest.mark.parametrize("nsteps", [3, 4])
def test_batch_matches_alone_bitwise(mhd, nsteps):
    probs = _problems()
    pre = [0, 1, 2, 0, 1, 2, 1, 2, 0]    # instances start at different axis-order phases
    alone = []
    for p, k in zip(probs, pre):
        with mhd.Solver.from_problem(p, prec=mhd.FP32) as s:
            s.step(k + 2 * nsteps, sync=True)
            alone.append(s.read())
    solvers = [mhd.Solver.from_problem(p, prec=mhd.FP32) for p in probs]
    for s, k in zip(solvers, pre):
        if k:
            s.step(k, sync=True)
    with mhd.Batch(solvers, z_tile_warps=16) as b:
        b.step(nsteps)
        b.step(nsteps)                    # a second launch (reused or rebuilt work list)
        assert b.sync() == mhd.MHD_OK
        ctas, items = b.info()
        assert ctas > 0 and items > 0
    for s, ref, k, p in zip(solvers, alone, pre, probs):
        got = s.read()
        t, _, stp, ph = s.state()
        assert stp == k + 2 * nsteps and ph == (k + 2 * nsteps) % 3
        assert np.array_equal(got, ref)
        s.close()
        # and the batched result against the FP64 oracle run from the same input (the
        # initial state rounded to FP32, as the FP32 context holds it), at the FP32
        # tolerance
        f32 = p.fields.astype(np.float32).astype(np.float64)
        o = oracle.Oracle(p.n, p.bc, p.h, p.gamma, p.cfl, f32)
        o.step(k + 2 * nsteps)
        assert abs(t - o.t) <= FP32_TOL * o.t
        err = rel_l1(got, o.f)
        assert np.all(err <= FP32_TOL), (p.name, err)


def test_batch_full_size_instances_vs_oracle(mhd):
    """Four instances of the batched workload at their own sizes (edges 48..192), 10 steps in
    one persistent launch, against the FP64 oracle at the FP32 tolerance."""
    probs = [I.batched_instance(i) for i in range(4)]
    solvers = [mhd.Solver.from_problem(p, prec=mhd.FP32) for p in probs]
    with mhd.Batch(solvers) as b:
        b.step(10)
        assert b.sync() == mhd.MHD_OK
    for s, p in zip(solvers, probs):
        got = s.read()
        s.close()
        o = oracle.Oracle.from_problem(p)
        o.step(10)
        err = rel_l1(got, o.f)
        assert np.all(err <= FP32_TOL), (p.name, err)


def test_batch_rejects_fp64_context(mhd):
    s = mhd.Solver.from_problem(I.random_smooth((8, 8, 8), seed=3), prec=mhd.FP64)
    with pytest.raises(mhd.MhdError):
        mhd.Batch([s])
    s.close()


def test_bounded_wait_times_out(mhd):
    lib = mhd.load_library()
    # ~10 ms of SM clock, then the wait gives up and reports it
    assert lib.mhd_batch_selftest_timeout(20_000_000) == mhd.MHD_ERR_TIMEOUT
    # the device is still usable afterwards
    with mhd.Solver.from_problem(I.random_smooth((10, 10, 10), seed=4), prec=mhd.FP32) as s:
        s.step(2, sync=True)


def test_batch_after_steps_alone(mhd):
    """Contexts stepped alone between batch launches (the single-grid steps run the middle
    CT pair in one launch, which swaps the B buffers; mhd_apply moves buffers too): the batch
    rebuilds their operations, and the result equals the same steps all taken alone."""
    probs = [I.batched_instance(i, lo=16, hi=40) for i in range(3)] + [I.blast3d(48)]
    alone = []
    for p in probs:
        with mhd.Solver.from_problem(p, prec=mhd.FP32) as s:
            s.step(3 + 4 + 2 + 3, sync=True)
            alone.append(s.read())
    solvers = [mhd.Solver.from_problem(p, prec=mhd.FP32) for p in probs]
    with mhd.Batch(solvers) as b:
        b.step(3)
        for s in solvers:
            s.step(4, sync=True)             # alone: buffers move
        b.step(2)
        assert b.sync() == mhd.MHD_OK
        for s in solvers:
            s.step(3, sync=True)
    for s, ref in zip(solvers, alone):
        assert s.state()[2] == 12
        assert np.array_equal(s.read(), ref)
        s.close()


def _shape_problems():
    # _problems() plus grids whose x or y extent spans several marching tiles of every
    # length (128, 192, 256) with a ragged last tile, with shared-row CT (z >= 48)
    return _problems() + [I.random_smooth((300, 20, 52), seed=24, bc=(0, 0, 1)),
                          I.random_smooth((16, 270, 48), seed=25, bc=(1, 0, 0)),
                          I.batched_instance(7, lo=40, hi=140)]


def _cycle(shapes, n):
    return [dict(shapes[i % len(shapes)]) for i in range(n)]


SHAPE_SETS = {
    "nt256_default": (256, [{}]),
    "len128_pencil_ct_k2": (128, [{"march_len": 128, "ct_march": 1, "seg_k": 2, "z_warps": 7}]),
    "len256_k3_w1": (256, [{"march_len": 256, "seg_k": 3, "z_warps": 1}]),
    "mixed_some_alone": (128, [{"march_len": 256}, {"alone": 1}, {"ct_march": 1, "seg_k": 3},
                               {"march_len": 128, "z_warps": 64}, {"alone": 1, "march_len": 128}]),
}


@pytest.mark.parametrize("name", list(SHAPE_SETS))
def test_batch_shapes_bitwise(mhd, name):
    """Every launch shape (threads per CTA, marching tile length, CT form, z segment length
    and items, the route through the single-grid kernels) gives the same bits as mhd_step."""
    nt, shapes = SHAPE_SETS[name]
    probs = _shape_problems()
    pre = [i % 3 for i in range(len(probs))]
    nsteps = 4
    alone = []
    for p, k in zip(probs, pre):
        with mhd.Solver.from_problem(p, prec=mhd.FP32) as s:
            s.step(k + 2 * nsteps, sync=True)
            alone.append(s.read())
    solvers = [mhd.Solver.from_problem(p, prec=mhd.FP32) for p in probs]
    for s, k in zip(solvers, pre):
        if k:
            s.step(k, sync=True)
    with mhd.Batch(solvers) as b:
        b.configure(threads_per_cta=nt, shapes=_cycle(shapes, len(probs)))
        b.step(nsteps)
        b.step(nsteps)
        assert b.sync() == mhd.MHD_OK
    for s, ref, k, p in zip(solvers, alone, pre, probs):
        assert s.state()[2] == k + 2 * nsteps
        assert np.array_equal(s.read(), ref), p.name
        s.close()


def test_batch_configure_rejects_bad_values(mhd):
    s = mhd.Solver.from_problem(I.random_smooth((8, 8, 8), seed=5), prec=mhd.FP32)
    with mhd.Batch([s]) as b:
        for kw in ({"threads_per_cta": 64}, {"ctas_per_sm": -1}, {"spin_cycles": -1},
                   {"shapes": [{"march_len": 100}]}, {"shapes": [{"seg_k": 4}]},
                   {"shapes": [{"ct_march": 2}]}, {"shapes": [{"alone": 3}]},
                   {"shapes": [{"z_warps": -2}]}):
            with pytest.raises(mhd.MhdError):
                b.configure(**kw)
        b.configure(threads_per_cta=256, shapes=[{"march_len": 256}])
        b.step(2)
        assert b.sync() == mhd.MHD_OK
    s.close()


def test_batch_timeout_marks_contexts(mhd):
    """A persistent launch whose waits give up (a bound of one SM cycle: the first item
    that finds its operation's predecessor unfinished gives up) reports MHD_ERR_TIMEOUT, and
    every context of the launch reports it from then on, until it is initialised again."""
    probs = [I.batched_instance(i, lo=24, hi=48) for i in range(4)]
    solvers = [mhd.Solver.from_problem(p, prec=mhd.FP32) for p in probs]
    with mhd.Batch(solvers) as b:
        b.configure(spin_cycles=1)
        b.step(2)
        assert b.sync() == mhd.MHD_ERR_TIMEOUT
        for s in solvers:
            with pytest.raises(mhd.MhdError) as ei:
                s.read()
            assert ei.value.status == mhd.MHD_ERR_TIMEOUT
        b.configure()                         # the default bound again
        for s, p in zip(solvers, probs):
            s.init_fields(p.fields)
        b.step(2)
        assert b.sync() == mhd.MHD_OK
    for s, p in zip(solvers, probs):
        with mhd.Solver.from_problem(p, prec=mhd.FP32) as r:
            r.step(2, sync=True)
            assert np.array_equal(s.read(), r.read())
        s.close()
