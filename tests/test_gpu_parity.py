"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, element by element on
the same seeded inputs.

Error measure: relative L1 per field, sum|gpu - oracle| / sum|oracle|, where the three
components of a vector (momentum, B) share the denominator of the whole vector,
sum over components of |oracle|; a component that starts at zero (B_z of a blast in the
x-y plane, m_n of a transverse wave) is thus measured against the size of its vector.
Tolerances: FP64 <= 1e-12 and FP32 <= 2e-5 after 10 steps; one sweep operator 1e-13 (FP64)
and 2e-6 (FP32).  The FP64 kernels are built without FMA contraction and follow the
oracle's operation order, so FP64 is in fact compared bit for bit as well."""
import numpy as np
import pytest

import oracle
from paper_0908_4362_gb300 import inputs as I
from parity import FP32_TOL, FP64_TOL, rel_l1

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mhd():
    import torch
    assert torch.cuda.is_available()
    from paper_0908_4362_gb300 import build, mhd as m
    build.build()
    m.load_library()
    return m


def run_both(mhd, prob, steps, prec):
    ref = oracle.Oracle.from_problem(prob)
    ref.step(steps)
    with mhd.Solver.from_problem(prob, prec=prec) as s:
        done = s.step(steps, sync=True)
        got = s.read()
        t, _, nst, ph = s.state()
    assert done == steps and nst == steps and ph == ref.phase
    assert abs(t - ref.t) <= (1e-13 if prec == mhd.FP64 else 2e-5) * max(1.0, abs(ref.t))
    return got, ref


# shapes chosen to exercise every kernel path: z extent a multiple of 4 (vector march
# along z in FP32 and FP64), of 2 only (vector march in FP64, tile kernel in FP32), odd
# (tile kernel), tiles longer than one march segment (> 64 cells) with a ragged tail,
# outflow on the vector axis, degenerate axes
OP_CASES = [
    ("periodic_ragged", lambda: I.random_smooth((37, 29, 23), seed=3)),
    ("mixed_bc", lambda: I.random_smooth((21, 40, 17), seed=4, bc=(1, 0, 1))),
    ("thin", lambda: I.random_smooth((70, 3, 1), seed=5, bc=(1, 1, 0))),
    ("zvec_outflow", lambda: I.random_smooth((13, 11, 72), seed=6, bc=(0, 1, 1))),
    ("zvec2_long", lambda: I.random_smooth((131, 6, 10), seed=15, bc=(1, 0, 0))),
    ("long_y", lambda: I.random_smooth((5, 150, 8), seed=16, bc=(0, 1, 1))),
    # x/y march blocks of 128 pencils spanning several z rows (nz = 36), and blocks that
    # start inside a periodic z row and end on its last pencil (nz = 132), with outflow
    # across the other transverse axis
    ("rows_per_block", lambda: I.random_smooth((9, 37, 36), seed=18)),
    ("block_wraps_z", lambda: I.random_smooth((6, 5, 132), seed=19, bc=(1, 1, 0))),
    # z extents that are multiples of 128 (the TMA-staged x/y fluid sweeps), periodic and
    # outflow along the sweeps, the tile along x shorter and longer than one march tile
    ("tma_periodic", lambda: I.random_smooth((37, 5, 128), seed=24)),
    ("tma_outflow", lambda: I.random_smooth((200, 3, 256), seed=25, bc=(1, 1, 1))),
]


@pytest.mark.parametrize("case", OP_CASES, ids=[c[0] for c in OP_CASES])
@pytest.mark.parametrize("op", [0, 1], ids=["fluid", "ct"])
@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_single_operator(mhd, case, op, axis, prec):
    prob = case[1]()
    p = mhd.FP64 if prec == "fp64" else mhd.FP32
    ref = oracle.Oracle.from_problem(prob)
    dt = 0.5 * ref.dt()
    (ref.fluid if op == 0 else ref.ct)(axis, dt)
    with mhd.Solver.from_problem(prob, prec=p) as s:
        s.apply(op, axis, dt)
        got = s.read()
    err = rel_l1(got, ref.f)
    tol = 1e-13 if p == mhd.FP64 else 2e-6
    assert np.all(err <= tol), err


STEP_CASES = [
    ("brio_wu_512", lambda: I.brio_wu(512)),
    ("brio_wu_y", lambda: I.brio_wu(256, axis=1)),
    ("orszag_tang_64", lambda: I.orszag_tang(64)),
    ("orszag_tang_ragged", lambda: I.orszag_tang(45, ny=37)),
    ("random3d_ragged", lambda: I.random_smooth((19, 23, 17), seed=7)),
    ("random3d_outflow", lambda: I.random_smooth((33, 18, 26), seed=8, bc=(1, 0, 1))),
    ("blast_40", lambda: I.blast3d(40)),
    ("degenerate_z", lambda: I.random_smooth((1, 1, 130), seed=9)),
    ("single_cell", lambda: I.random_smooth((1, 1, 1), seed=10)),
    ("batched_instance", lambda: I.batched_instance(3)),
    ("zvec_outflow", lambda: I.random_smooth((13, 11, 72), seed=6, bc=(0, 1, 1))),
    ("long_mixed", lambda: I.random_smooth((131, 9, 68), seed=17, bc=(1, 0, 1))),
    ("tma_mixed", lambda: I.random_smooth((21, 13, 128), seed=26, bc=(0, 1, 0))),
    ("dai_woodward_256", lambda: I.dai_woodward(256)),
    ("blast2d_64", lambda: I.blast2d(64)),
    ("rotor1_64", lambda: I.rotor(64, 1)),
    ("rotor2_64", lambda: I.rotor(64, 2)),
]


# Mirror-symmetric problems (the blast, both rotors) put exact ties of the constrained
# transport's edge velocity on their symmetry planes.  The (1,2,1) smoothing is evaluated so
# that it is exactly odd under the reflection, in every precision, so the edge velocity
# there is exactly 0 in FP32 as in the FP64 oracle and both take the printed upwind rule
# (Eq. "eq:first_flux"); the FP32 comparison runs on the symmetric problems themselves.
@pytest.mark.parametrize("case", STEP_CASES, ids=[c[0] for c in STEP_CASES])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_ten_steps(mhd, case, prec):
    p = mhd.FP64 if prec == "fp64" else mhd.FP32
    prob = case[1]()
    steps = 10 if prob.ncells < 2_000_000 else 3
    got, ref = run_both(mhd, prob, steps, p)
    err = rel_l1(got, ref.f)
    assert np.all(err <= (FP64_TOL if p == mhd.FP64 else FP32_TOL)), err


BITWISE_CASES = ["blast_40", "random3d_outflow", "orszag_tang_ragged", "brio_wu_512",
                 "batched_instance", "zvec_outflow", "long_mixed", "blast2d_64", "rotor1_64",
                 "dai_woodward_256"]


@pytest.mark.parametrize("name", BITWISE_CASES)
def test_fp64_bit_identical(mhd, name):
    """FP64 without FMA contraction reproduces the oracle bit for bit, including the exact
    upwind ties (edge velocity 0) of mirror-symmetric problems."""
    prob = dict(STEP_CASES)[name]()
    got, ref = run_both(mhd, prob, 10, mhd.FP64)
    assert np.array_equal(got, ref.f), np.abs(got - ref.f).max()


@pytest.mark.parametrize("b_dir", [(1.0, 1.0, 0.0), (1.0, 1.0, 1.0)], ids=["b110", "b111"])
def test_fp32_symmetric_blast(mhd, b_dir):
    """The blast centred on the grid's mirror planes, as benchmarked (B along (1,1,0)) and
    as in the paper's 3D run (B along (1,1,1)), 64^3 so that its radius spans 6.4 cells:
    FP32 within the FP32 tolerance of the FP64 oracle after 10 steps, mirror-plane ties
    included."""
    prob = I.blast3d(64, b_dir=b_dir)
    got, ref = run_both(mhd, prob, 10, mhd.FP32)
    err = rel_l1(got, ref.f)
    assert np.all(err <= FP32_TOL), err


SP_DP_CASES = [("rotor1_128", lambda: I.rotor(128, 1)), ("rotor2_128", lambda: I.rotor(128, 2)),
               ("orszag_tang_128", lambda: I.orszag_tang(128)),
               ("blast2d_128", lambda: I.blast2d(128))]


@pytest.mark.parametrize("case", SP_DP_CASES, ids=[c[0] for c in SP_DP_CASES])
def test_sp_dp_difference_at_final_time(mhd, case):
    """FP32 against FP64 on the GPU at the paper's final times (the paper reports the
    single/double precision differences of its own runs, Sect. 6): both reach t_end, and
    every field's rel-L1 difference stays small after hundreds of steps with shocks."""
    prob = case[1]()
    out = {}
    for p in (mhd.FP64, mhd.FP32):
        with mhd.Solver.from_problem(prob, prec=p) as s:
            n = s.run_to(prob.t_end)
            t, _, _, _ = s.state()
            out[p] = (n, t, s.read())
    (n64, t64, f64), (n32, t32, f32) = out[mhd.FP64], out[mhd.FP32]
    assert t64 == prob.t_end and t32 == prob.t_end
    assert abs(n64 - n32) <= max(2, n64 // 100)
    err = rel_l1(f32, f64)
    assert np.all(err <= 1e-2), err


def test_brio_wu_to_final_time_fp64(mhd):
    """Brio-Wu (config: 512 cells, gamma 2, CFL 0.8, outflow) run to t = 0.1 with the last
    dt clipped: same step count, same final time, same profile."""
    prob = I.brio_wu(512)
    ref = oracle.Oracle.from_problem(prob)
    nref = ref.run_to(0.1)
    with mhd.Solver.from_problem(prob, prec=mhd.FP64) as s:
        n = s.run_to(0.1)
        got = s.read()
        t, _, _, _ = s.state()
    assert n == nref and t == 0.1
    err = rel_l1(got, ref.f)
    assert np.all(err <= 1e-12), err


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_smooth_final_time(mhd, prec):
    """Smooth problems at their final time: the Alfven wave after a full period."""
    prob = I.alfven_circular(64, axis=2, cfl=0.4)
    p = mhd.FP64 if prec == "fp64" else mhd.FP32
    ref = oracle.Oracle.from_problem(prob)
    nref = ref.run_to(prob.t_end)
    with mhd.Solver.from_problem(prob, prec=p) as s:
        n = s.run_to(prob.t_end)
        got = s.read()
    assert n == nref
    err = rel_l1(got, ref.f)
    assert np.all(err <= (1e-11 if p == mhd.FP64 else 2e-5)), err


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_cmax_matches(mhd, prec):
    prob = I.random_smooth((24, 17, 30), seed=12)
    p = mhd.FP64 if prec == "fp64" else mhd.FP32
    ref = oracle.Oracle.from_problem(prob).cmax()
    with mhd.Solver.from_problem(prob, prec=p) as s:
        got = s.cmax()
    assert abs(got - ref) <= (1e-14 if p == mhd.FP64 else 2e-6) * ref


def test_conservation_and_divb_on_gpu(mhd):
    prob = I.random_smooth((40, 36, 44), seed=13)
    with mhd.Solver.from_problem(prob, prec=mhd.FP64) as s:
        s0 = s.sums()
        s.step(10, sync=True)
        s1 = s.sums()
        f = s.read()
    scale = np.abs(prob.fields).sum(axis=1)
    assert np.all(np.abs(s1 - s0) / scale <= 1e-13)
    ref = oracle.Oracle(prob.n, prob.bc, prob.h, prob.gamma, prob.cfl, f)
    assert ref.divb_max() * prob.h / np.abs(f[5:]).max() <= 1e-13


def test_determinism_and_checkpoint(mhd):
    """Two runs give identical bits, and n steps + checkpoint + restore + n steps equals
    2n steps."""
    prob = I.blast3d(32)
    with mhd.Solver.from_problem(prob, prec=mhd.FP32) as s:
        s.step(8, sync=True)
        a = s.read()
    with mhd.Solver.from_problem(prob, prec=mhd.FP32) as s:
        s.step(4, sync=True)
        mid = s.read()
        t, _, stp, ph = s.state()
    with mhd.Solver(prob.n, prob.bc, prob.h, prob.gamma, prob.cfl, prec=mhd.FP32) as s:
        s.init_fields(mid)
        s.set_state(t, stp, ph)
        s.step(4, sync=True)
        b = s.read()
        assert s.state()[2] == 8
    with mhd.Solver.from_problem(prob, prec=mhd.FP32) as s:
        s.step(8, sync=True)
        c = s.read()
    assert np.array_equal(a, c)
    assert np.array_equal(a, b)


def test_pressure_modes_low_beta(mhd):
    """The FP32 sweeps with each pressure recovery (plain FP32, FP64, compensated FP32) on
    the lowest-beta instance of the batched workload (beta = 0.126): all within the FP32
    tolerance of the FP64 oracle run from the same (FP32) input after 10 steps; the FP64 and
    compensated recoveries give nearly the same state, and not plain FP32's."""
    prob = I.batched_instance(52)
    f32 = prob.fields.astype(np.float32)
    ref = oracle.Oracle(prob.n, prob.bc, prob.h, prob.gamma, prob.cfl, f32.astype(np.float64))
    ref.step(10)
    got, errs = {}, {}
    for pm in (mhd.PRESSURE_FP32, mhd.PRESSURE_FP64, mhd.PRESSURE_COMPENSATED):
        with mhd.Solver(prob.n, prob.bc, prob.h, prob.gamma, prob.cfl, prec=mhd.FP32,
                        pressure=pm) as s:
            s.upload([f32[k] for k in range(8)])
            s.step(10, sync=True)
            got[pm] = s.read()
        errs[pm] = rel_l1(got[pm], ref.f)
        assert np.all(errs[pm] <= FP32_TOL), (pm, errs[pm])
    d_comp = rel_l1(got[mhd.PRESSURE_COMPENSATED], got[mhd.PRESSURE_FP64]).max()
    d_plain = rel_l1(got[mhd.PRESSURE_FP32], got[mhd.PRESSURE_FP64]).max()
    assert not np.array_equal(got[mhd.PRESSURE_FP32], got[mhd.PRESSURE_FP64])
    assert d_comp <= 0.25 * d_plain, (d_comp, d_plain)


def hypersonic_state(shape, axis, seed=5, gamma=5.0 / 3.0):
    """A hypersonic, unmagnetised FP32 state, constant along `axis` and random across it,
    whose thermal energy is a few FP32 ulps of its total energy: per pencil |v| in [50, 100],
    rho in [0.5, 2], B = 0, and E the first FP32 value above the kinetic energy of the
    stored rho and m.  The exact pressure of the stored values is then positive and below
    4e-8 of E.  Returns the (8, N) FP32 fields and that pressure per cell."""
    rng = np.random.default_rng(seed)
    cross = list(shape)
    cross[axis] = 1
    M = int(np.prod(cross))
    rho = rng.uniform(0.5, 2.0, M).astype(np.float32)
    d = rng.normal(size=(3, M))
    d /= np.linalg.norm(d, axis=0)
    m = (rho.astype(np.float64) * rng.uniform(50, 100, M) * d).astype(np.float32)
    ke = 0.5 * (m.astype(np.float64) ** 2).sum(axis=0) / rho.astype(np.float64)
    E = ke.astype(np.float32)
    E = np.where(E.astype(np.float64) > ke, E, np.nextafter(E, np.float32(np.inf)))
    f = np.zeros((8,) + tuple(cross), dtype=np.float32)
    f[0], f[1:4], f[4] = rho.reshape(cross), m.reshape((3,) + tuple(cross)), E.reshape(cross)
    f = np.ascontiguousarray(np.broadcast_to(f, (8,) + tuple(shape)).reshape(8, -1))
    p_exact = (gamma - 1.0) * (f[4].astype(np.float64) - 0.5 * (f[1:4].astype(np.float64) ** 2)
                               .sum(axis=0) / f[0].astype(np.float64))
    assert p_exact.min() > 0
    return f, p_exact


def test_pressure_recovery_hypersonic(mhd):
    """Where the pressure is below an ulp of E (kinetic energy ~1e8 times the thermal one),
    plain FP32 recovery cancels to the wrong sign in some pencils (a negative sound-speed
    radicand: MHD_ERR_UNPHYSICAL), while the FP64 and the compensated FP32 recoveries get the
    exact pressure of the stored values.  The state is constant along the sweep axis, so a
    fluid sweep must return it unchanged, bit for bit (the oracle does), and the CFL speed
    must be that of the exact pressure."""
    shape, h, gamma, dt = (24, 10, 12), 1.0 / 24, 5.0 / 3.0, 1e-6
    for axis in range(3):
        f, p_exact = hypersonic_state(shape, axis, seed=5 + axis)
        f64 = f.astype(np.float64)
        v = f64[1:4] / f64[0]
        cs = np.sqrt(gamma * p_exact / f64[0])
        cmax_exact = (np.abs(v).max(axis=0) + cs).max()
        ref = oracle.Oracle(shape, (0, 0, 0), h, gamma, 0.5, f64)
        ref.fluid(axis, dt)
        assert ref.status == 0 and np.array_equal(ref.f, f64)
        res, st, cm = {}, {}, {}
        for pm in (mhd.PRESSURE_FP32, mhd.PRESSURE_FP64, mhd.PRESSURE_COMPENSATED):
            with mhd.Solver(shape, (0, 0, 0), h, gamma, 0.5, prec=mhd.FP32, pressure=pm) as s:
                st_up = s.lib.mhd_upload(s.ctx, mhd._ptrs8([f[k].ctypes.data for k in range(8)]),
                                         0, 0, 0.0)
                s.apply(0, axis, dt)
                st[pm] = (st_up, s.sync(check=False))
                out = np.empty_like(f)
                s.download([out[k] for k in range(8)], check=False)
                res[pm] = out
                if pm != mhd.PRESSURE_FP32:
                    cm[pm] = s.cmax()
        assert st[mhd.PRESSURE_FP32][1] == mhd.MHD_ERR_UNPHYSICAL, st
        for pm in (mhd.PRESSURE_FP64, mhd.PRESSURE_COMPENSATED):
            assert st[pm] == (mhd.MHD_OK, mhd.MHD_OK), (axis, pm, st[pm])
            assert np.array_equal(res[pm], f), (axis, pm)
            assert abs(cm[pm] - cmax_exact) <= 1e-6 * cmax_exact, (axis, pm, cm[pm], cmax_exact)


def test_fp32_sums_exact_widening(mhd):
    """The FP64 sums of an FP32 state widen every value exactly (zeros of both signs,
    subnormals, magnitudes over many decades): within FP64 accumulation error of the exact
    sum of the stored values."""
    import math
    n = (16, 12, 20)
    N = n[0] * n[1] * n[2]
    rng = np.random.default_rng(31)
    f = np.zeros((8, N), dtype=np.float32)
    f[0] = 10.0 ** rng.uniform(-3, 3, N)
    special = np.array([0.0, -0.0, 1e-40, -3e-42, 1e-20, -7.5, 2.0 ** -126], dtype=np.float32)
    for k in (1, 2, 3, 5, 6, 7):
        v = (rng.standard_normal(N) * 10.0 ** rng.uniform(-8, 1, N)).astype(np.float32)
        pick = rng.random(N) < 0.3
        v[pick] = special[rng.integers(0, len(special), pick.sum())]
        f[k] = v
    m2 = (f[1:4].astype(np.float64) ** 2).sum(0)
    b2 = (f[5:8].astype(np.float64) ** 2).sum(0)
    f[4] = (0.5 * m2 / f[0] + 0.5 * b2 + 10.0 ** rng.uniform(-2, 2, N)).astype(np.float32)
    with mhd.Solver(n, (0, 0, 0), 1.0 / 20, 5.0 / 3.0, 0.7, prec=mhd.FP32) as s:
        s.upload([f[k] for k in range(8)])
        got = s.sums()
    for k in range(8):
        vals = f[k].astype(np.float64)
        exact = math.fsum(vals.tolist())
        assert abs(got[k] - exact) <= 1e-12 * np.abs(vals).sum() + 1e-300, (k, got[k], exact)


def test_unphysical_state_reported(mhd):
    prob = I.random_smooth((8, 8, 8), seed=14)
    f = prob.fields.copy()
    f[0, 5] = -1.0
    s = mhd.Solver(prob.n, prob.bc, prob.h, prob.gamma, prob.cfl, prec=mhd.FP64)
    st = s.init_fields(f, check=False)
    assert st == mhd.MHD_ERR_UNPHYSICAL
    s.close()


def test_invalid_config_rejected(mhd):
    with pytest.raises(mhd.MhdError):
        mhd.Solver((0, 4, 4))
    with pytest.raises(mhd.MhdError):
        mhd.Solver((4, 4, 4), cfl=1.5)


PAIR_CASES = [("periodic_k3", lambda: I.random_smooth((9, 7, 200), seed=31)),
              ("outflow_k3", lambda: I.random_smooth((6, 8, 130), seed=32, bc=(1, 1, 1))),
              ("mixed_k2", lambda: I.random_smooth((10, 9, 40), seed=33, bc=(0, 1, 0))),
              ("short_z", lambda: I.random_smooth((5, 6, 12), seed=34, bc=(1, 0, 1))),
              ("blast", lambda: I.blast3d(48))]


# x/y cases: the shared-row CT form (nz >= 48, 4+ rows across) with a periodic sweep axis
# runs the pair in one launch; outflow along the sweep falls back to two launches
PAIR_CASES_XY = [("rows_periodic", lambda: I.random_smooth((230, 9, 60), seed=35)),
                 ("rows_mixed", lambda: I.random_smooth((40, 30, 52), seed=36, bc=(0, 0, 1))),
                 ("rows_outflow_t", lambda: I.random_smooth((50, 7, 96), seed=37, bc=(0, 1, 1))),
                 ("outflow_sweep", lambda: I.random_smooth((30, 20, 64), seed=38, bc=(1, 1, 0))),
                 ("blast", lambda: I.blast3d(48))]


@pytest.mark.parametrize("case", PAIR_CASES, ids=[c[0] for c in PAIR_CASES])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_ct_z_pair_in_one_launch(mhd, case, prec):
    """The two CT_z operators that meet in the middle of a step, in one launch (op 2): the
    same bits as two single CT_z launches, and the oracle's two CT_z within tolerance."""
    _pair_case(mhd, case[1](), 2, prec)


@pytest.mark.parametrize("case", PAIR_CASES_XY, ids=[c[0] for c in PAIR_CASES_XY])
@pytest.mark.parametrize("axis", [0, 1])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_ct_xy_pair_in_one_launch(mhd, case, axis, prec):
    """The same for the x and y CT pairs (the shared-row two-pass march)."""
    _pair_case(mhd, case[1](), axis, prec)


def _pair_case(mhd, prob, axis, prec):
    p = mhd.FP64 if prec == "fp64" else mhd.FP32
    ref = oracle.Oracle.from_problem(prob)
    dt = 0.5 * ref.dt()
    ref.ct(axis, dt)
    ref.ct(axis, dt)
    got = []
    for ops in ((1, 1), (2,)):
        with mhd.Solver.from_problem(prob, prec=p) as s:
            for op in ops:
                s.apply(op, axis, dt)
            got.append(s.read())
    assert np.array_equal(got[0], got[1]), np.abs(got[0] - got[1]).max()
    err = rel_l1(got[1], ref.f)
    assert np.all(err <= (1e-13 if p == mhd.FP64 else 4e-6)), err


CTZ_FORM_CASES = ([c for c in OP_CASES if c[0] != "thin"] + [c for c in PAIR_CASES] +
                  [("rows_blocks_mixed", lambda: I.random_smooth((70, 47, 97), seed=41, bc=(1, 0, 1))),
                   ("rows_blocks_periodic", lambda: I.random_smooth((64, 31, 180), seed=42))])


@pytest.mark.parametrize("case", CTZ_FORM_CASES, ids=[c[0] for c in CTZ_FORM_CASES])
@pytest.mark.parametrize("op", [1, 2], ids=["ct", "pair"])
def test_ct_z_rows_same_bits_as_segments(mhd, monkeypatch, case, op):
    """FP32 CT along z: the marching shared-row kernel (each warp runs its own EMF pipelines,
    the upper rows' EMFs come from the next row of the march and the neighbouring warp)
    gives the same bits as the warp segments that run all four pipelines per pencil
    (MHD_CTZ_SEG=1 selects those), one pass and the middle pair, over periodic, outflow
    and mixed boundaries, ragged shapes, several row groups along x and y, and windows
    of 2 and 3 cells per lane."""
    prob = case[1]()
    dt = 0.5 * oracle.Oracle.from_problem(prob).dt()
    got = []
    for seg in ("1", "0"):
        monkeypatch.setenv("MHD_CTZ_SEG", seg)
        with mhd.Solver.from_problem(prob, prec=mhd.FP32) as s:
            s.apply(op, 2, dt)
            got.append(s.read())
    monkeypatch.delenv("MHD_CTZ_SEG")
    assert np.array_equal(got[0], got[1]), np.abs(got[0] - got[1]).max()


@pytest.mark.parametrize("case", CTZ_FORM_CASES, ids=[c[0] for c in CTZ_FORM_CASES])
def test_reverse_lz_in_one_launch(mhd, case):
    """The reverse z operator L_z (CT along z, then the fluid sweep along z) in one launch
    (mhd_apply op 3, FP32): the same bits as the two launches (op 1, then op 0), over the
    shapes and boundaries of the CT form test, and within tolerance of the oracle's CT_z then
    fluid_z."""
    prob = case[1]()
    ref = oracle.Oracle.from_problem(prob)
    dt = 0.5 * ref.dt()
    ref.ct(2, dt)
    ref.fluid(2, dt)
    got = []
    for ops in ((1, 0), (3,)):
        with mhd.Solver.from_problem(prob, prec=mhd.FP32) as s:
            for op in ops:
                s.apply(op, 2, dt)
            got.append(s.read())
    assert np.array_equal(got[0], got[1]), np.abs(got[0] - got[1]).max()
    err = rel_l1(got[1], ref.f)
    assert np.all(err <= 4e-6), err


def test_reverse_lz_one_launch_rejected_where_absent(mhd):
    """op 3 exists for FP32 contexts with plain FP32 pressure recovery only: FP64 contexts
    and the other pressure modes get MHD_ERR_INVALID, and their state is left as it was."""
    prob = I.random_smooth((6, 5, 40), seed=43)
    for kw in ({"prec": mhd.FP64}, {"prec": mhd.FP32, "pressure": mhd.PRESSURE_FP64}):
        with mhd.Solver.from_problem(prob, **kw) as s:
            before = s.read()
            with pytest.raises(mhd.MhdError) as e:
                s.apply(3, 2, 1e-3)
            assert e.value.status == mhd.MHD_ERR_INVALID
            assert np.array_equal(s.read(), before)
