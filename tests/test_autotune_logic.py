"""Host logic of the batched form's autotuner (no GPU): shape classes, the coordinate
descent over the batch-wide and per-class knobs, the 1% acceptance threshold, the route
knob's size rule, and the cache.  The solvers and the batch are fakes whose step time is a
function of the configured shapes."""
import pytest

from paper_0908_4362_gb300 import autotune, mhd


class FakeProblem:
    def __init__(self, n):
        self.n = tuple(n)
        self.ncells = n[0] * n[1] * n[2]


def test_shape_class_octave_pairs():
    assert autotune.shape_class((48, 48, 48)) == "2^15-2^17"        # 110,592 cells
    assert autotune.shape_class((64, 64, 64)) == "2^17-2^19"        # 2^18
    assert autotune.shape_class((128, 128, 128)) == "2^21-2^23"     # 2^21
    assert autotune.shape_class((256, 256, 256)) == "2^23-2^25"     # 2^24
    assert autotune.shape_class((1, 1, 1)) == "2^1-2^3"


def test_instance_shapes_by_class():
    probs = [FakeProblem((64, 64, 64)), FakeProblem((256, 256, 256)), FakeProblem((60, 70, 64))]
    classes = {"2^23-2^25": {"alone": 1}, "2^17-2^19": {"ct_march": 1}}
    assert autotune.instance_shapes(probs, classes) == [{"ct_march": 1}, {"alone": 1},
                                                         {"ct_march": 1}]


@pytest.fixture
def fake_gpu(monkeypatch, tmp_path):
    """Fake Solver/Batch: a batch step costs the sum over instances of a per-instance cost
    that depends on the instance's shape dict and the threads per CTA."""
    state = {"configs": []}

    def cost(prob, shape, nt):
        big = prob.ncells >= 1 << 21
        c = prob.ncells * 1e-9
        if big and shape.get("alone"):
            c *= 0.5                       # large grids: the single-grid route halves the cost
        if not big and shape.get("alone"):
            c *= 1.1                       # mid-size grids: the route is tried, and loses
        if not big and shape.get("ct_march"):
            c *= 0.995                     # below the 1% threshold: must not be taken
        if not big and shape.get("march_len") == 256:
            c *= 0.9                       # small grids: a real 10% gain
        if nt == 256:
            c *= 1.2
        return c

    class Solver:
        def __init__(self, prob):
            self.prob = prob

        @classmethod
        def from_problem(cls, prob, prec=None):
            return cls(prob)

        def close(self):
            pass

    class Batch:
        def __init__(self, solvers):
            self.solvers = solvers
            self.nt, self.shapes = 128, [{} for _ in solvers]

        def configure(self, threads_per_cta=0, ctas_per_sm=0, spin_cycles=0, shapes=None):
            self.nt = threads_per_cta or self.nt
            self.shapes = [dict(s) for s in shapes] if shapes else [{} for _ in self.solvers]
            state["configs"].append((self.nt, [dict(s) for s in self.shapes]))

        def step(self, n):
            state["t"] = n * sum(cost(s.prob, sh, self.nt)
                                 for s, sh in zip(self.solvers, self.shapes))

        def sync(self):
            return mhd.MHD_OK

        def __enter__(self):
            return self

        def __exit__(self, *a):
            pass

    clock = {"now": 0.0}

    def perf_counter():
        # every call after a step advances the clock by that step's cost
        clock["now"] += state.pop("t", 0.0)
        return clock["now"]

    monkeypatch.setattr(autotune.mhd, "Solver", Solver)
    monkeypatch.setattr(autotune.mhd, "Batch", Batch)
    monkeypatch.setattr(autotune.time, "perf_counter", perf_counter)
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "autotune.json"))
    monkeypatch.setattr(autotune, "_key", lambda shapes, nsteps: repr((sorted(shapes), nsteps)))
    return state


def test_tune_batch_descent(fake_gpu):
    probs = ([FakeProblem((256, 256, 256))] + [FakeProblem((60, 60, 60))] * 40 +
             [FakeProblem((96, 96, 96))] * 4)
    res = autotune.tune_batch(probs, nsteps=3, repeats=2)
    assert res["threads_per_cta"] == 128
    big, small = autotune.shape_class((256, 256, 256)), autotune.shape_class((60, 60, 60))
    mid = autotune.shape_class((96, 96, 96))
    assert res["classes"][big] == {"alone": 1}           # no tile shapes once routed alone
    assert res["classes"][small] == {"march_len": 256}   # 10% taken, 0.5% (ct_march) not
    assert "alone" not in res["classes"][small]          # small grids never try the route
    assert "alone" not in res["classes"][mid]            # tried (below), slower, not taken
    assert res["tuned_ms"] < res["default_ms"]
    tried = [cfg for cfg in fake_gpu["configs"]]
    routed = {p.n for _, shapes in tried for p, sh in zip(probs, shapes) if sh.get("alone")}
    assert routed == {(256, 256, 256), (96, 96, 96)}     # the route is offered from 2^19 cells
    assert 60 ** 3 < autotune.ALONE_MIN_CELLS <= 96 ** 3
    # the result is cached: a second call configures nothing
    n = len(fake_gpu["configs"])
    assert autotune.tune_batch(probs, nsteps=3, repeats=2) == res
    assert len(fake_gpu["configs"]) == n
