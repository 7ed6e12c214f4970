"""Host logic of the serving scheduler with a fake backend (no GPU): admission in arrival
order against the memory budget, continuous batching (requests join and leave between
iterations), every request finishes with exactly its number of steps."""
import numpy as np

from paper_0908_4362_gb300 import inputs as I
from paper_0908_4362_gb300 import serve


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 1e-3
        return self.t


class FakeHandle:
    def __init__(self, prob):
        self.prob = prob
        self.steps = 0
        self.closed = False


class FakeBatch:
    def __init__(self, be, handles):
        self.be, self.handles = be, handles
        be.batches.append(len(handles))

    def step_each(self, counts):
        assert len(counts) == len(self.handles) and max(counts) >= 1
        for h, k in zip(self.handles, counts):
            assert not h.closed and k >= 0
            h.steps += k

    def close(self):
        self.handles = []


class FakeBackend:
    def __init__(self):
        self.batches = []
        self.live = 0
        self.max_live = 0

    def create(self, prob, f32):
        self.live += 1
        self.max_live = max(self.max_live, self.live)
        return FakeHandle(prob)

    def batch(self, handles):
        return FakeBatch(self, handles)

    def step(self, h, n):
        h.steps += n

    def read(self, h):
        return np.array([h.steps])

    def sync(self, batch):
        pass

    def wait(self, h):
        pass

    def close(self, h):
        h.closed = True
        self.live -= 1


def _trace(n=12, rate=1e4):
    return I.serving_trace(n, rate, seed=3, ot_range=(16, 48), blast_range=(8, 16),
                           steps_range=(4, 11), quantum=4)


def test_every_request_gets_its_steps_and_budget_holds():
    tr = _trace()
    be = FakeBackend()
    budget = 3 * serve.device_bytes(16 ** 3)
    s = serve.Server(be, budget_bytes=budget, clock=FakeClock(), plain_min_cells=12 ** 3,
                     keep_results=True)
    jobs = s.run(tr)
    assert len(jobs) == len(tr)
    for j in jobs:
        assert j.done >= j.admitted >= j.req.arrival - 1e-9 or j.req.arrival > 0
        assert int(j.result[0]) == j.req.steps
    assert s.peak_bytes <= budget
    assert be.live == 0
    # continuous batching: batches of more than one request formed
    assert max(be.batches) > 1


def test_request_larger_than_budget_is_rejected():
    tr = _trace(4)
    be = FakeBackend()
    s = serve.Server(be, budget_bytes=serve.device_bytes(8), clock=FakeClock())
    jobs = s.run(tr)
    assert all(j.done != j.done for j in jobs)   # NaN: rejected
    assert serve.summarize(jobs)["rejected"] == len(tr)


def test_sequential_baseline_runs_in_arrival_order():
    tr = _trace(6)
    jobs = serve.serve_sequential(FakeBackend(), tr, clock=FakeClock(), keep_results=True)
    assert [j.req.rid for j in jobs] == [r.rid for r in sorted(tr, key=lambda r: r.arrival)]
    assert all(int(j.result[0]) == j.req.steps for j in jobs)
    summ = serve.summarize(jobs)
    assert summ["completed"] == 6 and summ["p99_s"] >= summ["p50_s"]


def test_budget_of_one_request_serialises():
    tr = [I.Request(i, 0.0, "blast3d", 16, 5) for i in range(4)]
    be = FakeBackend()
    s = serve.Server(be, budget_bytes=serve.device_bytes(16 ** 3), clock=FakeClock(), keep_results=True)
    jobs = s.run(tr)
    assert be.max_live == 1 and be.live == 0
    assert [int(j.result[0]) for j in jobs] == [5] * 4
    # admitted one after another: each is admitted after the previous one finished
    for a, b in zip(jobs, jobs[1:]):
        assert b.admitted >= a.done


def test_counts_share_work_and_keep_phase():
    be = FakeBackend()
    s = serve.Server(be, iter_ms=10.0, rate0=1e8, max_steps=240, clock=FakeClock())
    small = serve.Job(I.Request(0, 0.0, "ot2d", 16, 500), 0, remaining=500)
    big = serve.Job(I.Request(1, 0.0, "blast3d", 64, 500), 0, remaining=500)
    tail = serve.Job(I.Request(2, 0.0, "blast3d", 64, 2), 0, remaining=2)
    c = s.counts([small, big, tail])
    # equal cell updates per request: the 256-cell grid gets the cap, the 64^3 grid 1 step
    assert c == [240, 1, 1]
    s.rate = 3e9
    c = s.counts([small, big])
    assert c[0] == 240 and c[1] % 3 == 0 and c[1] >= 3
    assert all(x <= j.remaining for x, j in zip(c, [small, big]))
