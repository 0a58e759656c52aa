"""Host logic of the continuous-batching server, with a simulated backend (no GPU)."""
import random

from paper_2402_17794_gb300 import serve


class FakeBackend:
    """Completes a batch `cost(batch)` seconds of simulated time after launch."""

    def __init__(self, clock):
        self.clock = clock
        self.state = {}
        self.launches = []
        self.concurrent_max = 0

    def create_lane(self, lane):
        self.state[lane.key] = None

    def launch(self, lane, batch):
        t = self.clock.t
        dur = 1e-3 + sum(r.m * r.n * r.l for r in batch) * 1e-12
        self.state[lane.key] = (t + dur, [0] * len(batch))
        self.launches.append((lane.key, [r.rid for r in batch], t))
        busy = sum(1 for v in self.state.values() if v is not None and v[0] > t)
        self.concurrent_max = max(self.concurrent_max, busy)

    def poll(self, lane):
        end, _ = self.state[lane.key]
        return self.clock.t >= end

    def statuses(self, lane):
        return self.state[lane.key][1]

    def sigmas(self, lane):
        """Simulated FP32 singular values: sigma_i = exp(-i / r.decay) (each
        request may carry a ``decay``; default a flat-ish spectrum)."""
        import math
        return [[math.exp(-i / getattr(r, "decay", 1e3)) for i in range(r.k)] for r in lane.batch]


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 2e-5          # every poll advances simulated time
        return self.t


SPECS = [serve.LaneSpec("f32-small", 8, 8 * 4096, 8 * 2048, 80),
         serve.LaneSpec("f64-small", 8, 8 * 4096, 8 * 2048, 80),
         serve.LaneSpec("f32-big", 2, 2 * 8192, 2 * 8192, 288),
         serve.LaneSpec("f64-big", 2, 2 * 8192, 2 * 8192, 288)]


def _requests(n, seed=0, rate=2000.0):
    rng = random.Random(seed)
    t, out = 0.0, []
    for i in range(n):
        t += rng.expovariate(rate)
        big = rng.random() < 0.05
        if big:
            m = nn = 8192
            k, p, q = 256, 32, 2
        else:
            m, nn = rng.randint(256, 4096), rng.randint(256, 2048)
            k, p, q = rng.randint(10, 64), 10, 1
        tol = rng.choice([1e-3, 1e-6])
        out.append(serve.Request(i, m, nn, k, p, q, tol, i, t))
    return out


def test_request_classes():
    r = serve.Request(0, 1000, 800, 30, 10, 1, 1e-3, 0, 0.0)
    assert serve.request_class(r) == "f32-small"
    r.tol = 1e-6
    assert serve.request_class(r) == "f64-small"
    r.k = 256
    assert serve.request_class(r) == "f64-big"


def test_all_requests_complete_fifo_within_class_and_budget_respected():
    clock = Clock()
    be = FakeBackend(clock)
    budget = 2 * 10**9
    srv = serve.Server(SPECS, be, budget, lanes_per_class=2, clock=lambda: clock.t)
    reqs = _requests(400)
    peak = [0]
    orig_fill = srv._fill

    def fill(lane, now):
        out = orig_fill(lane, now)
        peak[0] = max(peak[0], srv.in_use)
        return out

    srv._fill = fill
    stats = serve.run(srv, reqs, clock)
    assert stats["completed"] == 400 and stats["failed"] == 0
    assert peak[0] <= budget
    assert srv.in_use == 0
    # FIFO: within a class, start times follow arrival order
    by_cls = {}
    for r in sorted(srv.finished, key=lambda r: r.arrival):
        by_cls.setdefault(serve.request_class(r), []).append(r.start)
    for starts in by_cls.values():
        assert starts == sorted(starts)
    # batches never exceed a lane's slots or row/column capacity
    for key, rids, _ in be.launches:
        spec = next(s for s in SPECS if key.startswith(s.name))
        batch = [reqs[i] for i in rids]
        assert len(batch) <= spec.max_count
        assert sum(r.m for r in batch) <= spec.rows_total
        assert sum(r.n for r in batch) <= spec.cols_total
        assert all(serve.request_class(r) == spec.name for r in batch)
    assert stats["p99_ms"] >= stats["p50_ms"] > 0


def test_lanes_overlap_and_late_arrivals_are_admitted_while_others_run():
    clock = Clock()
    be = FakeBackend(clock)
    srv = serve.Server(SPECS, be, 10**12, lanes_per_class=2, clock=lambda: clock.t)
    reqs = _requests(300, seed=3, rate=20000.0)
    serve.run(srv, reqs, clock)
    assert be.concurrent_max >= 2
    # some request started while a batch launched earlier was still running
    ends = {}
    for key, rids, t in be.launches:
        ends.setdefault(key, []).append(t)
    assert len(be.launches) > len(srv.lanes)


def test_admission_budget_stalls_but_never_deadlocks():
    clock = Clock()
    be = FakeBackend(clock)
    one_big = serve.footprint_bytes(serve.Request(0, 8192, 8192, 256, 32, 2, 1e-3, 0, 0.0))
    srv = serve.Server(SPECS, be, int(1.5 * one_big), lanes_per_class=2, clock=lambda: clock.t)
    reqs = [serve.Request(i, 8192, 8192, 256, 32, 2, 1e-3, i, 0.0) for i in range(5)]
    stats = serve.run(srv, reqs, clock)
    assert stats["completed"] == 5
    assert stats["admission_stalls"] > 0


def test_percentile():
    xs = list(range(1, 101))
    assert serve.percentile(xs, 50) == 50
    assert serve.percentile(xs, 99) == 99
    assert serve.percentile([3.0], 99) == 3.0


def test_requests_that_can_never_fit_are_refused_not_blocking():
    clock = Clock()
    be = FakeBackend(clock)
    srv = serve.Server(SPECS, be, 10**6, lanes_per_class=1, clock=lambda: clock.t)
    reqs = [serve.Request(0, 8192, 8192, 256, 32, 2, 1e-3, 0, 0.0),
            serve.Request(1, 300, 300, 10, 5, 1, 1e-3, 1, 0.0)]
    stats = serve.run(srv, reqs, clock)
    assert stats["completed"] == 2
    st = {r.rid: r.status for r in srv.finished}
    assert st[0] == 4 and st[1] == 0


def test_fp32_acceptance_rule():
    u = serve.FP32_UNIT * serve.FP32_ERR_COEF
    flat = [1.0, 0.9, 0.5]
    assert serve.fp32_meets(flat, 1e-3)
    # sigma_1 / sigma_k just inside / outside tol / (coef u)
    ratio = 1e-3 / u
    assert serve.fp32_meets([1.0, 1.0 / (0.99 * ratio)], 1e-3)
    assert not serve.fp32_meets([1.0, 1.0 / (1.01 * ratio)], 1e-3)
    assert not serve.fp32_meets([1.0, 0.0], 1e-3)
    assert not serve.fp32_meets([1.0, float("nan")], 1e-3)


def test_steep_spectrum_requests_are_promoted_to_fp64():
    """A 1e-3 request whose FP32 result cannot resolve sigma_k to 1e-3 is
    solved again on an FP64 lane; the others finish on FP32 lanes."""
    clock = Clock()
    be = FakeBackend(clock)
    srv = serve.Server(SPECS, be, 10**11, lanes_per_class=1, clock=lambda: clock.t)
    reqs = []
    for i in range(20):
        r = serve.Request(i, 1000, 800, 60, 10, 1, 1e-3, i, i * 1e-4)
        r.decay = 5.0 if i % 3 == 0 else 200.0     # e^(59/5) ~ 1.3e5 vs e^(59/200) ~ 1.3
        reqs.append(r)
    stats = serve.run(srv, reqs, clock)
    assert stats["completed"] == 20 and stats["failed"] == 0
    assert stats["promotions"] == 7
    for r in srv.finished:
        steep = r.rid % 3 == 0
        assert r.promoted == steep
        assert serve.request_class(r) == ("f64-small" if steep else "f32-small")
        assert r.lane.startswith("f64" if steep else "f32")
    # promoted requests ran twice: once on an FP32 lane, then on an FP64 lane
    ran = {}
    for key, rids, _ in be.launches:
        for rid in rids:
            ran.setdefault(rid, []).append(key.split("-")[0])
    for rid, lanes in ran.items():
        assert lanes == (["f32", "f64"] if rid % 3 == 0 else ["f32"]), (rid, lanes)
    assert srv.in_use == 0


def test_tight_tolerance_goes_straight_to_fp64():
    clock = Clock()
    be = FakeBackend(clock)
    srv = serve.Server(SPECS, be, 10**11, lanes_per_class=1, clock=lambda: clock.t)
    r = serve.Request(0, 500, 400, 20, 10, 1, 1e-6, 0, 0.0)
    stats = serve.run(srv, [r], clock)
    assert stats["completed"] == 1 and stats["promotions"] == 0
    assert r.lane.startswith("f64") and not r.promoted


def test_tensor_lanes_take_fp64_requests_one_at_a_time():
    clock = Clock()
    import pytest
    bad = [serve.LaneSpec("f64-big", 2, 2 * 8192, 2 * 8192, 288, engine="tensor")]
    with pytest.raises(ValueError):
        serve.Server(bad, FakeBackend(clock), 10**12)
    bad = [serve.LaneSpec("f32-big", 1, 8192, 8192, 288, engine="tensor")]
    with pytest.raises(ValueError):
        serve.Server(bad, FakeBackend(clock), 10**12)
    ok = [serve.LaneSpec("f64-big", 1, 8192, 8192, 288, engine="tensor", lanes=3),
          serve.LaneSpec("f64-small", 8, 8 * 4096, 8 * 2048, 80)]
    srv = serve.Server(ok, FakeBackend(clock), 10**12, lanes_per_class=2)
    assert sum(1 for l in srv.lanes if l.spec.name == "f64-big") == 3
    assert sum(1 for l in srv.lanes if l.spec.name == "f64-small") == 2


def test_drain_cap_counts_unserved_requests():
    clock = Clock()
    srv = serve.Server(SPECS, FakeBackend(clock), 10**12, lanes_per_class=1)
    reqs = _requests(400, seed=5, rate=1e6)
    stats = serve.run(srv, reqs, clock, max_wall=1e9, drain_s=0.0)
    assert stats["completed"] + stats["unserved"] == 400
    assert stats["unserved"] > 0
    assert len(srv.finished) == stats["completed"]
