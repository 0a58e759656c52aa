"""Continuous batching on the GPU: every served result equals the same
request solved alone (bitwise: the grouped kernels share no work between
problems), and every result meets its own request's tolerance, relative on
each sigma_i (i <= k), against the FP64 oracle on the stored matrix.
Requests whose FP32 result cannot meet the tolerance (a steep spectrum with
a large k) are promoted to FP64 lanes by the server."""
import time

import numpy as np
import pytest
import torch

import oracle
from paper_2402_17794_gb300 import rsvd as R
from paper_2402_17794_gb300 import serve
from paper_2402_17794_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def test_served_results_equal_solo_results_and_meet_their_tolerance():
    rng = np.random.default_rng(0)
    bases = []
    for i in range(6):
        m, n = int(rng.integers(300, 1500)), int(rng.integers(300, 1000))
        A = syn.lowrank_matrix(m, n, syn.spectrum("exp", 300, r=float(rng.uniform(10, 40))),
                               seed=50 + i).astype(np.float32).astype(np.float64)
        bases.append((A, R.from_numpy_f(A, dtype=torch.float32)))
    big = syn.lowrank_matrix(2000, 1500, syn.spectrum("poly", 1500, alpha=1.0), seed=9)
    big = big.astype(np.float32).astype(np.float64)
    bases.append((big, R.from_numpy_f(big, dtype=torch.float32)))
    # a steep spectrum (sigma_i = exp(-i/5)): sigma_60 / sigma_1 ~ 7e-6 is below
    # what FP32 resolves to 1e-3, so its 1e-3 requests must be promoted
    steep = syn.lowrank_matrix(1200, 900, syn.spectrum("exp", 200, r=5.0), seed=77)
    steep = steep.astype(np.float32).astype(np.float64)
    bases.append((steep, R.from_numpy_f(steep, dtype=torch.float32)))
    torch.cuda.synchronize()
    reqs, host = [], {}
    t = 0.0
    for i in range(44):
        t += float(rng.exponential(0.004))
        if i % 13 == 5:
            b = 6
            k, p, q = 100, 20, 2
        elif i % 11 == 3:
            b = 7
            k, p, q = 60, 10, 1
        else:
            b = i % 6
            k, p, q = int(rng.integers(10, 40)), 10, 1
        A, dA = bases[b]
        tol = 1e-6 if i % 4 == 0 else 1e-3
        m, n = A.shape
        reqs.append(serve.Request(i, m, n, k, p, q, tol, 1000 + i, t, A=dA))
        host[i] = A
    specs = [serve.LaneSpec("f32-small", 8, 8 * 1500, 8 * 1000, 80),
             serve.LaneSpec("f64-small", 8, 8 * 1500, 8 * 1000, 80),
             serve.LaneSpec("f32-big", 2, 2 * 2000, 2 * 1500, 288),
             serve.LaneSpec("f64-big", 2, 2 * 2000, 2 * 1500, 288)]
    srv = serve.Server(specs, serve.TorchBackend(), 8 * 10**9, lanes_per_class=2)
    stats = serve.run(srv, reqs, time.perf_counter, max_wall=120.0)
    torch.cuda.synchronize()
    assert stats["completed"] == 44 and stats["failed"] == 0
    assert stats["batches"] < 44             # requests were batched together
    steep_1e3 = [r for r in srv.finished if host[r.rid] is steep and r.tol == 1e-3]
    assert steep_1e3 and all(r.promoted for r in steep_1e3)
    for r in srv.finished:
        cls = serve.request_class(r)
        dt = R.F32 if cls.startswith("f32") else R.F64
        tdt = torch.float32 if dt == R.F32 else torch.float64
        solo = R.BatchPlan(1, r.m, r.n, r.l, dt)
        (U, S, VT), = solo.solve([(r.A.to(tdt), r.m, r.n, r.k, r.p, r.q, r.seed)])
        assert solo.status() == [0]
        for x, y in zip((U, S, VT), r.result):
            assert torch.equal(x, y), r.rid
    # every result meets its own request's tolerance on every sigma_i
    worst = 0.0
    for r in srv.finished:
        ref = oracle.rsvd(host[r.rid], r.k, r.p, r.q, r.seed)
        s = r.result[1].cpu().numpy()
        rel = (np.abs(s - ref.S) / ref.S).max()
        assert rel <= r.tol, (r.rid, serve.request_class(r), rel, r.tol)
        if serve.request_class(r).startswith("f32"):
            worst = max(worst, float(np.abs(s - ref.S).max() / ref.S[0]))
        elif host[r.rid] is not steep:
            # sigma_k / sigma_1 >= ~1e-3 here: the plain FP64 bar applies
            assert rel <= 1e-10, (r.rid, rel)
    # the acceptance rule's bound on FP32 sigma errors holds with room to spare
    assert worst <= serve.FP32_ERR_COEF * serve.FP32_UNIT, worst


def test_tensor_lane_serves_fp64_requests_like_a_solo_tensor_plan():
    """FP64 big requests on "tensor" lanes (one request at a time on a
    tensor-core FP64 plan): each result equals the same request solved alone
    on such a plan, and meets the plain FP64 bar against the oracle."""
    rng = np.random.default_rng(3)
    A = syn.lowrank_matrix(2000, 1500, syn.spectrum("poly", 1500, alpha=1.0), seed=19)
    dA = R.from_numpy_f(A)
    torch.cuda.synchronize()
    reqs = []
    t = 0.0
    for i in range(6):
        t += float(rng.exponential(0.003))
        k, p, q = (100, 20, 2) if i % 2 == 0 else (40, 10, 1)
        reqs.append(serve.Request(i, 2000, 1500, k, p, q, 1e-6, 300 + i, t, A=dA))
    specs = [serve.LaneSpec("f64-small", 4, 4 * 2000, 4 * 1500, 80),
             serve.LaneSpec("f64-big", 1, 2000, 1500, 288, engine="tensor", lanes=2)]
    srv = serve.Server(specs, serve.TorchBackend(), 8 * 10**9, lanes_per_class=1)
    stats = serve.run(srv, reqs, time.perf_counter, max_wall=120.0)
    torch.cuda.synchronize()
    assert stats["completed"] == 6 and stats["failed"] == 0
    for r in srv.finished:
        ref = oracle.rsvd(A, r.k, r.p, r.q, r.seed)
        s = r.result[1].cpu().numpy()
        assert (np.abs(s - ref.S) / ref.S).max() <= 1e-10, r.rid
        if serve.request_class(r) == "f64-big":
            solo = R.Plan(2000, 1500, r.l, mode=R.F64_TENSOR)
            U, S, VT = solo.solve(dA, r.m, r.n, r.k, r.p, r.q, r.seed)
            torch.cuda.synchronize()
            assert solo.status() == 0
            for x, y in zip((U, S, VT), r.result):
                assert torch.equal(x, y), r.rid
