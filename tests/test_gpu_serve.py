"""Continuous batching on the GPU: every served result equals the same
request solved alone (bitwise: the grouped kernels share no work between
problems), and results meet the oracle at the lane's precision."""
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


def test_served_results_equal_solo_results():
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
    torch.cuda.synchronize()
    reqs = []
    t = 0.0
    for i in range(40):
        t += float(rng.exponential(0.004))
        if i % 13 == 5:
            A, dA = bases[-1]
            k, p, q = 100, 20, 2
        else:
            A, dA = bases[i % 6]
            k, p, q = int(rng.integers(10, 40)), 10, 1
        tol = 1e-6 if i % 4 == 0 else 1e-3
        m, n = A.shape
        reqs.append(serve.Request(i, m, n, k, p, q, tol, 1000 + i, t, A=dA))
    specs = [serve.LaneSpec("f32-small", 8, 8 * 1500, 8 * 1000, 80),
             serve.LaneSpec("f64-small", 8, 8 * 1500, 8 * 1000, 80),
             serve.LaneSpec("f32-big", 2, 2 * 2000, 2 * 1500, 288),
             serve.LaneSpec("f64-big", 2, 2 * 2000, 2 * 1500, 288)]
    srv = serve.Server(specs, serve.TorchBackend(), 8 * 10**9, lanes_per_class=2)
    stats = serve.run(srv, reqs, time.perf_counter, max_wall=120.0)
    torch.cuda.synchronize()
    assert stats["completed"] == 40 and stats["failed"] == 0
    assert stats["batches"] < 40             # requests were batched together
    for r in srv.finished:
        cls = serve.request_class(r)
        dt = R.F32 if cls.startswith("f32") else R.F64
        tdt = torch.float32 if dt == R.F32 else torch.float64
        solo = R.BatchPlan(1, r.m, r.n, r.l, dt)
        (U, S, VT), = solo.solve([(r.A.to(tdt), r.m, r.n, r.k, r.p, r.q, r.seed)])
        assert solo.status() == [0]
        for x, y in zip((U, S, VT), r.result):
            assert torch.equal(x, y), r.rid
    # accuracy at the lane precision, against the oracle on the stored matrix
    for r in srv.finished[:12]:
        A = bases[-1][0] if r.k == 100 else bases[r.rid % 6][0]
        ref = oracle.rsvd(A, r.k, r.p, r.q, r.seed)
        s = r.result[1].cpu().numpy()
        if serve.request_class(r).startswith("f64"):
            assert (np.abs(s - ref.S) / ref.S).max() <= 1e-10
        else:
            assert np.abs(s - ref.S).max() <= 1e-5 * ref.S[0]
