"""Grouped (batched) solves through the C ABI (GPU required).

Every problem of a batch is compared with the CPU oracle on its own inputs:
FP64 batches at the plain tolerances (sigma within 1e-10 relative, residual
within 1.0001x), FP32 batches at 1e-3 relative on sigma where FP32 resolves
sigma_k (sigma_k / sigma_1 >= 1e-3) and 1e-5 sigma_1 absolute everywhere.
A problem's result must be bitwise the same alone and inside the mix (no work
is shared between problems).
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import analysis
from paper_2402_17794_gb300 import rsvd as R
from paper_2402_17794_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _problems(rng, count, dtype_np, r_range=(5.0, 50.0), mrange=(256, 4096), nrange=(256, 2048),
              kmax=64):
    items, host = [], []
    for i in range(count):
        m = int(np.exp(rng.uniform(np.log(mrange[0]), np.log(mrange[1]))))
        n = int(rng.integers(nrange[0], nrange[1] + 1))
        r = float(rng.uniform(*r_range))
        k = int(rng.integers(10, kmax + 1))
        p, q = 10, 1
        k = min(k, min(m, n) - p)
        terms = min(m, n, 400)
        A = syn.lowrank_matrix(m, n, syn.spectrum("exp", terms, r=r), seed=1000 + i)
        A = A.astype(dtype_np).astype(np.float64)
        host.append((A, k, p, q, 77 + i))
    return host


def _device(host, torch_dtype):
    items = []
    for (A, k, p, q, seed) in host:
        m, n = A.shape
        items.append((R.from_numpy_f(A, dtype=torch_dtype), m, n, k, p, q, seed))
    return items


def _plan_for(items, l_max, a_dtype):
    rows = sum(it[1] for it in items)
    cols = sum(it[2] for it in items)
    return R.BatchPlan(len(items), rows, cols, l_max, a_dtype)


def test_batched_fp64_matches_oracle_per_problem():
    rng = np.random.default_rng(0)
    host = _problems(rng, 24, np.float64, mrange=(256, 1500), nrange=(256, 1200))
    items = _device(host, torch.float64)
    plan = _plan_for(items, 74, R.F64)
    res = plan.solve(items)
    codes = plan.status()
    assert codes == [0] * len(items), codes
    for (A, k, p, q, seed), (U, S, VT) in zip(host, res):
        ref = oracle.rsvd(A, k, p, q, seed)
        s = S.cpu().numpy()
        rel = np.abs(s - ref.S) / ref.S
        assert rel.max() <= 1e-10, rel.max()
        u, vt = R.to_numpy_f(U), R.to_numpy_f(VT)
        assert np.abs(u.T @ u - np.eye(k)).max() < 1e-12
        r_gpu = analysis.lowrank_residual(A, u, s, vt)
        r_orc = analysis.lowrank_residual(A, ref.U, ref.S, ref.Vt)
        assert r_gpu <= 1.0001 * r_orc + 1e-15 * ref.S[0]


def test_batched_fp32_matches_oracle_per_problem():
    rng = np.random.default_rng(1)
    host = _problems(rng, 24, np.float32, r_range=(20.0, 50.0), mrange=(256, 2048),
                     nrange=(256, 1500))
    items = _device(host, torch.float32)
    plan = _plan_for(items, 74, R.F32)
    res = plan.solve(items)
    assert plan.status() == [0] * len(items)
    for (A, k, p, q, seed), (U, S, VT) in zip(host, res):
        ref = oracle.rsvd(A, k, p, q, seed)
        s = S.cpu().numpy()
        assert np.abs(s - ref.S).max() <= 1e-5 * ref.S[0]
        resolved = ref.S / ref.S[0] >= 1e-3
        rel = np.abs(s - ref.S)[resolved] / ref.S[resolved]
        assert rel.max() <= 1e-3, rel.max()
        u = R.to_numpy_f(U)
        assert np.abs(u.T @ u - np.eye(k)).max() < 1e-4


@pytest.mark.parametrize("a_dtype,tdt,npdt", [(R.F64, torch.float64, np.float64),
                                              (R.F32, torch.float32, np.float32)])
def test_batch_result_is_the_same_alone_and_in_the_mix(a_dtype, tdt, npdt):
    rng = np.random.default_rng(2)
    host = _problems(rng, 12, npdt, mrange=(300, 1200), nrange=(300, 900))
    items = _device(host, tdt)
    mix = _plan_for(items, 74, a_dtype).solve(items)
    torch.cuda.synchronize()
    for i in (0, 5, 11):
        alone = _plan_for([items[i]], 74, a_dtype)
        (U, S, VT), = alone.solve([items[i]])
        assert alone.status() == [0]
        for x, y in zip((U, S, VT), mix[i]):
            assert torch.equal(x, y)


def test_batched_fp64_agrees_with_single_problem_solve():
    A = syn.lowrank_matrix(900, 600, syn.spectrum("poly", 600, alpha=1.5), seed=3)
    dA = R.from_numpy_f(A)
    single = R.Plan(900, 600, 40)
    U1, S1, VT1 = single.solve(dA, 900, 600, 30, 10, 2, 5)
    assert single.status() == 0
    bp = R.BatchPlan(1, 900, 600, 40, R.F64)
    (U2, S2, VT2), = bp.solve([(dA, 900, 600, 30, 10, 2, 5)])
    assert bp.status() == [0]
    s1, s2 = S1.cpu().numpy(), S2.cpu().numpy()
    assert (np.abs(s1 - s2) / s1).max() <= 1e-12
    assert np.abs(R.to_numpy_f(U1) - R.to_numpy_f(U2)).max() < 1e-9


def test_batched_mixed_q_and_statuses():
    """Problems with different q in one batch; a NaN problem fails alone."""
    rng = np.random.default_rng(4)
    host = _problems(rng, 6, np.float64, mrange=(300, 800), nrange=(300, 600))
    host = [(A, k, p, i % 3, seed) for i, (A, k, p, q, seed) in enumerate(host)]
    bad = host[2][0].copy()
    bad[3, 4] = np.nan
    host[2] = (bad,) + host[2][1:]
    items = _device(host, torch.float64)
    plan = _plan_for(items, 74, R.F64)
    res = plan.solve(items)
    codes = plan.status()
    assert codes[2] == 6 and all(c == 0 for i, c in enumerate(codes) if i != 2), codes
    for i, ((A, k, p, q, seed), (U, S, VT)) in enumerate(zip(host, res)):
        if i == 2:
            continue
        ref = oracle.rsvd(A, k, p, q, seed)
        rel = np.abs(S.cpu().numpy() - ref.S) / ref.S
        assert rel.max() <= 1e-10, (i, q, rel.max())


def test_batched_argument_errors():
    A = torch.zeros(64, 100, dtype=torch.float64, device="cuda")
    U = torch.zeros(8, 100, dtype=torch.float64, device="cuda")
    S = torch.zeros(8, dtype=torch.float64, device="cuda")
    VT = torch.zeros(64, 8, dtype=torch.float64, device="cuda")
    plan = R.BatchPlan(2, 200, 200, 16, R.F64)
    from paper_2402_17794_gb300 import _lib
    good = _lib.RsvdProblem(A.data_ptr(), 100, 64, 100, 8, 4, 1, 0, U.data_ptr(), 100,
                            S.data_ptr(), VT.data_ptr(), 8)
    bad = _lib.RsvdProblem(A.data_ptr(), 100, 64, 99, 8, 4, 1, 0, U.data_ptr(), 100,
                           S.data_ptr(), VT.data_ptr(), 8)
    assert R.rsvd_solve_batched(plan.handle, [good, bad]) == -101
    assert R.rsvd_solve_batched(plan.handle, [good, good, good]) == -2
    big = _lib.RsvdProblem(A.data_ptr(), 100, 64, 100, 8, 9, 1, 0, U.data_ptr(), 100,
                           S.data_ptr(), VT.data_ptr(), 8)
    assert R.rsvd_solve_batched(plan.handle, [big]) == 4          # l = 17 > l_max
