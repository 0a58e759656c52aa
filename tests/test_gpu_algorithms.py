"""Algorithms 2, 3 and 6 through rsvd_solve_algorithm (GPU required).

Algorithm 3 (Section 3.2: q power steps with no orthonormalisation in
between, then one orth) is compared with the oracle's Algorithm 3 on the same
seeded A and Omega: residual within 1.0001x the oracle's, sigma_i within
max(1e-10, u (sigma_1/sigma_i)^(2q+1)) relative -- the sample holds
direction i at relative size (sigma_i/sigma_1)^(2q+1), so FP64 rounding moves
it by that much, which is the round-off the thesis cites against Algorithm 3.
Cases include samples of condition number (sigma_1/sigma_l)^(2q+1) ~ 6e9 and
8e10, whose Gram squares past 1/u: plain CholeskyQR2 cannot orthonormalise
them, shifted CholeskyQR3 does.
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


def _solve(alg, A, k, p, q, seed):
    m, n = A.shape
    dA = R.from_numpy_f(A)
    plan = R.Plan(m, n, k + p)
    U, S, VT = plan.solve_algorithm(alg, dA, m, n, k, p, q, seed)
    st = plan.status()
    assert st == 0, R.rsvd_status_string(st)
    return U, S, VT


@pytest.mark.parametrize("m,n,k,p,q,spec", [
    (1000, 777, 20, 10, 1, ("poly", 1.0)),
    (777, 1200, 15, 5, 1, ("poly", 1.5)),
    (2048, 1024, 64, 16, 1, ("exp", 30.0)),
    (1024, 512, 20, 10, 2, ("twos", 0.0)),     # sigma_i = 2^(-i/4): cond(Y) ~ 8e10
    (777, 1200, 15, 5, 2, ("poly", 1.5)),      # cond(Y) ~ 5.7e9
])
def test_algorithm3_matches_oracle(m, n, k, p, q, spec):
    kind, arg = spec
    r = min(m, n)
    if kind == "twos":
        sig = 2.0 ** (-np.arange(r) / 4.0)
    elif kind == "poly":
        sig = syn.spectrum("poly", r, alpha=arg)
    else:
        sig = syn.spectrum("exp", r, r=arg)
    A = syn.lowrank_matrix(m, n, sig, seed=m + n + q)
    ref = oracle.rsvd(A, k, p, q, seed=4, algorithm=3)
    U, S, VT = _solve(3, A, k, p, q, 4)
    s = S.cpu().numpy()
    rel = np.abs(s - ref.S) / ref.S
    # Algorithm 3's sample carries direction i at relative size (sigma_i /
    # sigma_1)^(2q+1), so FP64 rounding (different summation orders on the
    # two sides) moves it by ~u (sigma_1/sigma_i)^(2q+1): the bar is 1e-10 or
    # that, whichever is larger (the round-off regime Section 3.3 cites)
    tol = np.maximum(1e-10, 1.1e-16 * (sig[0] / sig[:k]) ** (2 * q + 1))
    assert np.all(rel <= tol), (rel / tol).max()
    u, vt = R.to_numpy_f(U), R.to_numpy_f(VT)
    assert np.abs(u.T @ u - np.eye(k)).max() < 1e-12
    r_gpu = analysis.lowrank_residual(A, u, s, vt)
    r_orc = analysis.lowrank_residual(A, ref.U, ref.S, ref.Vt)
    assert r_gpu <= 1.0001 * r_orc + 1e-15 * ref.S[0], (r_gpu, r_orc)


def test_algorithm2_is_algorithm4_without_power_steps():
    A = syn.lowrank_matrix(900, 600, syn.spectrum("poly", 600, alpha=1.5), seed=1)
    a = _solve(2, A, 30, 10, 3, 7)      # q ignored
    b = _solve(4, A, 30, 10, 0, 7)
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    ref = oracle.rsvd(A, 30, 10, 0, seed=7, algorithm=2)
    assert (np.abs(a[1].cpu().numpy() - ref.S) / ref.S).max() <= 1e-10


def test_algorithm6_is_the_single_pass_solve():
    A = syn.lowrank_matrix(800, 700, syn.spectrum("exp", 700, r=10.0), seed=2)
    dA = R.from_numpy_f(A)
    plan = R.Plan(800, 700, 30)
    a = plan.solve_algorithm(6, dA, 800, 700, 20, 10, 5, 9)
    b = plan.solve_singlepass(dA, 800, 700, 20, 10, 9)
    assert plan.status() == 0
    for x, y in zip(a, b):
        assert torch.equal(x, y)


def test_algorithm_argument_errors():
    plan = R.Plan(100, 80, 16)
    A = torch.zeros(80, 100, dtype=torch.float64, device="cuda")
    U = torch.zeros(8, 100, dtype=torch.float64, device="cuda")
    S = torch.zeros(8, dtype=torch.float64, device="cuda")
    VT = torch.zeros(80, 8, dtype=torch.float64, device="cuda")
    assert R.rsvd_solve_algorithm(plan.handle, 5, A, 100, 80, 100, 8, 4, 1, 0, U, 100, S, VT, 8) == -2
    assert R.rsvd_solve_algorithm(plan.handle, 3, A, 100, 80, 99, 8, 4, 1, 0, U, 100, S, VT, 8) == -6
    assert R.rsvd_solve_algorithm(plan.handle, 3, A, 100, 80, 100, 8, 4, -1, 0, U, 100, S, VT, 8) == -9
    mplan = R.Plan(100, 80, 16, a_dtype=R.BF16, mode=R.MIXED)
    assert R.rsvd_solve_algorithm(mplan.handle, 3, A, 100, 80, 104, 8, 4, 1, 0, U, 100, S, VT, 8) == 7


def test_algorithm6_config_full_size_fp64():
    """The benchmark's Algorithm 6 solve: A 16384 x 8192 FP64, Haar factors,
    sigma_i = i^-1.5, k = 64, p = 16, seed 2: sigma within 1e-10 relative and
    the residual within 1.0001x of the oracle's single-pass solve."""
    from oracle import singlepass as sp
    m, n, k, p, seed = 16384, 8192, 64, 16, 2
    dA = syn.lowrank_matrix_torch(m, n, syn.spectrum("poly", n, alpha=1.5), seed=0)
    A = np.asfortranarray(dA.cpu().numpy().T)
    plan = R.Plan(m, n, k + p)
    U, S, VT = plan.solve_algorithm(6, dA, m, n, k, p, 0, seed)
    st = plan.status()
    assert st == 0, R.rsvd_status_string(st)
    ref = sp.singlepass_rsvd(A, k, p, seed)
    s = S.cpu().numpy()
    rel = np.abs(s - ref.S) / ref.S
    assert rel.max() <= 1e-10, rel.max()
    u, vt = R.to_numpy_f(U), R.to_numpy_f(VT)
    r_gpu = analysis.lowrank_residual(A, u, s, vt)
    r_orc = analysis.lowrank_residual(A, ref.U, ref.S, ref.Vt)
    assert r_gpu <= 1.0001 * r_orc + 1e-15 * ref.S[0], (r_gpu, r_orc)
