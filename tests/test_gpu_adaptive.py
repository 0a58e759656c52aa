"""Parity of the adaptive range finder and the adaptive SVD (Adaptive_randRF;
Halko, Martinsson and Tropp 2011, Algorithm 4.2) with the CPU oracle through
the C ABI (GPU required).

Same seeded A and the same Gaussian samples (Philox stream 0 of the seed,
column i-1 for omega_i) on both sides.  The rank is an integer decided by
FP64 comparisons on both sides, so it must match exactly; every case checks
first that no lookahead maximum of the oracle lies within 1e-6 of the
threshold (else rounding order could flip the decision).  The GPU orthonormal-
ises blocks of up to 64 samples (two Gram-Schmidt projections + shifted
CholeskyQR3); the oracle takes one vector at a time, so agreement is about the
method.  Q columns are Gram-Schmidt vectors, unique up to sign: 1 - |q_gpu .
q_oracle| <= 1e-8.  The SVD: singular values within 1e-10 relative (plain
FP64 tolerance) for sigma_i >= 1e-4 sigma_1, and within 1e-14 sigma_1
absolute below that, where both sides sit at rounding of ||A||.
"""
import numpy as np
import pytest
import torch

from oracle import adaptive as ad
from oracle import analysis
from paper_2402_17794_gb300 import rsvd as R
from paper_2402_17794_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _device(A, lda_pad=0):
    m, n = A.shape
    dA = torch.zeros(n, m + lda_pad, dtype=torch.float64, device="cuda")
    dA[:, :m] = R.from_numpy_f(A)
    return dA, m + lda_pad


def _margin_ok(ref):
    looks = np.array(ref.lookahead)
    return np.abs(looks / ref.threshold - 1.0).min() > 1e-6


def _compare_range(A, eps, r, l_cap, seed, plan_l=None, lda_pad=0):
    m, n = A.shape
    ref = ad.adaptive_range_finder(A, eps, r, seed, l_max=l_cap)
    assert _margin_ok(ref)
    dA, lda = _device(A, lda_pad)
    plan = R.Plan(m, n, plan_l or l_cap)
    Q, converged = plan.range_adaptive(dA, m, n, eps, r, l_cap, seed, lda=lda)
    assert plan.status() == 0
    assert converged == ref.converged
    assert Q.shape[0] == ref.rank, (Q.shape[0], ref.rank)
    q = R.to_numpy_f(Q)
    j = ref.rank
    if j:
        assert np.abs(q.T @ q - np.eye(j)).max() <= 1e-12
        d = np.abs(np.sum(q * ref.Q, axis=0))
        assert (1.0 - d).max() <= 1e-8, (1.0 - d).max()
    return ref


@pytest.mark.parametrize("m,n,spec,eps,r,seed", [
    (300, 200, 3.0, 1e-3, 10, 9),          # one block
    (2000, 1500, 15.0, 1e-2, 10, 4),       # several blocks of 64
    (1500, 2100, 12.0, 1e-4, 5, 1),        # wide, smaller lookahead
    (1031, 517, 6.0, 1e-6, 20, 7),         # ragged sizes, long lookahead
])
def test_range_matches_oracle(m, n, spec, eps, r, seed):
    A = syn.lowrank_matrix(m, n, syn.spectrum("exp", min(m, n), r=spec), seed=m + n)
    ref = _compare_range(A, eps, r, min(m, n, 288), seed)
    assert ref.converged and ref.rank > 0


def test_range_ragged_lda_and_plan_larger_than_cap():
    m, n = 777, 640
    A = syn.lowrank_matrix(m, n, syn.spectrum("exp", n, r=10.0), seed=3)
    _compare_range(A, 1e-3, 8, 120, seed=2, plan_l=200, lda_pad=5)


@pytest.mark.parametrize("k", [1, 7, 70])
def test_exact_rank_stops_at_rank(k):
    m, n = 900, 700
    sig = np.geomspace(1.0, 1e-2, k)
    A = syn.lowrank_matrix(m, n, sig, seed=k)
    ref = _compare_range(A, 1e-8, 6, 200, seed=3)
    assert ref.rank == k


def test_capacity_not_reached():
    m, n = 1200, 900
    A = syn.lowrank_matrix(m, n, syn.spectrum("poly", n, alpha=0.5), seed=1)
    ref = _compare_range(A, 1e-6, 5, 90, seed=2)
    assert not ref.converged and ref.rank == 90


def test_tolerance_met_on_gpu():
    m, n = 1600, 1000
    sig = syn.spectrum("poly", n, alpha=3.0)
    A = syn.lowrank_matrix(m, n, sig, seed=5)
    dA, lda = _device(A)
    plan = R.Plan(m, n, 288)
    for eps in (1e-2, 1e-4):
        Q, conv = plan.range_adaptive(dA, m, n, eps, 10, 288, seed=11)
        q = R.to_numpy_f(Q)
        assert conv
        err = np.linalg.norm(A - q @ (q.T @ A), 2)
        assert sig[q.shape[1]] * (1 - 1e-12) <= err <= eps


@pytest.mark.parametrize("m,n,spec,eps,r", [(1000, 800, 10.0, 1e-5, 10), (600, 1400, 5.0, 1e-9, 8)])
def test_solve_matches_oracle(m, n, spec, eps, r):
    A = syn.lowrank_matrix(m, n, syn.spectrum("exp", min(m, n), r=spec), seed=m)
    ref = ad.adaptive_rsvd(A, eps, r, seed=6, l_max=288)
    assert _margin_ok(ref.range)
    dA, lda = _device(A)
    plan = R.Plan(m, n, 288)
    U, S, VT, conv = plan.solve_adaptive(dA, m, n, eps, r, 288, seed=6)
    assert plan.status() == 0 and conv
    j = ref.range.rank
    assert S.numel() == j
    s = S.cpu().numpy()
    big = ref.S >= 1e-4 * ref.S[0]
    rel = np.abs(s[big] - ref.S[big]) / ref.S[big]
    assert rel.max() <= 1e-10, rel.max()
    assert np.abs(s[~big] - ref.S[~big]).max(initial=0.0) <= 1e-14 * ref.S[0]
    u, vt = R.to_numpy_f(U), R.to_numpy_f(VT)
    assert np.abs(u.T @ u - np.eye(j)).max() < 1e-12
    r_gpu = analysis.lowrank_residual(A, u, s, vt)
    r_orc = analysis.lowrank_residual(A, ref.U, ref.S, ref.Vt)
    assert r_gpu <= 1.0001 * r_orc + 1e-15 * ref.S[0], (r_gpu, r_orc)
    # the leading vectors (well separated sigma) agree with the oracle's signs
    lead = int(big.sum() // 2)
    assert np.abs(u[:, :lead] - ref.U[:, :lead]).max() < 1e-7


def test_adaptive_argument_errors():
    plan = R.Plan(100, 80, 40)
    A = torch.zeros(80, 100, dtype=torch.float64, device="cuda")
    Q = torch.zeros(40, 100, dtype=torch.float64, device="cuda")
    f = R.rsvd_range_adaptive
    assert f(plan.handle, A, 100, 80, 99, 1e-3, 5, 20, 0, Q, 100)[0] == -5
    assert f(plan.handle, A, 100, 80, 100, 0.0, 5, 20, 0, Q, 100)[0] == -6
    assert f(plan.handle, A, 100, 80, 100, float("nan"), 5, 20, 0, Q, 100)[0] == -6
    assert f(plan.handle, A, 100, 80, 100, 1e-3, 0, 20, 0, Q, 100)[0] == -7
    assert f(plan.handle, A, 100, 80, 100, 1e-3, 40, 20, 0, Q, 100)[0] == -7   # r >= l_max
    assert f(plan.handle, A, 100, 80, 100, 1e-3, 5, 81, 0, Q, 100)[0] == -8
    assert f(plan.handle, A, 100, 80, 100, 1e-3, 5, 41, 0, Q, 100)[0] == 4
    assert f(plan.handle, A, 100, 80, 100, 1e-3, 5, 20, 0, Q, 99)[0] == -11
    # A = 0: the first r samples already meet any tolerance, rank 0
    code, rank = f(plan.handle, A, 100, 80, 100, 1e-3, 5, 20, 0, Q, 100)
    assert code == 0 and rank == 0


def test_adaptive_config_full_size_fp64():
    """The benchmark's adaptive solve: A 16384 x 8192 FP64, Haar factors,
    sigma_i = i^-1.5, eps = 0.25, r = 10, l_cap = 128, in the launch
    configuration the benchmark times."""
    m, n = 16384, 8192
    eps, r, cap = 0.25, 10, 128
    dA = syn.lowrank_matrix_torch(m, n, syn.spectrum("poly", n, alpha=1.5), seed=0)
    A = np.asfortranarray(dA.cpu().numpy().T)
    ref = ad.adaptive_rsvd(A, eps, r, seed=2, l_max=cap)
    assert _margin_ok(ref.range) and ref.range.converged
    plan = R.Plan(m, n, cap)
    U, S, VT, conv = plan.solve_adaptive(dA, m, n, eps, r, cap, seed=2)
    assert plan.status() == 0 and conv
    j = ref.range.rank
    assert S.numel() == j
    s = S.cpu().numpy()
    rel = np.abs(s - ref.S) / ref.S
    assert rel.max() <= 1e-10, rel.max()
    u, vt = R.to_numpy_f(U), R.to_numpy_f(VT)
    r_gpu = analysis.lowrank_residual(A, u, s, vt)
    r_orc = analysis.lowrank_residual(A, ref.U, ref.S, ref.Vt)
    assert r_gpu <= 1.0001 * r_orc, (r_gpu, r_orc)
    assert r_gpu <= eps
