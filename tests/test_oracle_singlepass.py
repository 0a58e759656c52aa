"""Pins of the single-pass oracle (Algorithm 6, Section 3.4.2).

What ties it to the method rather than to itself: exact recovery of a
matrix of rank k (both sketches then capture the full row and column
spaces and the joint system is consistent), the stacked Kronecker least
squares for the joint system, the exact solution of a consistent system,
the transposition symmetry of the method (swap A with A* and the two test
matrices and U, V swap), Eckart-Young, orthonormality, and a planted
mistake (the listing's literal Y_r = A Omega_r) that the pins catch.
"""
import numpy as np
import pytest

from oracle import analysis, philox, randsvd
from oracle import singlepass as sp
from paper_2402_17794_gb300 import synthetic as syn


@pytest.mark.parametrize("m,n,k,p", [(300, 200, 10, 5), (150, 400, 12, 8), (256, 256, 20, 10)])
def test_exact_rank_k_recovery(m, n, k, p):
    sig = np.array([3.0 * 2.0 ** (-i / 2) for i in range(k)])
    A = syn.lowrank_matrix(m, n, sig, seed=m + n)
    r = sp.singlepass_rsvd(A, k, p, seed=7)
    assert np.abs(r.S - sig).max() <= 1e-12 * sig[0]
    assert np.linalg.norm(A - r.U @ np.diag(r.S) @ r.Vt, 2) <= 1e-12 * sig[0]


def _sylvester_normal_equations(M, P, N, R):
    """Test-side cross-check of step 4 by a different route: the normal
    equations of the joint problem are the Sylvester equation
    (M* M) C + C (N N*) = M* P + R N*, whose SPD coefficients are
    diagonalised by their eigendecompositions."""
    la, Va = np.linalg.eigh(M.T @ M)
    lb, Vb = np.linalg.eigh(N @ N.T)
    G = (Va.T @ (M.T @ P + R @ N.T) @ Vb) / (la[:, None] + lb[None, :])
    return Va @ G @ Vb.T


def test_joint_lstsq_minimises_both_residuals():
    """The stacked solution is a stationary point of the joint objective (its
    gradient M*(MC-P) + (CN-R)N* vanishes), it agrees with the Sylvester
    normal equations, and no perturbation lowers the objective."""
    rng = np.random.default_rng(0)
    for l, k in [(9, 4), (12, 12), (20, 7)]:
        M, P = rng.standard_normal((l, k)), rng.standard_normal((l, k))
        N, R = rng.standard_normal((k, l)), rng.standard_normal((k, l))
        C = sp.joint_lstsq(M, P, N, R)
        grad = M.T @ (M @ C - P) + (C @ N - R) @ N.T
        assert np.abs(grad).max() <= 1e-11 * max(1.0, np.abs(C).max())
        ref = _sylvester_normal_equations(M, P, N, R)
        assert np.abs(C - ref).max() <= 1e-11 * max(1.0, np.abs(ref).max())

        def obj(X):
            return np.linalg.norm(M @ X - P) ** 2 + np.linalg.norm(X @ N - R) ** 2
        f0 = obj(C)
        for _ in range(5):
            assert obj(C + 1e-3 * rng.standard_normal(C.shape)) > f0


def test_joint_lstsq_planted_mistake_one_equation_only():
    """Planted mistake: solving only the first equation (M C = P) is not the
    joint least squares; the stationarity pin catches it."""
    rng = np.random.default_rng(2)
    l, k = 12, 5
    M, P = rng.standard_normal((l, k)), rng.standard_normal((l, k))
    N, R = rng.standard_normal((k, l)), rng.standard_normal((k, l))
    bad = np.linalg.lstsq(M, P, rcond=None)[0]
    grad = M.T @ (M @ bad - P) + (bad @ N - R) @ N.T
    assert np.abs(grad).max() > 1e-3


def test_joint_lstsq_recovers_a_consistent_solution():
    rng = np.random.default_rng(1)
    l, k = 15, 6
    C0 = rng.standard_normal((k, k))
    M, N = rng.standard_normal((l, k)), rng.standard_normal((k, l))
    C = sp.joint_lstsq(M, M @ C0, N, C0 @ N)
    assert np.abs(C - C0).max() <= 1e-12


def test_transposition_symmetry():
    m, n, k, p = 220, 160, 12, 6
    A = syn.lowrank_matrix(m, n, syn.spectrum("poly", 160, alpha=1.5), seed=3)
    l = k + p
    Oc = philox.gaussian_matrix(n, l, 5, stream=0)
    Or = philox.gaussian_matrix(m, l, 5, stream=1)
    a = sp.singlepass_rsvd(A, k, p, 5, Omega_c=Oc, Omega_r=Or)
    b = sp.singlepass_rsvd(A.T, k, p, 5, Omega_c=Or, Omega_r=Oc)
    assert np.abs(a.S - b.S).max() <= 1e-12 * a.S[0]
    # U of one is V of the other, up to the sign of each pair
    d = np.abs(np.sum(a.U * b.Vt.T, axis=0))
    assert np.abs(d - 1.0).max() <= 1e-9


def test_eckart_young_and_orthonormality():
    m, n, k, p = 400, 300, 15, 10
    A = syn.lowrank_matrix(m, n, syn.spectrum("poly", 300, alpha=1.0), seed=4)
    r = sp.singlepass_rsvd(A, k, p, seed=2)
    sig = np.linalg.svd(A, compute_uv=False)
    err = np.linalg.norm(A - r.U @ np.diag(r.S) @ r.Vt, 2)
    assert err >= sig[k] * (1 - 1e-12)
    assert np.abs(r.U.T @ r.U - np.eye(k)).max() <= 1e-12
    assert np.abs(r.Vt @ r.Vt.T - np.eye(k)).max() <= 1e-12
    # the single-pass estimate is less accurate than Algorithm 2 but of the
    # same order on a decaying spectrum
    two = randsvd.rsvd(A, k, p, 0, seed=2)
    err2 = analysis.lowrank_residual(A, two.U, two.S, two.Vt)
    assert err <= 20 * err2


def _literal_listing(A, k, p, seed):
    """Planted mistake: Y_r = A Omega_r as the listing prints it (square A)."""
    m, n = A.shape
    l = k + p
    Oc = philox.gaussian_matrix(n, l, seed, stream=0)
    Or = philox.gaussian_matrix(m, l, seed, stream=1)
    Yc, Yr = A @ Oc, A @ Or
    Qc, Qr = sp.dominant_left(Yc, k), sp.dominant_left(Yr, k)
    C = sp.joint_lstsq(Or.T @ Qc, Yr.T @ Qr, Qr.T @ Oc, Qc.T @ Yc)
    return np.linalg.svd(C, compute_uv=False)


def test_planted_mistake_is_caught():
    m = n = 200
    k, p = 10, 5
    sig = np.array([2.0 ** -i for i in range(k)])
    A = syn.lowrank_matrix(m, n, sig, seed=11)      # square, not symmetric
    s_bad = _literal_listing(A, k, p, seed=7)
    assert np.abs(s_bad - sig).max() > 1e-6 * sig[0]
    s_good = sp.singlepass_rsvd(A, k, p, seed=7).S
    assert np.abs(s_good - sig).max() <= 1e-12 * sig[0]
