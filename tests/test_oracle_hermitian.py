"""Pins of the Algorithm 5 oracle (single-pass randomized EVD of a Hermitian
matrix, Section 3.4.1), CPU only.

What ties it to the method rather than to itself:
* exact recovery of a symmetric matrix of rank k (Y then spans its range,
  Eq. 3.7 holds exactly and Eq. 3.13 is consistent), with an indefinite
  spectrum so that the order by magnitude is exercised;
* the solved C is Hermitian (Eq. 3.9) when Eq. 3.12 holds exactly;
* brute force: with k + p = k = n the method returns the full
  eigendecomposition, compared with LAPACK's symmetric eigensolver;
* Eckart-Young for Hermitian matrices (the best rank-k error in the
  2-norm is the (k+1)-th largest |lambda|) and orthonormality of U;
* accuracy of the same order as the two-pass Algorithm 2 on a decaying
  spectrum (the thesis notes the single pass is less accurate);
* planted mistakes (a transposed lift, ordering by signed value, C formed
  without the least-squares solve) that the pins must catch.
"""
import numpy as np
import pytest

from oracle import hermitian as oh
from oracle import randsvd
from oracle.philox import gaussian_matrix
from paper_2402_17794_gb300 import synthetic as syn


def _check_exact_rank(fn, n=240, k=12, p=6, seed=3):
    lam = syn.signed_spectrum(3.0 * 2.0 ** (-np.arange(k) / 2), seed=11)
    A = syn.symmetric_matrix(n, lam, seed=n + k)
    r = fn(A, k, p, seed)
    ref = lam[np.argsort(-np.abs(lam), kind="stable")]
    assert np.abs(r.D - ref).max() <= 1e-12 * np.abs(lam).max()
    assert np.linalg.norm(A - (r.U * r.D) @ r.U.T, 2) <= 1e-12 * np.abs(lam).max()


@pytest.mark.parametrize("n,k,p", [(240, 12, 6), (300, 20, 10), (128, 5, 0)])
def test_exact_rank_k_recovery_indefinite(n, k, p):
    _check_exact_rank(oh.hermitian_singlepass, n, k, p)


def test_solved_C_is_hermitian_for_exact_rank():
    n, k, p = 200, 10, 5
    lam = syn.signed_spectrum(np.linspace(2.0, 0.5, k), seed=4)
    A = syn.symmetric_matrix(n, lam, seed=9)
    r = oh.hermitian_singlepass(A, k, p, seed=1)
    assert np.abs(r.C - r.C.T).max() <= 1e-12 * np.abs(r.C).max()


def test_full_rank_brute_force_evd():
    """k = n, p = 0: Q spans everything, Q* Omega is invertible and the system
    of step 4 is square and exact, so C = Q* A Q and the method returns the
    full eigendecomposition."""
    n = 40
    lam = syn.signed_spectrum(np.exp(-np.arange(n) / 8.0) + 0.01 * np.arange(n)[::-1] / n, seed=5)
    A = syn.symmetric_matrix(n, lam, seed=6)
    r = oh.hermitian_singlepass(A, n, 0, seed=2)
    w, V = np.linalg.eigh(A)
    order = np.argsort(-np.abs(w), kind="stable")
    w, V = w[order], V[:, order]
    assert np.abs(r.D - w).max() <= 1e-12 * np.abs(w).max()
    d = np.abs(np.sum(r.U * V, axis=0))
    assert np.abs(d - 1.0).max() <= 1e-9


def test_eckart_young_and_orthonormality():
    n, k, p = 400, 15, 10
    lam = syn.signed_spectrum(syn.spectrum("poly", 400, alpha=1.0), seed=7)
    A = syn.symmetric_matrix(n, lam, seed=8)
    r = oh.hermitian_singlepass(A, k, p, seed=3)
    mags = np.sort(np.abs(lam))[::-1]
    err = np.linalg.norm(A - (r.U * r.D) @ r.U.T, 2)
    assert err >= mags[k] * (1 - 1e-12)
    assert np.abs(r.U.T @ r.U - np.eye(k)).max() <= 1e-12
    # same order as the two-pass method (Algorithm 2) on the same Omega
    two = randsvd.rsvd(A, k, p, 0, seed=3)
    err2 = np.linalg.norm(A - (two.U * two.S) @ two.Vt, 2)
    assert err <= 20 * err2


def test_positive_definite_gives_positive_eigenvalues():
    n, k, p = 150, 8, 8
    lam = syn.spectrum("exp", 150, r=3.0)
    A = syn.symmetric_matrix(n, lam, seed=12)
    r = oh.hermitian_singlepass(A, k, p, seed=4)
    assert (r.D > 0).all()
    np.testing.assert_allclose(r.D[:3], lam[:3], rtol=5e-2)   # tail sum ~ 0.018


# -- planted mistakes -------------------------------------------------------

def _mutant(kind):
    def fn(A, k, p, seed):
        n = A.shape[0]
        Om = gaussian_matrix(n, k + p, seed, stream=0)
        Y = A @ Om
        Q = oh.dominant_left(Y, k)
        if kind == "no_solve":
            C = (Q.T @ Y) @ (Q.T @ Om).T
        else:
            C = oh.solve_step4(Q.T @ Om, Q.T @ Y)
        lam, Uh = np.linalg.eigh(0.5 * (C + C.T))
        order = np.argsort(-lam if kind == "signed_order" else -np.abs(lam), kind="stable")
        lam, Uh = lam[order], Uh[:, order]
        U = Q @ (Uh.T if kind == "transposed_lift" else Uh)
        return oh.HermitianResult(U=U, D=lam, C=C, Q=Q)
    return fn


@pytest.mark.parametrize("kind", ["no_solve", "signed_order", "transposed_lift"])
def test_planted_mistakes_are_caught(kind):
    _check_exact_rank(_mutant("none"))          # the test-side copy is sound
    with pytest.raises(AssertionError):
        _check_exact_rank(_mutant(kind))
