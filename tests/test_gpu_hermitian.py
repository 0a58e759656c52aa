"""Parity of the single-pass Hermitian solve (Algorithm 5, Section 3.4.1) with
the CPU oracle through the C ABI (GPU required).

Same seeded symmetric A (Haar eigenvectors, prescribed signed eigenvalues)
and the same Gaussian test matrix (Philox stream 0 of the seed) on both
sides; the plain FP64 tolerances: eigenvalues within 1e-10 relative,
residual ||A - U D U^T||_2 within 1.0001x the oracle's.  The GPU forms the
dominant singular vectors of Y through CholeskyQR2 + Jacobi, solves the
least squares of Eq. 3.13 through its normal equations and decomposes the
symmetric part of C by a one-sided Jacobi SVD; the oracle uses LAPACK's SVD,
least-squares solver and symmetric eigensolver.
"""
import numpy as np
import pytest
import torch

from oracle import analysis
from oracle import hermitian as oh
from paper_2402_17794_gb300 import rsvd as R
from paper_2402_17794_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _check(A, dA, k, p, seed, lda, exact_rank=False):
    n = A.shape[0]
    ref = oh.hermitian_singlepass(A, k, p, seed)
    plan = R.Plan(n, n, k + p)
    U, D = plan.solve_hermitian(dA, n, k, p, seed, lda=lda)
    st = plan.status()
    assert st == 0, R.rsvd_status_string(st)
    d = D.cpu().numpy()
    u = R.to_numpy_f(U)
    rel = np.abs(d - ref.D) / np.abs(ref.D)
    assert rel.max() <= 1e-10, (rel.max(), d[:4], ref.D[:4])
    assert np.abs(u.T @ u - np.eye(k)).max() < 1e-12
    r_gpu = analysis.lowrank_residual(A, u, d, u.T)
    r_orc = analysis.lowrank_residual(A, ref.U, ref.D, ref.U.T)
    scale = np.abs(ref.D).max()
    if exact_rank:
        assert max(r_gpu, r_orc) <= 1e-12 * scale, (r_gpu, r_orc)
    else:
        assert r_gpu <= 1.0001 * r_orc + 1e-15 * scale, (r_gpu, r_orc)
    assert np.abs(u - ref.U).max() < 1e-7
    return rel.max()


@pytest.mark.parametrize("n,k,p,decay", [(1000, 20, 10, 8.0), (777, 15, 5, 6.0),
                                         (2048, 64, 16, 20.0), (300, 30, 10, 10.0),
                                         (129, 40, 24, 30.0)])
def test_hermitian_matches_oracle(n, k, p, decay):
    lam = syn.signed_spectrum(syn.spectrum("exp", n, r=decay), seed=n)
    A = syn.symmetric_matrix(n, lam, seed=n + k)
    _check(A, R.from_numpy_f(A), k, p, seed=k + p, lda=n)


def test_hermitian_ragged_lda_and_exact_rank():
    n, k, p = 900, 12, 8
    lam = syn.signed_spectrum(np.array([2.0 ** (-i / 2) for i in range(k)]), seed=1)
    A = syn.symmetric_matrix(n, lam, seed=5)
    lda = n + 13
    dA = torch.zeros(n, lda, dtype=torch.float64, device="cuda")
    dA[:, :n] = R.from_numpy_f(A)
    _check(A, dA, k, p, seed=3, lda=lda, exact_rank=True)


def test_hermitian_argument_errors():
    plan = R.Plan(100, 100, 16)
    A = torch.zeros(100, 100, dtype=torch.float64, device="cuda")
    U = torch.zeros(8, 100, dtype=torch.float64, device="cuda")
    D = torch.zeros(8, dtype=torch.float64, device="cuda")
    h = plan.handle
    assert R.rsvd_solve_hermitian(h, A, 100, 99, 8, 4, 0, U, 100, D) == -4
    assert R.rsvd_solve_hermitian(h, A, 100, 100, 0, 4, 0, U, 100, D) == -5
    assert R.rsvd_solve_hermitian(h, A, 100, 100, 8, 93, 0, U, 100, D) == -6
    assert R.rsvd_solve_hermitian(h, A, 100, 100, 8, 4, 0, U, 99, D) == -9
    assert R.rsvd_solve_hermitian(h, A, 100, 100, 8, 9, 0, U, 100, D) == 4   # l > l_max
    mplan = R.Plan(100, 100, 16, a_dtype=R.BF16, mode=R.MIXED)
    assert R.rsvd_solve_hermitian(mplan.handle, A, 100, 104, 8, 4, 0, U, 100, D) == 7


def test_hermitian_full_size():
    """A 16384 x 16384 symmetric FP64 (Haar eigenvectors, 4096 eigenvalues of
    magnitude i^-1.5 with random signs), k = 64, p = 16, seed 2."""
    n, k, p, seed = 16384, 64, 16, 2
    lam = syn.signed_spectrum(syn.spectrum("poly", 4096, alpha=1.5), seed=9)
    dA = syn.symmetric_matrix_torch(n, lam, seed=0)
    A = np.asfortranarray(dA.cpu().numpy())
    _check(A, dA, k, p, seed, lda=n)
