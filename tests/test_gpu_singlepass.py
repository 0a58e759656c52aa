"""Parity of the single-pass solve (Algorithm 6, Section 3.4.2) with the CPU
oracle through the C ABI (GPU required).

Same seeded A and the same two Gaussian test matrices (Philox streams 0 and
1 of the seed) on both sides; the plain FP64 tolerances: singular values
within 1e-10 relative, residual ||A - U S V^T||_2 within 1.0001x the
oracle's.  The GPU path forms the dominant singular vectors through
CholeskyQR2 + Jacobi and solves the joint system through its Sylvester
normal equations; the oracle uses LAPACK's SVD and eigensolver, so agreement
is about the method.
"""
import numpy as np
import pytest
import torch

from oracle import analysis
from oracle import singlepass as sp
from paper_2402_17794_gb300 import rsvd as R
from paper_2402_17794_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _compare(A, k, p, seed, lda_pad=0, exact_rank=False):
    m, n = A.shape
    lda = m + lda_pad
    dA = torch.zeros(n, lda, dtype=torch.float64, device="cuda")
    dA[:, :m] = R.from_numpy_f(A)
    ref = sp.singlepass_rsvd(A, k, p, seed)
    plan = R.Plan(m, n, k + p)
    U, S, VT = plan.solve_singlepass(dA, m, n, k, p, seed, lda=lda)
    st = plan.status()
    assert st == 0, R.rsvd_status_string(st)
    s = S.cpu().numpy()
    u, vt = R.to_numpy_f(U), R.to_numpy_f(VT)
    rel = np.abs(s - ref.S) / ref.S
    assert rel.max() <= 1e-10, rel.max()
    assert np.abs(u.T @ u - np.eye(k)).max() < 1e-12
    assert np.abs(vt @ vt.T - np.eye(k)).max() < 1e-12
    r_gpu = analysis.lowrank_residual(A, u, s, vt)
    r_orc = analysis.lowrank_residual(A, ref.U, ref.S, ref.Vt)
    if exact_rank:
        # A has rank k: both residuals are rounding (the ratio means nothing);
        # both must be at the rounding level of ||A||
        assert max(r_gpu, r_orc) <= 1e-12 * ref.S[0], (r_gpu, r_orc)
    else:
        assert r_gpu <= 1.0001 * r_orc + 1e-15 * ref.S[0], (r_gpu, r_orc)
    # same vectors up to rounding (sign convention shared)
    assert np.abs(u - ref.U).max() < 1e-7
    return rel.max()


@pytest.mark.parametrize("m,n,k,p", [(1000, 777, 20, 10), (777, 1200, 15, 5), (2048, 1024, 64, 16),
                                     (300, 300, 30, 10), (4100, 129, 40, 24)])
def test_singlepass_matches_oracle(m, n, k, p):
    A = syn.lowrank_matrix(m, n, syn.spectrum("exp", min(m, n), r=8.0), seed=m + n)
    _compare(A, k, p, seed=k + p)


def test_singlepass_ragged_lda_and_exact_rank():
    m, n, k, p = 900, 650, 12, 8
    sig = np.array([2.0 ** (-i / 2) for i in range(k)])
    A = syn.lowrank_matrix(m, n, sig, seed=5)
    _compare(A, k, p, seed=3, lda_pad=13, exact_rank=True)


def test_singlepass_argument_errors():
    plan = R.Plan(100, 80, 16)
    A = torch.zeros(80, 100, dtype=torch.float64, device="cuda")
    U = torch.zeros(8, 100, dtype=torch.float64, device="cuda")
    S = torch.zeros(8, dtype=torch.float64, device="cuda")
    VT = torch.zeros(80, 8, dtype=torch.float64, device="cuda")
    assert R.rsvd_solve_singlepass(plan.handle, A, 100, 80, 99, 8, 4, 0, U, 100, S, VT, 8) == -5
    assert R.rsvd_solve_singlepass(plan.handle, A, 100, 80, 100, 8, 9, 0, U, 100, S, VT, 8) == 4
    mplan = R.Plan(100, 80, 16, a_dtype=R.BF16, mode=R.MIXED)
    assert R.rsvd_solve_singlepass(mplan.handle, A, 100, 80, 104, 8, 4, 0, U, 100, S, VT, 8) == 7


@pytest.mark.slow
def test_singlepass_full_size():
    """The plain workload's matrix (16384 x 8192 FP64, sigma_i = i^-1.5), k=64, p=16."""
    m, n, k, p = 16384, 8192, 64, 16
    dA = syn.lowrank_matrix_torch(m, n, syn.spectrum("poly", n, alpha=1.5), seed=0)
    A = np.asfortranarray(dA.cpu().numpy().T)
    ref = sp.singlepass_rsvd(A, k, p, seed=2)
    plan = R.Plan(m, n, k + p)
    U, S, VT = plan.solve_singlepass(dA, m, n, k, p, 2)
    assert plan.status() == 0
    s = S.cpu().numpy()
    assert (np.abs(s - ref.S) / ref.S).max() <= 1e-10
    u, vt = R.to_numpy_f(U), R.to_numpy_f(VT)
    r_gpu = analysis.lowrank_residual(A, u, s, vt)
    r_orc = analysis.lowrank_residual(A, ref.U, ref.S, ref.Vt)
    assert r_gpu <= 1.0001 * r_orc + 1e-15 * ref.S[0]
