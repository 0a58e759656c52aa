"""FP64 passes over A on the tensor cores (RSVD_MODE_F64_TENSOR) through the
C ABI (GPU required).

Single passes are compared with the host's FP64 products at the mode's
worst-case bound: each output within 2^-43 K max_j|a_ij| max_j|x_jc| of the
exact value (six balanced base-256 digits per operand leave at most
2^-48 of the row and column scales per element, the dropped digit products
at most 5 * 2^-48, and the two FP32-accumulated weights less; each scale is
below twice the largest entry).  Their typical error, which the test also
reports, is far below that.  Full solves on tensor plans meet the oracle at
the plain FP64 tolerances: sigma within 1e-10 relative, residual within
1.0001x, up to the 16384 x 8192 workload the benchmark times.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import analysis
from oracle import hermitian as oh
from oracle import singlepass as osp
from paper_2402_17794_gb300 import rsvd as R
from paper_2402_17794_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

SIG_RTOL = 1e-10
RESID_RATIO = 1.0001


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _tplan(m, n, l):
    return R.Plan(m, n, l, mode=R.F64_TENSOR)


def _ok(plan):
    st = plan.status()
    assert st == 0, R.rsvd_status_string(st)


def _bound(A, X, trans):
    """Worst-case bound per output: 2^-43 K max|row of op(A)| max|column of X|."""
    Op = A.T if trans else A
    K = Op.shape[1]
    return 2.0 ** -43 * K * np.abs(Op).max(axis=1)[:, None] * np.abs(X).max(axis=0)[None, :]


@pytest.mark.parametrize("m,n,l", [(1000, 777, 37), (64, 64, 16), (130, 4097, 80),
                                   (5000, 300, 96), (3, 2, 1), (2000, 1500, 161),
                                   (4096, 2048, 80)])
def test_tensor_passes_within_bound(m, n, l):
    rng = np.random.default_rng(m * 5 + n + l)
    A = np.asfortranarray(rng.standard_normal((m, n)))
    # rows of very different scale: the per-row exponent must follow them
    A *= np.exp2(rng.integers(-30, 31, size=m))[:, None]
    lda = m + 3
    dA = R.colmajor(m, n, ld=lda, zero=True)
    dA[:, :m] = torch.from_numpy(A.T.copy()).cuda()
    plan = _tplan(m, n, l)
    X = np.asfortranarray(rng.standard_normal((n, l)))
    Y = R.colmajor(m, l)
    assert R.rsvd_apply_a(plan.handle, dA, m, n, lda, R.from_numpy_f(X), n, l, Y, m) == 0
    Xt = np.asfortranarray(rng.standard_normal((m, l)) * np.exp2(rng.integers(-8, 9, size=l)))
    Z = R.colmajor(n, l)
    assert R.rsvd_apply_at(plan.handle, dA, m, n, lda, R.from_numpy_f(Xt), m, l, Z, n) == 0
    _ok(plan)
    ey = np.abs(R.to_numpy_f(Y) - A @ X)
    ez = np.abs(R.to_numpy_f(Z) - A.T @ Xt)
    assert np.isfinite(ey).all() and np.isfinite(ez).all()
    by, bz = _bound(A, X, False), _bound(A, Xt, True)
    assert (ey <= by).all(), (ey / by).max()
    assert (ez <= bz).all(), (ez / bz).max()
    # well inside the worst case (random-sign digit errors; rows of very
    # different scale put the A^T pass closest to it)
    assert (ey / by).max() < 0.5 and (ez / bz).max() < 0.5, ((ey / by).max(), (ez / bz).max())


def test_tensor_pass_zero_and_exact_inputs():
    """Zero rows and columns give exact zeros; small integers are exact."""
    m, n, l = 300, 200, 24
    rng = np.random.default_rng(3)
    A = rng.integers(-100, 101, size=(m, n)).astype(np.float64)
    A[5] = 0.0
    A[:, 7] = 0.0
    X = rng.integers(-50, 51, size=(n, l)).astype(np.float64)
    plan = _tplan(m, n, l)
    Y = R.colmajor(m, l)
    assert R.rsvd_apply_a(plan.handle, R.from_numpy_f(A), m, n, m, R.from_numpy_f(X), n, l, Y,
                          m) == 0
    _ok(plan)
    got = R.to_numpy_f(Y)
    np.testing.assert_array_equal(got, A @ X)
    assert (got[5] == 0).all()


def _solve_compare(A, k, p, q, seed, lda_pad=0):
    m, n = A.shape
    ref = oracle.rsvd(A, k, p, q, seed)
    plan = _tplan(m, n, k + p)
    lda = m + lda_pad
    dA = R.colmajor(m, n, ld=lda, zero=True)
    dA[:, :m] = torch.from_numpy(np.ascontiguousarray(A.T)).cuda()
    U, S, VT = plan.solve(dA, m, n, k, p, q, seed, lda=lda)
    _ok(plan)
    s = S.cpu().numpy()
    u, vt = R.to_numpy_f(U), R.to_numpy_f(VT)
    rel = np.abs(s - ref.S) / ref.S
    assert rel.max() <= SIG_RTOL, rel.max()
    assert np.abs(u.T @ u - np.eye(k)).max() < 1e-12
    r_gpu = analysis.lowrank_residual(A, u, s, vt)
    r_orc = analysis.lowrank_residual(A, ref.U, ref.S, ref.Vt)
    assert r_gpu <= RESID_RATIO * r_orc + 1e-15 * ref.S[0], (r_gpu, r_orc)
    return rel.max()


def test_tensor_solve_config_small():
    """1024 x 512, Haar factors, sigma_i = 2^(-i/4), k=20, p=10, q=0."""
    A = syn.lowrank_matrix(1024, 512, syn.spectrum("geometric4", 512), seed=0)
    _solve_compare(A, 20, 10, 0, seed=2)


@pytest.mark.parametrize("m,n,k,p,q", [(1000, 700, 15, 10, 2), (300, 900, 25, 5, 1),
                                       (2048, 1024, 64, 16, 2), (600, 600, 100, 60, 1)])
def test_tensor_solve_ragged(m, n, k, p, q):
    r = min(m, n)
    A = syn.lowrank_matrix(m, n, syn.spectrum("poly", r, alpha=1.5), seed=m + n)
    _solve_compare(A, k, p, q, seed=k * 31 + p, lda_pad=5)


def test_tensor_plan_other_algorithms():
    """Algorithms 3, 5 and 6 on a tensor plan meet their oracles."""
    m, n, k, p = 1500, 900, 20, 10
    A = syn.lowrank_matrix(m, n, syn.spectrum("exp", n, r=8.0), seed=21)
    dA = R.from_numpy_f(A)
    plan = _tplan(m, n, k + p)
    # Algorithm 6
    ref6 = osp.singlepass_rsvd(A, k, p, 4)
    U, S, VT = plan.solve_singlepass(dA, m, n, k, p, 4)
    _ok(plan)
    assert (np.abs(S.cpu().numpy() - ref6.S) / ref6.S).max() <= SIG_RTOL
    # Algorithm 3: its sample holds direction i at relative size
    # (sigma_i/sigma_1)^3 (q = 1), so a pass error of ~1e-13 of the scale moves
    # sigma_i by ~1e-13 (sigma_1/sigma_i)^3 relative
    ref3 = oracle.rsvd(A, k, p, 1, 4, algorithm=3)
    U, S, VT = plan.solve_algorithm(3, dA, m, n, k, p, 1, 4)
    _ok(plan)
    rel3 = np.abs(S.cpu().numpy() - ref3.S) / ref3.S
    tol3 = np.maximum(SIG_RTOL, 1e-13 * (ref3.S[0] / ref3.S) ** 3)
    assert np.all(rel3 <= tol3), (rel3 / tol3).max()
    # Algorithm 5 (symmetric input)
    nn = 900
    lam = syn.signed_spectrum(syn.spectrum("exp", nn, r=8.0), seed=2)
    B = syn.symmetric_matrix(nn, lam, seed=3)
    ref5 = oh.hermitian_singlepass(B, k, p, 6)
    hplan = _tplan(nn, nn, k + p)
    Uh, D = hplan.solve_hermitian(R.from_numpy_f(B), nn, k, p, 6)
    _ok(hplan)
    d = D.cpu().numpy()
    # relative on the eigenvalues the single pass resolves; the method's tiny
    # trailing estimates (here 3.6e-5 against 0.9) are held absolutely
    big = np.abs(ref5.D) >= 1e-3 * np.abs(ref5.D[0])
    assert (np.abs(d - ref5.D)[big] / np.abs(ref5.D[big])).max() <= SIG_RTOL
    assert np.abs(d - ref5.D).max() <= SIG_RTOL * np.abs(ref5.D[0])


def test_tensor_wait_limit_expires_and_recovers():
    """The tensor pass's bounded waits: a limit of a few cycles expires,
    RSVD_ERR_TIMEOUT is reported, and the plan then solves correctly."""
    m, n, l = 2048, 1024, 40
    rng = np.random.default_rng(9)
    A = np.asfortranarray(rng.standard_normal((m, n)))
    plan = _tplan(m, n, l)
    X = R.from_numpy_f(rng.standard_normal((n, l)))
    Y = R.colmajor(m, l)
    assert R.rsvd_plan_set_wait_limit(plan.handle, 8) == 0
    assert R.rsvd_apply_a(plan.handle, R.from_numpy_f(A), m, n, m, X, n, l, Y, m) == 0
    assert plan.status() == 3
    assert R.rsvd_plan_set_wait_limit(plan.handle, 0) == 0
    B = syn.lowrank_matrix(m, n, syn.spectrum("poly", n, alpha=1.5), seed=8)
    ref = oracle.rsvd(B, 30, 10, 1, 5)
    U, S, VT = plan.solve(R.from_numpy_f(B), m, n, 30, 10, 1, 5)
    _ok(plan)
    assert (np.abs(S.cpu().numpy() - ref.S) / ref.S).max() <= SIG_RTOL


def test_tensor_solve_full_size():
    """16384 x 8192 FP64, Haar factors, sigma_i = i^-1.5, k=64, p=16, q=2 (the
    benchmark's workload): full-size parity at the plain FP64 tolerances."""
    m, n, k, p, q = 16384, 8192, 64, 16, 2
    dA = syn.lowrank_matrix_torch(m, n, syn.spectrum("poly", n, alpha=1.5), seed=0)
    A = np.asfortranarray(dA.cpu().numpy().T)
    ref = oracle.rsvd(A, k, p, q, seed=2)
    plan = _tplan(m, n, k + p)
    U, S, VT = plan.solve(dA, m, n, k, p, q, 2)
    _ok(plan)
    s = S.cpu().numpy()
    rel = np.abs(s - ref.S) / ref.S
    assert rel.max() <= SIG_RTOL, rel.max()
    u, vt = R.to_numpy_f(U), R.to_numpy_f(VT)
    r_gpu = analysis.lowrank_residual(A, u, s, vt)
    r_orc = analysis.lowrank_residual(A, ref.U, ref.S, ref.Vt)
    assert r_gpu <= RESID_RATIO * r_orc, (r_gpu, r_orc)


def test_prepared_matrix_is_reused_and_released():
    """rsvd_plan_prepare_a keeps A's digit slices: passes on the prepared
    matrix equal the unprepared ones bitwise; a pass on another matrix
    replaces them; after release the first matrix is prepared again."""
    m, n, l = 1500, 1100, 48
    rng = np.random.default_rng(5)
    A = R.from_numpy_f(rng.standard_normal((m, n)))
    B = R.from_numpy_f(rng.standard_normal((m, n)))
    X = R.from_numpy_f(rng.standard_normal((n, l)))
    plan = _tplan(m, n, l)
    Y0, Y1, Y2, Y3 = (R.colmajor(m, l) for _ in range(4))
    assert R.rsvd_apply_a(plan.handle, A, m, n, m, X, n, l, Y0, m) == 0
    assert R.rsvd_plan_prepare_a(plan.handle, A, m, n, m) == 0
    assert R.rsvd_apply_a(plan.handle, A, m, n, m, X, n, l, Y1, m) == 0
    assert R.rsvd_apply_a(plan.handle, B, m, n, m, X, n, l, Y2, m) == 0
    assert R.rsvd_plan_release_a(plan.handle) == 0
    assert R.rsvd_apply_a(plan.handle, A, m, n, m, X, n, l, Y3, m) == 0
    _ok(plan)
    assert torch.equal(Y0, Y1) and torch.equal(Y0, Y3)
    ref_b = R.to_numpy_f(B) @ R.to_numpy_f(X)
    assert np.abs(R.to_numpy_f(Y2) - ref_b).max() <= 1e-9
    assert R.rsvd_plan_prepare_a(plan.handle, A, m, n, m - 1) == -5
    # plain plans accept and ignore it
    pplan = R.Plan(m, n, l)
    assert R.rsvd_plan_prepare_a(pplan.handle, A, m, n, m) == 0
    assert R.rsvd_plan_release_a(pplan.handle) == 0
