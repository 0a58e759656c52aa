"""Parity of the plain FP64 CUDA path with the CPU oracle, step by step and
end to end, through the C ABI (GPU required).

Tolerances (plain FP64 form): singular values within 1e-10 relative of the
oracle's, residual ||A - U S V^T||_2 within 1.0001x the oracle's; per-step
products within a few hundred ulps of the magnitude |A||X| they sum.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import analysis
from oracle.philox import gaussian_matrix
from paper_2402_17794_gb300 import rsvd as R
from paper_2402_17794_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

SIG_RTOL = 1e-10
RESID_RATIO = 1.0001


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _plan(m, n, l):
    return R.Plan(m, n, l)


def _ok(plan):
    st = plan.status()
    assert st == 0, R.rsvd_status_string(st)


@pytest.mark.parametrize("n,l,seed", [(1000, 37, 3), (512, 30, 2), (8192, 80, 2**40 + 7),
                                      (33, 1, 0)])
def test_gaussian_matches_oracle(n, l, seed):
    plan = _plan(n, n, min(l, 288))
    out = R.colmajor(n, l)
    assert R.rsvd_gaussian(plan.handle, n, l, seed, 0, R.F64, out, n) == 0
    _ok(plan)
    got = R.to_numpy_f(out)
    ref = gaussian_matrix(n, l, seed)
    np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-14)
    # BF16 output rounds the same value (ties may round apart by one ulp)
    out16 = R.colmajor(n, l, dtype=torch.bfloat16)
    assert R.rsvd_gaussian(plan.handle, n, l, seed, 0, R.BF16, out16, n) == 0
    _ok(plan)
    g16 = R.to_numpy_f(out16)
    r16 = syn.bf16_round(ref)
    assert np.mean(g16 == r16) > 0.999
    np.testing.assert_allclose(g16, r16, rtol=2 ** -7, atol=0)


@pytest.mark.parametrize("m,n,l", [(1000, 777, 37), (64, 64, 16), (130, 4097, 80),
                                   (5000, 300, 96), (3, 2, 1), (2000, 1500, 150)])
def test_apply_a_and_at_match_products(m, n, l):
    rng = np.random.default_rng(m * 7 + n)
    A = np.asfortranarray(rng.standard_normal((m, n)))
    lda = m + 3
    dA = R.colmajor(m, n, ld=lda, zero=True)
    dA[:, :m] = torch.from_numpy(A.T.copy()).cuda()
    plan = _plan(m, n, l)
    X = np.asfortranarray(rng.standard_normal((n, l)))
    Y = R.colmajor(m, l)
    assert R.rsvd_apply_a(plan.handle, dA, m, n, lda, R.from_numpy_f(X), n, l, Y, m) == 0
    Xt = np.asfortranarray(rng.standard_normal((m, l)))
    Z = R.colmajor(n, l)
    assert R.rsvd_apply_at(plan.handle, dA, m, n, lda, R.from_numpy_f(Xt), m, l, Z, n) == 0
    _ok(plan)
    ref_y = A @ X
    ref_z = A.T @ Xt
    tol_y = 64 * 2.0 ** -52 * (np.abs(A) @ np.abs(X)).max()
    tol_z = 64 * 2.0 ** -52 * (np.abs(A.T) @ np.abs(Xt)).max()
    assert np.abs(R.to_numpy_f(Y) - ref_y).max() <= tol_y
    assert np.abs(R.to_numpy_f(Z) - ref_z).max() <= tol_z


@pytest.mark.parametrize("rows,l,cond", [(5000, 80, 1e3), (777, 37, 1e6), (300, 288, 10.0),
                                         (64, 1, 1.0)])
def test_orth_is_cholesky_qr(rows, l, cond):
    rng = np.random.default_rng(rows + l)
    U = np.linalg.qr(rng.standard_normal((rows, l)))[0]
    V = np.linalg.qr(rng.standard_normal((l, l)))[0]
    Y = np.asfortranarray((U * np.geomspace(1, 1 / cond, l)) @ V.T)
    plan = _plan(rows, rows, l)
    Q = R.colmajor(rows, l)
    Rm = R.colmajor(l, l)
    assert R.rsvd_orth(plan.handle, R.from_numpy_f(Y), rows, l, rows, Q, rows, Rm, l) == 0
    _ok(plan)
    q = R.to_numpy_f(Q)
    r = R.to_numpy_f(Rm)
    assert np.abs(q.T @ q - np.eye(l)).max() < 1e-13
    assert np.abs(np.tril(r, -1)).max() == 0.0
    assert np.abs(q @ r - Y).max() < 1e-13 * np.abs(Y).max() * np.sqrt(l)
    ref_q = oracle.orth(Y)
    assert analysis.sin_canonical_angles(ref_q, q).max() < 1e-12 * cond


def test_orth_drops_dependent_columns():
    rng = np.random.default_rng(5)
    rows, l = 400, 12
    Y = rng.standard_normal((rows, l))
    Y[:, 5] = Y[:, 1] - 2 * Y[:, 3]      # exactly dependent
    Y[:, 9] = 0.0
    Y = np.asfortranarray(Y)
    plan = _plan(rows, rows, l)
    Q = R.colmajor(rows, l)
    assert R.rsvd_orth(plan.handle, R.from_numpy_f(Y), rows, l, rows, Q, rows) == 0
    _ok(plan)
    q = R.to_numpy_f(Q)
    norms = np.linalg.norm(q, axis=0)
    assert norms[5] < 1e-6 and norms[9] == 0.0
    keep = [j for j in range(l) if j not in (5, 9)]
    qk = q[:, keep]
    assert np.abs(qk.T @ qk - np.eye(len(keep))).max() < 1e-12
    # range(Y) is still spanned
    assert np.abs(Y - qk @ (qk.T @ Y)).max() < 1e-11 * np.abs(Y).max()


@pytest.mark.parametrize("l,cond", [(30, 1e2), (80, 1e6), (160, 1e3), (7, 1.0), (288, 1e4)])
def test_small_svd_one_sided_jacobi(l, cond):
    rng = np.random.default_rng(l)
    U = np.linalg.qr(rng.standard_normal((l, l)))[0]
    V = np.linalg.qr(rng.standard_normal((l, l)))[0]
    sig = np.geomspace(1, 1 / cond, l)
    M = np.asfortranarray((U * sig) @ V.T)
    plan = _plan(l, l, l)
    s = torch.empty(l, dtype=torch.float64, device="cuda")
    Um = R.colmajor(l, l)
    Vm = R.colmajor(l, l)
    assert R.rsvd_small_svd(plan.handle, R.from_numpy_f(M), l, l, s, Um, l, Vm, l) == 0
    _ok(plan)
    s = s.cpu().numpy()
    # the stored M carries rounding of ~eps*sigma_1, so compare against its
    # exact spectrum to that absolute level
    np.testing.assert_allclose(s, np.linalg.svd(M, compute_uv=False), rtol=1e-13,
                               atol=1e-14 * np.sqrt(l))
    np.testing.assert_allclose(s, sig, rtol=1e-13, atol=1e-14 * np.sqrt(l))
    um, vm = R.to_numpy_f(Um), R.to_numpy_f(Vm)
    assert np.abs(um.T @ um - np.eye(l)).max() < 1e-12
    assert np.abs(vm.T @ vm - np.eye(l)).max() < 1e-12
    assert np.abs((um * s) @ vm.T - M).max() < 1e-13 * np.sqrt(l)


def _solve_and_compare(A, k, p, q, seed, lda_pad=0, exact_resid=True):
    m, n = A.shape
    ref = oracle.rsvd(A, k, p, q, seed)
    plan = _plan(m, n, k + p)
    lda = m + lda_pad
    dA = R.colmajor(m, n, ld=lda, zero=True)
    dA[:, :m] = torch.from_numpy(np.ascontiguousarray(A.T)).cuda()
    U, S, VT = plan.solve(dA, m, n, k, p, q, seed, lda=lda)
    _ok(plan)
    s = S.cpu().numpy()
    u = R.to_numpy_f(U)
    vt = R.to_numpy_f(VT)
    rel = np.abs(s - ref.S) / ref.S
    assert rel.max() <= SIG_RTOL, rel.max()
    assert np.abs(u.T @ u - np.eye(k)).max() < 1e-12
    assert np.abs(vt @ vt.T - np.eye(k)).max() < 1e-12
    # element-wise vectors where the singular values are well separated
    gaps = np.minimum(np.abs(np.diff(np.r_[np.inf, ref.S])), np.abs(np.diff(np.r_[ref.S, 0.0])))
    sep = gaps / ref.S[0] > 1e-4
    assert np.abs(u[:, sep] - ref.U[:, sep]).max() < 1e-7
    assert np.abs(vt[sep] - ref.Vt[sep]).max() < 1e-7
    if exact_resid:
        r_gpu = analysis.lowrank_residual(A, u, s, vt)
        r_orc = analysis.lowrank_residual(A, ref.U, ref.S, ref.Vt)
        assert r_gpu <= RESID_RATIO * r_orc + 1e-15 * ref.S[0], (r_gpu, r_orc)
    return s, ref


def test_solve_config_small_fp64():
    """1024 x 512, Haar factors, sigma_i = 2^(-i/4), k=20, p=10, q=0."""
    m, n = 1024, 512
    A = syn.lowrank_matrix(m, n, syn.spectrum("geometric4", n), seed=0)
    _solve_and_compare(A, 20, 10, 0, seed=2)


@pytest.mark.parametrize("m,n,k,p,q", [(1000, 700, 15, 10, 2), (300, 900, 25, 5, 1),
                                       (777, 555, 33, 0, 3), (129, 65, 1, 1, 1),
                                       (2048, 1024, 64, 16, 2), (600, 600, 100, 60, 1)])
def test_solve_ragged_shapes(m, n, k, p, q):
    r = min(m, n)
    A = syn.lowrank_matrix(m, n, syn.spectrum("poly", r, alpha=1.5), seed=m + n)
    _solve_and_compare(A, k, p, q, seed=k * 31 + p, lda_pad=5)


def test_solve_exact_rank_deficient():
    """rank(A) = 10 < k + p: top-10 triplets exact, rest near zero."""
    m, n, r = 500, 300, 10
    sig = syn.spectrum("geometric4", r) * 2
    A = syn.lowrank_matrix(m, n, sig, seed=4)
    plan = _plan(m, n, 16)
    U, S, VT = plan.solve(R.from_numpy_f(A), m, n, 10, 6, 1, 9)
    _ok(plan)
    np.testing.assert_allclose(S.cpu().numpy(), sig, rtol=1e-12)
    resid = analysis.lowrank_residual(A, R.to_numpy_f(U), S.cpu().numpy(), R.to_numpy_f(VT))
    assert resid < 1e-13 * sig[0]


def test_solve_controlled_gap_eq41():
    """Section 4.3 setting: 3000 x 300, gap = 2, k = 25, p = 5, q = 2."""
    A = syn.controlled_gap(3000, 300, gap=2.0, seed=6)
    _solve_and_compare(A, 25, 5, 2, seed=17)


def test_nonfinite_input_reports_status():
    m, n = 200, 100
    A = syn.lowrank_matrix(m, n, syn.spectrum("poly", n), seed=1)
    A[17, 33] = np.nan
    plan = _plan(m, n, 12)
    plan.solve(R.from_numpy_f(A), m, n, 8, 4, 1, 3)
    assert plan.status() == 6
    # the plan recovers for the next solve
    A[17, 33] = 0.5
    plan.solve(R.from_numpy_f(A), m, n, 8, 4, 1, 3)
    assert plan.status() == 0


def test_invalid_arguments_are_rejected():
    plan = _plan(100, 80, 20)
    A = R.colmajor(100, 80, zero=True)
    U = R.colmajor(100, 10)
    S = torch.empty(10, dtype=torch.float64, device="cuda")
    VT = R.colmajor(10, 80)
    assert R.rsvd_solve(plan.handle, A, 100, 80, 100, 0, 5, 1, 0, U, 100, S, VT, 10) == -6
    assert R.rsvd_solve(plan.handle, A, 100, 80, 99, 5, 5, 1, 0, U, 100, S, VT, 10) == -5
    assert R.rsvd_solve(plan.handle, A, 100, 80, 100, 5, -1, 1, 0, U, 100, S, VT, 10) == -7
    assert R.rsvd_solve(plan.handle, A, 100, 80, 100, 5, 5, 1, 0, U, 100, S, VT, 4) == -14
    assert R.rsvd_solve(plan.handle, A, 100, 80, 100, 15, 10, 1, 0, U, 100, S, VT, 15) == 4
    assert R.rsvd_solve(plan.handle, A, 200, 80, 200, 5, 5, 1, 0, U, 200, S, VT, 5) == 4


def test_repeat_solves_are_bitwise_deterministic():
    m, n = 900, 400
    A = R.from_numpy_f(syn.lowrank_matrix(m, n, syn.spectrum("poly", n), seed=3))
    plan = _plan(m, n, 40)
    a = [t.clone() for t in plan.solve(A, m, n, 30, 10, 2, 77)]
    b = plan.solve(A, m, n, 30, 10, 2, 77)
    _ok(plan)
    for x, y in zip(a, b):
        assert torch.equal(x, y)


@pytest.mark.slow
def test_solve_config_full_size_fp64():
    """16384 x 8192 FP64, Haar factors, sigma_i = i^-1.5, k=64, p=16, q=2:
    full-size parity with the oracle in the launch configuration the
    benchmark times (residual compared through the Lanczos estimator)."""
    m, n, k, p, q = 16384, 8192, 64, 16, 2
    dA = syn.lowrank_matrix_torch(m, n, syn.spectrum("poly", n, alpha=1.5), seed=0)
    A = dA.cpu().numpy().T
    A = np.asfortranarray(A)
    ref = oracle.rsvd(A, k, p, q, seed=2)
    plan = _plan(m, n, k + p)
    U, S, VT = plan.solve(dA, m, n, k, p, q, 2)
    _ok(plan)
    s = S.cpu().numpy()
    rel = np.abs(s - ref.S) / ref.S
    assert rel.max() <= SIG_RTOL, rel.max()
    u, vt = R.to_numpy_f(U), R.to_numpy_f(VT)
    r_gpu = analysis.lowrank_residual(A, u, s, vt)
    r_orc = analysis.lowrank_residual(A, ref.U, ref.S, ref.Vt)
    assert r_gpu <= RESID_RATIO * r_orc, (r_gpu, r_orc)
