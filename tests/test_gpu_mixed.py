"""Parity of the mixed-precision path (BF16 A on tcgen05 tensor cores, FP32
elsewhere) with the CPU oracle, through the C ABI (GPU required).

The oracle runs in FP64 on the stored (BF16-rounded, exactly dequantised) A
with the same Omega and the same number of power steps as the mixed path
(q BF16 steps plus its refinement step = q + 1).  Tolerances (mixed form):
singular values within 1e-3 relative, residual within 1.05x the oracle's.
Single passes over A are compared with FP64 products of the same BF16
inputs; FP32 accumulation bounds their error by ~K 2^-24 |A||X| (checked at
2e-6 relative to max |A||X|, far above the ~5e-8 seen, far below any layout
mistake).
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import analysis
from paper_2402_17794_gb300 import rsvd as R
from paper_2402_17794_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

SIG_RTOL = 1e-3
RESID_RATIO = 1.05


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _bf16_matrix(A, lda=None):
    """Device BF16 column-major copy (n, lda) and the exact FP64 dequantised A."""
    m, n = A.shape
    lda = lda or m
    t = torch.zeros(n, lda, dtype=torch.bfloat16, device="cuda")
    t[:, :m] = torch.from_numpy(np.ascontiguousarray(A.T)).to(torch.float32).to(torch.bfloat16).cuda()
    A16 = np.asfortranarray(t[:, :m].float().cpu().numpy().T.astype(np.float64))
    return t, A16


def _ok(plan):
    st = plan.status()
    assert st == 0, R.rsvd_status_string(st)


@pytest.mark.parametrize("m,n,l", [(256, 128, 16), (1000, 777, 37), (3000, 2000, 160),
                                   (4096, 640, 256), (129, 4100, 80), (8, 8, 1),
                                   (20000, 300, 48)])
@pytest.mark.parametrize("ax", [True, False])
def test_tcgen05_pass_matches_fp64_product(m, n, l, ax):
    rng = np.random.default_rng(m * 3 + n + l)
    lda = (m + 7) // 8 * 8 + (8 if m % 3 == 0 else 0)
    dA, A16 = _bf16_matrix(rng.standard_normal((m, n)), lda)
    rows = n if ax else m
    ldx = (rows + 7) // 8 * 8
    X = rng.standard_normal((rows, l))
    dX = torch.zeros(l, ldx, dtype=torch.bfloat16, device="cuda")
    dX[:, :rows] = torch.from_numpy(X.T.copy()).float().to(torch.bfloat16).cuda()
    X16 = dX[:, :rows].float().cpu().numpy().T.astype(np.float64)
    plan = R.Plan(m, n, max(l, 1), a_dtype=R.BF16, mode=R.MIXED)
    out_rows = m if ax else n
    Y = torch.full((l, out_rows), float("nan"), dtype=torch.float32, device="cuda")
    f = R.rsvd_apply_a if ax else R.rsvd_apply_at
    assert f(plan.handle, dA, m, n, lda, dX, ldx, l, Y, out_rows) == 0
    _ok(plan)
    got = Y.cpu().numpy().T.astype(np.float64)
    ref = A16 @ X16 if ax else A16.T @ X16
    mag = (np.abs(A16) @ np.abs(X16) if ax else np.abs(A16.T) @ np.abs(X16)).max()
    assert np.isfinite(got).all()
    assert np.abs(got - ref).max() <= 2e-6 * mag


def test_tcgen05_rejects_unaligned_leading_dimension():
    plan = R.Plan(100, 64, 16, a_dtype=R.BF16, mode=R.MIXED)
    A = torch.zeros(64, 101, dtype=torch.bfloat16, device="cuda")
    X = torch.zeros(16, 64, dtype=torch.bfloat16, device="cuda")
    Y = torch.zeros(16, 100, dtype=torch.float32, device="cuda")
    assert R.rsvd_apply_a(plan.handle, A, 100, 64, 101, X, 64, 16, Y, 100) == 7


def _mixed_solve_and_compare(A, k, p, q, seed, lda_pad=0):
    m, n = A.shape
    lda = (m + 7) // 8 * 8 + lda_pad
    dA, A16 = _bf16_matrix(A, lda)
    ref = oracle.rsvd(A16, k, p, q + 1, seed)
    plan = R.Plan(m, n, k + p, a_dtype=R.BF16, mode=R.MIXED)
    U, S, VT = plan.solve(dA, m, n, k, p, q, seed, lda=lda)
    _ok(plan)
    s = S.cpu().numpy()
    u = R.to_numpy_f(U)
    vt = R.to_numpy_f(VT)
    rel = np.abs(s - ref.S) / ref.S
    assert rel.max() <= SIG_RTOL, rel.max()
    assert np.abs(u.T @ u - np.eye(k)).max() < 1e-4
    assert np.abs(vt @ vt.T - np.eye(k)).max() < 1e-4
    r_gpu = analysis.lowrank_residual(A16, u, s, vt)
    r_orc = analysis.lowrank_residual(A16, ref.U, ref.S, ref.Vt)
    assert r_gpu <= RESID_RATIO * r_orc, (r_gpu, r_orc)
    return rel.max(), r_gpu / r_orc


def test_mixed_solve_exp_spectrum_with_noise():
    """Scaled-down mixed workload: sigma_i = exp(-i/40) + 1e-4 noise floor."""
    m, n = 4096, 2048
    A = syn.lowrank_matrix(m, n, syn.spectrum("exp", 640, r=40.0), seed=3, noise_2norm=1e-4)
    _mixed_solve_and_compare(A, 64, 16, 2, seed=5)


@pytest.mark.parametrize("m,n,k,p,q", [(1000, 777, 20, 10, 1), (777, 1200, 15, 5, 0),
                                       (2048, 1024, 128, 32, 3), (512, 512, 200, 56, 1)])
def test_mixed_solve_ragged(m, n, k, p, q):
    r = min(m, n)
    A = syn.lowrank_matrix(m, n, syn.spectrum("poly", r, alpha=1.0), seed=m + 2 * n)
    _mixed_solve_and_compare(A, k, p, q, seed=k + p + q, lda_pad=8)


def test_mixed_solve_is_deterministic():
    m, n = 3000, 1500
    A = syn.lowrank_matrix(m, n, syn.spectrum("exp", 400, r=30.0), seed=9)
    dA, _ = _bf16_matrix(A)
    plan = R.Plan(m, n, 48, a_dtype=R.BF16, mode=R.MIXED)
    a = [t.clone() for t in plan.solve(dA, m, n, 32, 16, 2, 11)]
    b = plan.solve(dA, m, n, 32, 16, 2, 11)
    _ok(plan)
    for x, y in zip(a, b):
        assert torch.equal(x, y)


@pytest.mark.slow
def test_mixed_solve_full_size_bf16():
    """A 65536 x 16384 BF16, sigma_i = exp(-i/40) + 1e-4 noise, k=128, p=32,
    q=3: full-size parity with the FP64 oracle on the dequantised A."""
    m, n, k, p, q = 65536, 16384, 128, 32, 3
    sig = syn.spectrum("exp", 640, r=40.0)
    dA = syn.lowrank_matrix_torch(m, n, sig, seed=0, dtype=torch.bfloat16,
                                  factor_dtype=torch.float32, noise_2norm=1e-4)
    A16 = np.asfortranarray(dA.float().cpu().numpy().T.astype(np.float64))
    ref = oracle.rsvd(A16, k, p, q + 1, seed=2)
    plan = R.Plan(m, n, k + p, a_dtype=R.BF16, mode=R.MIXED)
    U, S, VT = plan.solve(dA, m, n, k, p, q, 2)
    _ok(plan)
    s = S.cpu().numpy()
    rel = np.abs(s - ref.S) / ref.S
    assert rel.max() <= SIG_RTOL, rel.max()
    u, vt = R.to_numpy_f(U), R.to_numpy_f(VT)
    r_gpu = analysis.lowrank_residual(A16, u, s, vt)
    r_orc = analysis.lowrank_residual(A16, ref.U, ref.S, ref.Vt)
    assert r_gpu <= RESID_RATIO * r_orc, (r_gpu, r_orc)


@pytest.mark.parametrize("ax", [True, False])
def test_bounded_wait_expires_and_plan_recovers(ax):
    """Failure detection without a GPU fault: a wait limit of a few cycles
    makes the first incomplete pipeline wait of a tensor-core pass expire.
    The pass drains what it issued, frees its tensor memory and reports
    RSVD_ERR_TIMEOUT through rsvd_plan_status(); with the default limit
    restored, a full solve on the same plan meets the oracle."""
    m, n, l = 4096, 2048, 48
    rng = np.random.default_rng(17)
    dA, _ = _bf16_matrix(rng.standard_normal((m, n)))
    rows = n if ax else m
    dX = torch.from_numpy(rng.standard_normal((l, rows))).to(torch.bfloat16).cuda()
    out_rows = m if ax else n
    Y = torch.zeros(l, out_rows, dtype=torch.float32, device="cuda")
    plan = R.Plan(m, n, l, a_dtype=R.BF16, mode=R.MIXED)
    assert R.rsvd_plan_set_wait_limit(plan.handle, -1) == -2
    assert R.rsvd_plan_set_wait_limit(plan.handle, 8) == 0
    f = R.rsvd_apply_a if ax else R.rsvd_apply_at
    assert f(plan.handle, dA, m, n, m, dX, rows, l, Y, out_rows) == 0
    assert plan.status() == 3          # RSVD_ERR_TIMEOUT
    assert plan.status() == 0          # reading the status clears it
    assert R.rsvd_plan_set_wait_limit(plan.handle, 0) == 0
    A = syn.lowrank_matrix(m, n, syn.spectrum("exp", 400, r=30.0), seed=21)
    dA2, A16 = _bf16_matrix(A)
    k, p, q, seed = 32, 16, 1, 4
    ref = oracle.rsvd(A16, k, p, q + 1, seed)
    U, S, VT = plan.solve(dA2, m, n, k, p, q, seed)
    _ok(plan)
    rel = np.abs(S.cpu().numpy() - ref.S) / ref.S
    assert rel.max() <= SIG_RTOL, rel.max()
