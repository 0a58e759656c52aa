"""Parity of the FP8 form of the mixed path (A stored as E4M3 codes with one
power-of-two FP32 scale per 128 x 128 tile) through the C ABI (GPU required).

The oracle runs on the exactly dequantised A (code value times tile scale,
in FP64), so the comparison checks the computation, not the quantisation.
Single passes are compared with FP64 products of the same inputs: the
converted operand is exact in BF16 and FP32 accumulation bounds the error by
~K 2^-24 |A||X| (checked at 2e-6 of max |A||X|).  Solves: singular values
within 1e-3 relative and residual within 1.05x the oracle's (the mixed form's
tolerances).
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import analysis, fp8
from paper_2402_17794_gb300 import rsvd as R
from paper_2402_17794_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

SIG_RTOL = 1e-3
RESID_RATIO = 1.05


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _fp8_matrix(A, lda=None, spread_scales=False):
    """Device codes (n, lda) uint8, device scales (n_tiles, m_tiles), and the
    exact FP64 dequantised A."""
    m, n = A.shape
    at = torch.from_numpy(np.ascontiguousarray(A.T))
    if spread_scales:   # tiles of very different magnitude
        rng = np.random.default_rng(m + n)
        for J in range((n + 127) // 128):
            for I in range((m + 127) // 128):
                at[J * 128:(J + 1) * 128, I * 128:(I + 1) * 128] *= float(2.0 ** rng.integers(-6, 7))
    codes, scales = syn.quantize_e4m3_tiles(at, m, lda)
    Aq = fp8.dequantize_tiles(codes.numpy(), scales.numpy().T, m, n, columns_as_rows=True)
    return codes.cuda(), scales.cuda(), np.asfortranarray(Aq)


def _ok(plan):
    st = plan.status()
    assert st == 0, R.rsvd_status_string(st)


@pytest.mark.parametrize("m,n,l", [(256, 128, 16), (1000, 777, 37), (3000, 2000, 160),
                                   (4096, 640, 256), (129, 4100, 80), (20000, 300, 48)])
@pytest.mark.parametrize("ax", [True, False])
def test_fp8_pass_matches_fp64_product(m, n, l, ax):
    rng = np.random.default_rng(m * 5 + n + l)
    lda = (m + 15) // 16 * 16 + (16 if m % 3 == 0 else 0)
    dA, dS, Aq = _fp8_matrix(rng.standard_normal((m, n)), lda, spread_scales=True)
    rows = n if ax else m
    ldx = (rows + 7) // 8 * 8
    X = rng.standard_normal((rows, l))
    dX = torch.zeros(l, ldx, dtype=torch.bfloat16, device="cuda")
    dX[:, :rows] = torch.from_numpy(X.T.copy()).float().to(torch.bfloat16).cuda()
    X16 = dX[:, :rows].float().cpu().numpy().T.astype(np.float64)
    plan = R.Plan(m, n, max(l, 1), a_dtype=R.FP8E4M3, mode=R.MIXED)
    plan.set_tile_scales(dS)
    out_rows = m if ax else n
    Y = torch.full((l, out_rows), float("nan"), dtype=torch.float32, device="cuda")
    f = R.rsvd_apply_a if ax else R.rsvd_apply_at
    assert f(plan.handle, dA, m, n, lda, dX, ldx, l, Y, out_rows) == 0
    _ok(plan)
    got = Y.cpu().numpy().T.astype(np.float64)
    ref = Aq @ X16 if ax else Aq.T @ X16
    mag = (np.abs(Aq) @ np.abs(X16) if ax else np.abs(Aq.T) @ np.abs(X16)).max()
    assert np.isfinite(got).all()
    assert np.abs(got - ref).max() <= 2e-6 * mag


@pytest.mark.parametrize("m,n,l", [(1000, 777, 37), (3000, 2000, 160), (129, 4100, 80),
                                   (4096, 640, 256), (20000, 300, 48)])
@pytest.mark.parametrize("trans", [0, 1])
@pytest.mark.parametrize("dtype", ["fp8", "bf16"])
def test_split_pass_within_slicing_bound(m, n, l, trans, dtype):
    """rsvd_apply_split, the pass as the solve runs it: an FP32 operand split
    on the device into slices.  BF16 plans: `s` BF16 slices, each leaving at
    most 2^-8 of what it rounds.  FP8 plans: 2s E4M3 slices on block-scaled
    MMAs, each leaving at most 2^-4.  Either way the operand is carried to
    2^-8s relative per element, so with FP32 accumulation
    |Y - A X| <= (2^-8s + K 2^-23) (|A| |X|) elementwise (A exact: the
    dequantised codes, or BF16)."""
    rng = np.random.default_rng(m + 3 * n + l + trans)
    lda = (m + 15) // 16 * 16 + (16 if m % 3 == 0 else 0)
    if dtype == "fp8":
        dA, dS, Aq = _fp8_matrix(rng.standard_normal((m, n)), lda, spread_scales=True)
        plan = R.Plan(m, n, l, a_dtype=R.FP8E4M3, mode=R.MIXED)
        plan.set_tile_scales(dS)
    else:
        a16 = torch.zeros(n, lda, dtype=torch.bfloat16)
        a16[:, :m] = torch.from_numpy(rng.standard_normal((n, m))).to(torch.bfloat16)
        Aq = np.asfortranarray(a16[:, :m].double().numpy().T)
        dA = a16.cuda()
        plan = R.Plan(m, n, l, a_dtype=R.BF16, mode=R.MIXED)
    rows, orows = (m, n) if trans else (n, m)
    ldx = rows + 5
    X = np.zeros((l, ldx), dtype=np.float32)
    # columns of very different magnitude, and a zero column
    X[:, :rows] = (rng.standard_normal((l, rows)) *
                   np.exp2(rng.integers(-20, 20, size=(l, 1)))).astype(np.float32)
    X[l // 2, :rows] = 0.0
    dX = torch.from_numpy(X).cuda()
    X64 = X[:, :rows].T.astype(np.float64)
    AT = Aq.T if trans else Aq
    ref = AT @ X64
    mag = np.abs(AT) @ np.abs(X64)
    K = m if trans else n
    for s in (1, 2, 3):
        Y = torch.full((l, orows + 3), float("nan"), dtype=torch.float32, device="cuda")
        assert R.rsvd_apply_split(plan.handle, dA, m, n, lda, trans, dX, ldx, l, s, Y,
                                  orows + 3) == 0
        _ok(plan)
        got = Y[:, :orows].cpu().numpy().T.astype(np.float64)
        assert np.isfinite(got).all()
        bound = (2.0 ** (-8 * s) + K * 2.0 ** -23) * mag
        assert (np.abs(got - ref) <= bound + 1e-300).all(), (s, (np.abs(got - ref) / (bound + 1e-300)).max())
        assert (got[:, l // 2] == 0).all()


def test_split_pass_argument_errors():
    m, n, l = 256, 128, 16
    plan = R.Plan(m, n, l, a_dtype=R.FP8E4M3, mode=R.MIXED)
    plan.set_tile_scales(torch.ones(1, 2, device="cuda"))
    A = torch.zeros(n, m, dtype=torch.uint8, device="cuda")
    X = torch.zeros(l, m, device="cuda")
    Y = torch.zeros(l, m, device="cuda")
    f = R.rsvd_apply_split
    assert f(plan.handle, A, m, n, m, 2, X, n, l, 1, Y, m) == -6
    assert f(plan.handle, A, m, n, m, 0, X, n - 1, l, 1, Y, m) == -8
    assert f(plan.handle, A, m, n, m, 0, X, n, l, 4, Y, m) == -10
    assert f(plan.handle, A, m, n, m, 1, X, m, l, 0, Y, n) == -10
    assert f(plan.handle, A, m, n, m, 0, X, n, l, 1, Y, m - 1) == -12
    pplan = R.Plan(m, n, l)
    assert f(pplan.handle, A, m, n, m, 0, X, n, l, 1, Y, m) == 7


def _fp8_solve_and_compare(A, k, p, q, seed, lda_pad=0):
    m, n = A.shape
    lda = (m + 15) // 16 * 16 + lda_pad
    dA, dS, Aq = _fp8_matrix(A, lda)
    ref = oracle.rsvd(Aq, k, p, q + 1, seed)
    plan = R.Plan(m, n, k + p, a_dtype=R.FP8E4M3, mode=R.MIXED)
    plan.set_tile_scales(dS)
    U, S, VT = plan.solve(dA, m, n, k, p, q, seed, lda=lda)
    _ok(plan)
    s = S.cpu().numpy()
    u, vt = R.to_numpy_f(U), R.to_numpy_f(VT)
    rel = np.abs(s - ref.S) / ref.S
    assert rel.max() <= SIG_RTOL, rel.max()
    assert np.abs(u.T @ u - np.eye(k)).max() < 1e-4
    r_gpu = analysis.lowrank_residual(Aq, u, s, vt)
    r_orc = analysis.lowrank_residual(Aq, ref.U, ref.S, ref.Vt)
    assert r_gpu <= RESID_RATIO * r_orc, (r_gpu, r_orc)


def test_fp8_solve_exp_spectrum_with_noise():
    """Scaled-down FP8 workload: sigma_i = exp(-i/40) + 1e-4 noise floor."""
    A = syn.lowrank_matrix(4096, 2048, syn.spectrum("exp", 640, r=40.0), seed=3,
                           noise_2norm=1e-4)
    _fp8_solve_and_compare(A, 64, 16, 2, seed=5)


@pytest.mark.parametrize("m,n,k,p,q", [(1000, 777, 20, 10, 1), (777, 1200, 15, 5, 0),
                                       (2048, 1024, 128, 32, 3)])
def test_fp8_solve_ragged(m, n, k, p, q):
    A = syn.lowrank_matrix(m, n, syn.spectrum("poly", min(m, n), alpha=1.0), seed=m + 2 * n)
    _fp8_solve_and_compare(A, k, p, q, seed=k + p + q, lda_pad=16)


def test_fp8_argument_errors():
    m, n = 300, 200
    plan = R.Plan(m, n, 16, a_dtype=R.FP8E4M3, mode=R.MIXED)
    A = torch.zeros(n, 304, dtype=torch.uint8, device="cuda")
    U = torch.zeros(8, m, dtype=torch.float32, device="cuda")
    S = torch.zeros(8, dtype=torch.float64, device="cuda")
    VT = torch.zeros(n, 8, dtype=torch.float32, device="cuda")
    # no scales yet
    assert R.rsvd_solve(plan.handle, A, m, n, 304, 8, 4, 1, 0, U, m, S, VT, 8) == 7
    bad = torch.full((2, 3), 0.75, dtype=torch.float32, device="cuda")   # not a power of two
    assert R.rsvd_set_tile_scales(plan.handle, bad, 3, 2, 3) == -2
    neg = torch.full((2, 3), -2.0, dtype=torch.float32, device="cuda")
    assert R.rsvd_set_tile_scales(plan.handle, neg, 3, 2, 3) == -2
    good = torch.full((2, 3), 0.125, dtype=torch.float32, device="cuda")
    assert R.rsvd_set_tile_scales(plan.handle, good, 3, 2, 3) == 0
    # lda not a multiple of 16
    A2 = torch.zeros(n, 308, dtype=torch.uint8, device="cuda")
    assert R.rsvd_solve(plan.handle, A2, m, n, 308, 8, 4, 1, 0, U, m, S, VT, 8) == 7
    # scales smaller than the matrix
    small = torch.full((1, 1), 1.0, dtype=torch.float32, device="cuda")
    assert R.rsvd_set_tile_scales(plan.handle, small, 1, 1, 1) == 0
    assert R.rsvd_solve(plan.handle, A, m, n, 304, 8, 4, 1, 0, U, m, S, VT, 8) == 7
    # a BF16 plan refuses scales
    bplan = R.Plan(m, n, 16, a_dtype=R.BF16, mode=R.MIXED)
    assert R.rsvd_set_tile_scales(bplan.handle, good, 3, 2, 3) == 7


@pytest.mark.slow
def test_fp8_solve_full_size():
    """A 65536 x 16384 FP8 E4M3 with 128 x 128-tile scales, sigma_i =
    exp(-i/40) + 1e-4 noise, k=128, p=32, q=3: full-size parity with the FP64
    oracle on the dequantised A."""
    m, n, k, p, q = 65536, 16384, 128, 32, 3
    sig = syn.spectrum("exp", 640, r=40.0)
    at = syn.lowrank_matrix_torch(m, n, sig, seed=0, dtype=torch.float32,
                                  factor_dtype=torch.float32, noise_2norm=1e-4)
    codes, scales = syn.quantize_e4m3_tiles(at, m)
    del at
    Aq = fp8.dequantize_tiles(codes.cpu().numpy(), scales.cpu().numpy().T, m, n,
                              columns_as_rows=True)
    ref = oracle.rsvd(np.asfortranarray(Aq), k, p, q + 1, seed=2)
    plan = R.Plan(m, n, k + p, a_dtype=R.FP8E4M3, mode=R.MIXED)
    plan.set_tile_scales(scales)
    U, S, VT = plan.solve(codes, m, n, k, p, q, 2)
    _ok(plan)
    s = S.cpu().numpy()
    rel = np.abs(s - ref.S) / ref.S
    assert rel.max() <= SIG_RTOL, rel.max()
    u, vt = R.to_numpy_f(U), R.to_numpy_f(VT)
    r_gpu = analysis.lowrank_residual(Aq, u, s, vt)
    r_orc = analysis.lowrank_residual(Aq, ref.U, ref.S, ref.Vt)
    assert r_gpu <= RESID_RATIO * r_orc, (r_gpu, r_orc)
