"""Pins of the CPU oracle to the thesis and to the mathematics (no GPU).

Each check ties ``oracle/`` to something other than itself:
* matrices of known spectrum (A = U diag(sigma) V^T, Haar U, V): exact
  recovery when rank(A) <= k, exact SVD when k+p = min(m, n);
* Eckart-Young, Eq. 3.1 (Section 3.1) and interlacing;
* orthonormality of Q (Algorithm 4 step 3), U and V;
* the expected-error bounds of Theorem 2 (Section 3.1), Theorem 3
  (Section 3.2) and Theorem 6 / Eq. 3.4 (Section 3.3), averaged over seeds
  on the controlled-gap matrices of Eq. 4.1 with the sweeps of Section 4.2;
* the canonical-angle bounds of Theorem 5 with the parameters of Section 4.3;
* the singular-vector identity of Eq. 3.2 (power steps keep U, V);
* distribution tests of the Gaussian test matrix;
* planted mistakes: each mutant of the oracle must fail at least one check.
"""
import math
import pathlib

import numpy as np
import pytest
from scipy import stats

import oracle
from oracle import analysis
from oracle import randsvd as orsvd
from oracle.philox import gaussian_matrix, philox4x32_10, philox_words
from paper_2402_17794_gb300 import synthetic as syn


# ---------------------------------------------------------------------------
# Checks (plain functions so the mutant tests can reuse them)
# ---------------------------------------------------------------------------

def check_exact_rank_recovery(fn=orsvd.rsvd):
    """rank(A) = r <= k: sigma recovered to ~1e-13, residual ~ 0."""
    m, n, r = 300, 200, 12
    sig = syn.spectrum("geometric4", r) * 3.0
    A = syn.lowrank_matrix(m, n, sig, seed=7)
    res = fn(A, k=r, p=4, q=0, seed=3)
    np.testing.assert_allclose(res.S, sig, rtol=1e-12, atol=0)
    resid = analysis.lowrank_residual(A, res.U, res.S, res.Vt)
    assert resid <= 1e-13 * sig[0], resid
    U, _, V = syn.lowrank_factors(m, n, sig, seed=7)
    assert analysis.sin_canonical_angles(U, res.U).max() < 1e-11
    assert analysis.sin_canonical_angles(V, res.Vt.T).max() < 1e-11


def check_full_rank_exact_svd(fn=orsvd.rsvd, q=1):
    """k + p = min(m, n): the method returns the exact SVD of A."""
    m, n = 120, 80
    sig = syn.spectrum("poly", n, alpha=1.0)
    A = syn.lowrank_matrix(m, n, sig, seed=11)
    res = fn(A, k=n - 5, p=5, q=q, seed=5)
    np.testing.assert_allclose(res.S, sig[: n - 5], rtol=1e-11, atol=0)
    U, _, V = syn.lowrank_factors(m, n, sig, seed=11)
    # distinct singular values: vectors agree up to sign, which the
    # normalisation fixes; compare |u_i^T u^_i|
    dots = np.abs(np.sum(U[:, : n - 5] * res.U, axis=0))
    np.testing.assert_allclose(dots, 1.0, atol=1e-9)


def check_orthonormal(fn=orsvd.rsvd):
    m, n = 400, 150
    A = syn.lowrank_matrix(m, n, syn.spectrum("exp", n, r=10.0), seed=2)
    res = fn(A, k=20, p=10, q=2, seed=9)
    l = res.Q.shape[1]
    assert np.abs(res.Q.T @ res.Q - np.eye(l)).max() < 1e-13
    assert np.abs(res.U.T @ res.U - np.eye(20)).max() < 1e-13
    assert np.abs(res.Vt @ res.Vt.T - np.eye(20)).max() < 1e-13


def check_eckart_young_and_interlacing(fn=orsvd.rsvd):
    m, n = 500, 300
    sig = syn.spectrum("poly", n, alpha=1.5)
    A = syn.lowrank_matrix(m, n, sig, seed=4)
    for (k, p, q) in [(10, 5, 0), (20, 10, 1), (30, 5, 2)]:
        res = fn(A, k=k, p=p, q=q, seed=100 + k)
        resid = analysis.lowrank_residual(A, res.U, res.S, res.Vt)
        assert resid >= sig[k] * (1 - 1e-12)                   # Eq. 3.1, rank k
        rng_err = analysis.range_error(A, res.Q)
        assert rng_err >= sig[k + p] * (1 - 1e-12)             # Eq. 3.1, rank k+p
        assert np.all(res.S <= sig[:k] * (1 + 1e-12))          # interlacing
        assert np.all(np.diff(res.S) <= 0)                     # descending


def check_projection_consistency(fn=orsvd.rsvd):
    """U diag(S) Vt must equal the best rank-k approximation of Q Q^T A
    (steps 6-8 in the thesis' order)."""
    m, n = 200, 120
    A = syn.lowrank_matrix(m, n, syn.spectrum("exp", n, r=15.0), seed=8)
    res = fn(A, k=10, p=6, q=1, seed=21)
    QQA = res.Q @ (res.Q.T @ A)
    u, s, vt = np.linalg.svd(QQA, full_matrices=False)
    best = (u[:, :10] * s[:10]) @ vt[:10]
    np.testing.assert_allclose((res.U * res.S) @ res.Vt, best, atol=1e-13)
    np.testing.assert_allclose(res.S, s[:10], rtol=1e-12)


def check_power_steps_meet_theorem6(fn=orsvd.rsvd):
    """Slowly decaying spectrum (sigma_j = 1/j, no gap): with q = 2 the mean
    range error over seeds sits below the Theorem 6 bound (Eq. 3.4), which
    is tight enough that dropping the power steps breaks it."""
    m, n, k, p, q = 1500, 400, 10, 5, 2
    sig = syn.spectrum("poly", n, alpha=1.0)
    A = syn.lowrank_matrix(m, n, sig, seed=13)
    errs = [analysis.range_error(A, fn(A, k=k, p=p, q=q, seed=s).Q) for s in range(6)]
    assert np.mean(errs) <= analysis.thm6_bound(sig, k, p, q), (np.mean(errs), analysis.thm6_bound(sig, k, p, q))


def check_gaussian_omega(gen=gaussian_matrix):
    z = gen(4000, 40, seed=2024)
    flat = z.ravel()
    assert stats.kstest(flat, "norm").pvalue > 1e-3
    assert abs(flat.mean()) < 5.0 / math.sqrt(flat.size)
    assert abs(flat.var() - 1.0) < 6.0 * math.sqrt(2.0 / flat.size)
    c = np.corrcoef(z[:, :8].T)
    assert np.abs(c - np.eye(8)).max() < 5.0 / math.sqrt(4000)


PINS = [
    check_exact_rank_recovery,
    check_full_rank_exact_svd,
    check_orthonormal,
    check_eckart_young_and_interlacing,
    check_projection_consistency,
    check_power_steps_meet_theorem6,
]


# ---------------------------------------------------------------------------
# Tests
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("check", PINS, ids=lambda f: f.__name__)
def test_pin(check):
    check()


@pytest.mark.parametrize("q", [0, 1, 3])
def test_full_rank_exact_svd_any_q(q):
    check_full_rank_exact_svd(q=q)


def test_gaussian_omega_distribution():
    check_gaussian_omega()


def test_philox_words_uniform_and_distinct_streams():
    w0, w1, w2, w3 = philox_words(512, 64, seed=99)
    for w in (w0, w1, w2, w3):
        top = (w >> np.uint64(28)).ravel().astype(np.int64)     # 16 bins
        counts = np.bincount(top, minlength=16)
        assert stats.chisquare(counts).pvalue > 1e-4
    # a different seed or stream gives a different matrix
    a = gaussian_matrix(64, 8, seed=1)
    b = gaussian_matrix(64, 8, seed=2)
    c = gaussian_matrix(64, 8, seed=1, stream=1)
    assert np.abs(a - b).max() > 0.1 and np.abs(a - c).max() > 0.1
    # seeds above 2^32 use the high key word
    d = gaussian_matrix(64, 8, seed=1 + (1 << 32))
    assert np.abs(a - d).max() > 0.1


def _read_kat():
    rows = []
    path = pathlib.Path(__file__).parent / "golden" / "philox4x32_10_kat.txt"
    for line in path.read_text().splitlines():
        if line.strip() and not line.startswith("#"):
            rows.append([int(x, 16) for x in line.split()])
    return rows


def check_philox_kat(fn=philox4x32_10):
    """The published Philox4x32-10 known-answer vectors (Salmon et al., SC'11;
    Random123's known-answer file): counter (c0..c3) and key (k0, k1) map to
    the four printed output words."""
    rows = _read_kat()
    assert len(rows) == 3
    for r in rows:
        c = [np.array([x], dtype=np.uint64) for x in r[:4]]
        out = [int(w[0]) for w in fn(*c, r[4], r[5])]
        assert out == r[6:], (r, [hex(x) for x in out])


def test_philox_known_answer_vectors():
    check_philox_kat()


def _philox_mutant(swap_multipliers=False, permute=False, rounds=10):
    """Philox4x32 with one plausible mistake planted (a test-side copy of the
    round structure, not the oracle's code)."""
    mask = (1 << 32) - 1
    m0, m1 = 0xD2511F53, 0xCD9E8D57
    if swap_multipliers:
        m0, m1 = m1, m0

    def fn(c0, c1, c2, c3, k0, k1):
        c = [int(x[0]) for x in (c0, c1, c2, c3)]
        k = [int(k0), int(k1)]
        for rnd in range(rounds):
            if rnd:
                k = [(k[0] + 0x9E3779B9) & mask, (k[1] + 0xBB67AE85) & mask]
            p0, p1 = m0 * c[0], m1 * c[2]
            c = [(p1 >> 32) ^ c[1] ^ k[0], p1 & mask, (p0 >> 32) ^ c[3] ^ k[1], p0 & mask]
        if permute:
            c = [c[1], c[0], c[3], c[2]]
        return [np.array([x], dtype=np.uint64) for x in c]
    return fn


@pytest.mark.parametrize("mutant", [
    dict(swap_multipliers=True), dict(permute=True), dict(rounds=9)])
def test_philox_kat_catches_planted_mistakes(mutant):
    # the unmutated test-side copy passes, so the pin, not the copy, decides
    check_philox_kat(_philox_mutant())
    with pytest.raises(AssertionError):
        check_philox_kat(_philox_mutant(**mutant))


def test_omega_prefix_property():
    """Column j of Omega depends only on (seed, j, i): an n x l matrix is the
    leading block of an n x l' one (l' > l), as the column-major counter
    layout states."""
    a = gaussian_matrix(100, 5, seed=77)
    b = gaussian_matrix(100, 9, seed=77)
    np.testing.assert_array_equal(a, b[:, :5])


def test_power_identity_eq32():
    """Eq. 3.2: (AA*)^q A has the singular vectors of A and singular values
    sigma^(2q+1)."""
    m, n = 60, 40
    sig = syn.spectrum("exp", n, r=8.0)
    A = syn.lowrank_matrix(m, n, sig, seed=31)
    U, _, V = syn.lowrank_factors(m, n, sig, seed=31)
    Aq = np.linalg.matrix_power(A @ A.T, 2) @ A
    u, s, vt = np.linalg.svd(Aq)
    np.testing.assert_allclose(s[:10], sig[:10] ** 5, rtol=1e-9)
    dots = np.abs(np.sum(u[:, :10] * U[:, :10], axis=0))
    np.testing.assert_allclose(dots, 1.0, atol=1e-8)


def test_power_steps_shrink_angles():
    """More power steps give smaller canonical angles to U_k (Section 4.3)."""
    m, n = 1000, 200
    A = syn.controlled_gap(m, n, gap=2.0, seed=3)
    sig = syn.spectrum("gap", n, gap=2.0)
    U, _, _ = syn.lowrank_factors(m, n, sig, seed=3)
    worst = []
    for q in (0, 1, 2):
        res = orsvd.rsvd(A, k=15, p=5, q=q, seed=8)
        worst.append(analysis.sin_canonical_angles(U[:, :15], res.Q).max())
    assert worst[0] > worst[1] > worst[2]


def test_alg3_alg4_same_range_small_q():
    """Algorithms 3 and 4 span the same range in exact arithmetic; for a
    well-conditioned case and q = 1 they agree to rounding."""
    m, n = 300, 100
    A = syn.lowrank_matrix(m, n, syn.spectrum("poly", n, alpha=0.5), seed=5)
    q3, _ = orsvd.range_finder(A, 20, 1, seed=4, algorithm=3)
    q4, _ = orsvd.range_finder(A, 20, 1, seed=4, algorithm=4)
    assert analysis.sin_canonical_angles(q3, q4).max() < 1e-10


def test_bound_formulas_agree_in_special_cases():
    """Theorem 3 at q = 0 is Theorem 2; Theorem 6 with a flat tail is
    Eq. 3.5 -- two independently typed formulas of the thesis."""
    sig = syn.spectrum("gap", 300, gap=10.0)
    for k, p in [(5, 5), (20, 5), (20, 25)]:
        assert math.isclose(analysis.thm3_bound(sig, k, p, 0, 3000, 300),
                            analysis.thm2_bound(sig, k, p, 3000, 300), rel_tol=1e-14)
    flat = np.concatenate([np.linspace(5, 2, 20), np.full(280, 0.5)])
    for q in (0, 1, 2):
        a = analysis.thm6_bound(flat, 20, 5, q)
        b = analysis.eq35_bound(0.5, 20, 5, q, 3000, 300)
        assert math.isclose(a, b, rel_tol=1e-13)
    # Theorem 6 with q -> large tends to sigma_{k+1} (Section 3.3)
    assert analysis.thm6_bound(sig, 20, 5, 40) < 1.2 * sig[20]


def _mean_range_error(A, k, p, q, algorithm, seeds):
    errs = []
    for s in seeds:
        Q, _ = orsvd.range_finder(A, k + p, q, seed=s, algorithm=algorithm)
        errs.append(analysis.range_error(A, Q))
    return float(np.mean(errs))


@pytest.fixture(scope="module")
def gap10():
    m, n = 3000, 300
    return syn.controlled_gap(m, n, gap=10.0, seed=1), syn.spectrum("gap", n, gap=10.0)


def test_theorem2_fixed_p_sweep_k(gap10):
    """Section 4.2.1: p = 5, k = 5..30; Algorithm 1 error below Theorem 2."""
    A, sig = gap10
    for k in (5, 10, 15, 20, 25, 30):
        e = _mean_range_error(A, k, 5, 0, 1, range(10))
        assert sig[k + 5] <= e <= analysis.thm2_bound(sig, k, 5, 3000, 300)


def test_theorem2_fixed_k_sweep_p(gap10):
    A, sig = gap10
    for p in (5, 10, 15, 20, 25):
        e = _mean_range_error(A, 20, p, 0, 1, range(10))
        assert e <= analysis.thm2_bound(sig, 20, p, 3000, 300)


def test_theorem3_alg3_q1(gap10):
    """Section 4.2.2: Algorithm 3, q = 1, below Theorem 3."""
    A, sig = gap10
    for k in (5, 15, 30):
        e = _mean_range_error(A, k, 5, 1, 3, range(10))
        assert e <= analysis.thm3_bound(sig, k, 5, 1, 3000, 300)


def test_theorem6_alg4_q1_sweeps(gap10):
    """Section 4.2.3: Algorithm 4, q = 1, k and p sweeps, below Eq. 3.4."""
    A, sig = gap10
    for k in (5, 10, 15, 20, 25, 30):
        e = _mean_range_error(A, k, 5, 1, 4, range(10))
        assert e <= analysis.thm6_bound(sig, k, 5, 1), (k, e)
    for p in (5, 10, 15, 20, 25):
        e = _mean_range_error(A, 20, p, 1, 4, range(10))
        assert e <= analysis.thm6_bound(sig, 20, p, 1), (p, e)


def test_theorem6_average_100_runs(gap10):
    """Section 4.2.3: k = 20, p = 5, q = 1, the mean over 100 runs."""
    A, sig = gap10
    e = _mean_range_error(A, 20, 5, 1, 4, range(100))
    assert sig[25] <= e <= analysis.thm6_bound(sig, 20, 5, 1)


@pytest.mark.parametrize("q", [0, 1, 2])
@pytest.mark.parametrize("algorithm", [3, 4])
def test_theorem5_canonical_angles(q, algorithm):
    """Section 4.3: gap = 2, k = 25, p = 5; computed sin theta_j, sin nu_j
    below the Theorem 5 bounds (Assumption 4 holds: gamma_k < 1)."""
    m, n, k, p = 3000, 300, 25, 5
    sig = syn.spectrum("gap", n, gap=2.0)
    A = syn.controlled_gap(m, n, gap=2.0, seed=6)
    U, _, V = syn.lowrank_factors(m, n, sig, seed=6)
    res = orsvd.rsvd(A, k=k, p=p, q=q, seed=17, algorithm=algorithm, truncate=False)
    bu, bv = analysis.thm5_bounds(V, res.Omega, sig, k, q)
    su = analysis.sin_canonical_angles(U[:, :k], res.Q)
    sv = analysis.sin_canonical_angles(V[:, :k], res.Vt.T)
    assert np.all(su <= bu * (1 + 1e-9) + 1e-13), (su, bu)
    assert np.all(sv <= bv * (1 + 1e-9) + 1e-13), (sv, bv)


def test_spectral_norm_lanczos_matches_exact():
    rng = np.random.default_rng(0)
    M = rng.standard_normal((300, 200)) @ np.diag(np.linspace(1, 0.01, 200)) @ rng.standard_normal((200, 200))
    exact = np.linalg.norm(M, 2)
    est = analysis.spectral_norm(lambda x: M @ x, lambda y: M.T @ y, M.shape)
    assert abs(est - exact) <= 1e-10 * exact


# ---------------------------------------------------------------------------
# Planted mistakes: every mutant must fail at least one pin
# ---------------------------------------------------------------------------

def _mutant_orth_normalise_only(Y):
    return Y / np.linalg.norm(Y, axis=0)


def _mutant_power_steps_skipped(A, l, q, seed, algorithm=4, Omega=None):
    return _ORIG_RANGE_FINDER(A, l, 0, seed, algorithm, Omega)


def _mutant_truncate_tail(A, k, p, q, seed, algorithm=4, Omega=None, truncate=True):
    full = _ORIG_RSVD(A, k, p, q, seed, algorithm, Omega, truncate=False)
    U, S, Vt = full.U[:, p:], full.S[p:], full.Vt[p:]
    return orsvd.RsvdResult(U=U, S=S, Vt=Vt, Q=full.Q, Omega=full.Omega)


def _mutant_lift_transposed(A, k, p, q, seed, algorithm=4, Omega=None, truncate=True):
    A = np.asarray(A)
    Q, Om = orsvd.range_finder(A, k + p, q, seed, algorithm, Omega)
    Ut, S, Vt = np.linalg.svd(Q.T @ A, full_matrices=False)
    U = Q @ Ut.T
    return orsvd.RsvdResult(U=U[:, :k], S=S[:k], Vt=Vt[:k], Q=Q, Omega=Om)


def _mutant_sign_u_only(A, k, p, q, seed, algorithm=4, Omega=None, truncate=True):
    r = _ORIG_RSVD(A, k, p, q, seed, algorithm, Omega, truncate)
    U = r.U.copy()
    U[:, 0] *= -1
    return orsvd.RsvdResult(U=U, S=r.S, Vt=r.Vt, Q=r.Q, Omega=r.Omega)


def _mutant_sigma_of_sample(A, k, p, q, seed, algorithm=4, Omega=None, truncate=True):
    """Reports the singular values of the sample Y = A Omega instead of B's."""
    r = _ORIG_RSVD(A, k, p, q, seed, algorithm, Omega, truncate)
    s = np.linalg.svd(np.asarray(A) @ r.Omega, compute_uv=False)[:k]
    return orsvd.RsvdResult(U=r.U, S=s, Vt=r.Vt, Q=r.Q, Omega=r.Omega)


_ORIG_RANGE_FINDER = orsvd.range_finder
_ORIG_RSVD = orsvd.rsvd


def _all_pins_pass(fn):
    for check in PINS:
        try:
            check(fn)
        except AssertionError:
            return False
    return True


def test_pins_pass_on_oracle():
    assert _all_pins_pass(orsvd.rsvd)


@pytest.mark.parametrize("mutant", [
    _mutant_truncate_tail, _mutant_lift_transposed, _mutant_sign_u_only,
    _mutant_sigma_of_sample,
], ids=lambda f: f.__name__)
def test_planted_mistake_is_caught(mutant):
    assert not _all_pins_pass(mutant)


def test_planted_orth_mistake_is_caught(monkeypatch):
    monkeypatch.setattr(orsvd, "orth", _mutant_orth_normalise_only)
    assert not _all_pins_pass(orsvd.rsvd)


def test_planted_power_step_mistake_is_caught(monkeypatch):
    monkeypatch.setattr(orsvd, "range_finder", _mutant_power_steps_skipped)
    assert not _all_pins_pass(orsvd.rsvd)


def test_planted_box_muller_mistake_is_caught():
    def bad(n, l, seed, stream=0):
        w0, w1, w2, w3 = philox_words(n, l, seed, stream)
        u1 = ((w0 >> np.uint64(11)).astype(np.float64) + 0.5) * 2.0 ** -53
        u2 = ((w2 >> np.uint64(11)).astype(np.float64) + 0.5) * 2.0 ** -53
        return np.sqrt(-2.0 * np.log(u1)) * np.cos(np.pi * u2)   # pi, not 2 pi
    with pytest.raises(AssertionError):
        check_gaussian_omega(bad)
