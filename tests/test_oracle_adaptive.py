"""Pins of the adaptive range finder oracle (Adaptive_randRF; Halko,
Martinsson and Tropp 2011, Algorithm 4.2).

What ties it to the method rather than to itself:
  * brute force: the Q the vector loop builds is the Householder Q of the
    first j samples A omega_1..A omega_j (Gram-Schmidt order, so unique up
    to column signs), and the j where it stops is the first j at which the
    residuals of the next r samples against that Q, formed from scratch,
    all fall below the threshold;
  * a matrix of exact rank k stops at exactly j = k;
  * the tolerance guarantee ||(I - QQ*) A||_2 <= eps on decaying spectra,
    across seeds, and Eckart-Young's lower bound sigma_{j+1} on that error;
  * the a-posteriori estimate: 10 sqrt(2/pi) times the last lookahead
    maximum bounds the true error;
  * planted mistakes (the lookahead vectors not deflated by each new q_j;
    the threshold without the a-posteriori factor) that the pins catch.
"""
import numpy as np
import pytest

from oracle import adaptive as ad
from oracle import philox
from paper_2402_17794_gb300 import synthetic as syn


def _brute_force(A, eps, r, seed, cap):
    m, n = A.shape
    Om = philox.gaussian_matrix(n, cap + r, seed, stream=0)
    Y = A @ Om
    thr = eps / (10.0 * np.sqrt(2.0 / np.pi))
    for j in range(cap + 1):
        if j:
            Qj, _ = np.linalg.qr(Y[:, :j])
            R = Y[:, j:j + r] - Qj @ (Qj.T @ Y[:, j:j + r])
        else:
            Qj, R = np.zeros((m, 0)), Y[:, :r]
        look = np.linalg.norm(R, axis=0).max()
        if look <= thr:
            return j, Qj, look
    return cap, Qj, look


@pytest.mark.parametrize("m,n,kind,eps,r", [
    (300, 200, "exp", 1e-3, 10),
    (200, 320, "poly", 1e-2, 6),
    (256, 256, "geometric4", 1e-5, 4),
])
def test_matches_brute_force(m, n, kind, eps, r):
    sig = syn.spectrum(kind, min(m, n), alpha=1.5, r=8.0)
    A = syn.lowrank_matrix(m, n, sig, seed=m + 3 * n)
    res = ad.adaptive_range_finder(A, eps, r, seed=9)
    j, Qb, look = _brute_force(A, eps, r, 9, min(m, n))
    assert res.converged and res.rank == j and j > 0
    # same columns up to sign (Gram-Schmidt order makes them unique)
    d = np.abs(np.sum(res.Q * Qb, axis=0))
    assert np.abs(d - 1.0).max() <= 1e-9
    assert abs(res.lookahead[-1] - look) <= 1e-9 * sig[0]
    assert np.abs(res.Q.T @ res.Q - np.eye(j)).max() <= 1e-13


@pytest.mark.parametrize("k", [1, 7, 20])
def test_exact_rank_stops_at_rank(k):
    m, n = 240, 180
    sig = np.geomspace(1.0, 1e-2, k)
    A = syn.lowrank_matrix(m, n, sig, seed=k)
    res = ad.adaptive_range_finder(A, 1e-8, 5, seed=3)
    assert res.converged and res.rank == k
    assert np.linalg.norm(A - res.Q @ (res.Q.T @ A), 2) <= 1e-13


def test_tolerance_guarantee_and_eckart_young():
    m, n = 400, 250
    sig = syn.spectrum("poly", n, alpha=2.0)
    A = syn.lowrank_matrix(m, n, sig, seed=5)
    for eps in (1e-2, 1e-3):
        for seed in range(8):
            res = ad.adaptive_range_finder(A, eps, 10, seed=seed)
            err = np.linalg.norm(A - res.Q @ (res.Q.T @ A), 2)
            assert err <= eps
            assert err >= sig[res.rank] * (1 - 1e-12)
            # the a-posteriori estimate behind the threshold
            assert err <= ad.POSTERIOR_FACTOR * res.lookahead[-1]


def test_capacity_ends_the_loop_unconverged():
    m, n = 200, 150
    A = syn.lowrank_matrix(m, n, syn.spectrum("poly", n, alpha=0.5), seed=1)
    res = ad.adaptive_range_finder(A, 1e-6, 5, seed=2, l_max=30)
    assert not res.converged and res.rank == 30
    assert np.abs(res.Q.T @ res.Q - np.eye(30)).max() <= 1e-13


def test_adaptive_rsvd_stage_b():
    m, n = 300, 200
    sig = syn.spectrum("exp", n, r=6.0)
    A = syn.lowrank_matrix(m, n, sig, seed=8)
    out = ad.adaptive_rsvd(A, 1e-6, 8, seed=4)
    j = out.range.rank
    assert j == out.S.size and out.U.shape == (m, j)
    # sigma of Q Q* A interlace A's and, past the tolerance, match them
    assert np.all(out.S <= sig[:j] * (1 + 1e-12))
    big = sig[:j] > 1e3 * 1e-6
    assert np.abs(out.S[big] - sig[:j][big]).max() <= 1e-10 * sig[0]
    err = np.linalg.norm(A - out.U @ np.diag(out.S) @ out.Vt, 2)
    assert err <= 1e-6


def _undeflated(A, eps, r, seed, cap):
    """Planted mistake: lookahead vectors are not deflated by each new q_j."""
    m, n = A.shape
    Om = philox.gaussian_matrix(n, cap + r, seed, stream=0)
    thr = ad.threshold(eps)
    ys = [A @ Om[:, i] for i in range(r)]
    Q = np.zeros((m, 0))
    j = 0
    while max(np.linalg.norm(ys[i]) for i in range(j, j + r)) > thr and j < cap:
        y = ys[j] - Q @ (Q.T @ ys[j])
        Q = np.column_stack([Q, y / np.linalg.norm(y)])
        j += 1
        ynew = A @ Om[:, j - 1 + r]
        ys.append(ynew - Q @ (Q.T @ ynew))
    return j


def _bare_threshold(A, eps, r, seed, cap):
    """Planted mistake: the loop compares against eps itself, without the
    a-posteriori factor 10 sqrt(2/pi)."""
    m, n = A.shape
    Om = philox.gaussian_matrix(n, cap + r, seed, stream=0)
    Y = A @ Om
    for j in range(1, cap + 1):
        Qj, _ = np.linalg.qr(Y[:, :j])
        R = Y[:, j:j + r] - Qj @ (Qj.T @ Y[:, j:j + r])
        if np.linalg.norm(R, axis=0).max() <= eps:
            return j
    return cap


def test_planted_mistakes_are_caught():
    m, n = 300, 200
    sig = syn.spectrum("exp", n, r=8.0)
    A = syn.lowrank_matrix(m, n, sig, seed=21)
    eps, r = 1e-3, 10
    good = ad.adaptive_range_finder(A, eps, r, seed=9).rank
    assert good == _brute_force(A, eps, r, 9, n)[0]
    assert _undeflated(A, eps, r, 9, n) != good
    assert _bare_threshold(A, eps, r, 9, n) != good
