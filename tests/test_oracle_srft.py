"""Pins of the SRFT oracle (the toolbox's SRFT and FastRandRF; Halko,
Martinsson and Tropp 2011, Algorithm 4.5).

What ties it to the definitions rather than to itself:
  * A D F R built entry by entry equals numpy's FFT of the rows of A D,
    sampled at R's coordinates and scaled by sqrt(n/l) n^-1/2 (a library
    routine with its own sign and normalisation conventions);
  * F is unitary; D's entries have modulus 1 with uniformly distributed
    angles (Kolmogorov-Smirnov);
  * Floyd's sampler returns l distinct ascending coordinates in [0, n), each
    l-subset of a small n equally often (chi-square over many seeds);
  * the range finder: Q^H Q = I, exact capture of a matrix of rank < l,
    and the SRFT bound ||(I - QQ^H) A|| <= sqrt(1 + 7n/l) sigma_{k+1} of
    Halko et al. (Theorem 11.2) on decaying spectra;
  * a planted mistake (D left out) fails on a matrix whose rows are DFT
    modes outside the sample, where the true method succeeds.
"""
import itertools

import numpy as np
import pytest
from scipy import stats

from oracle import srft
from paper_2402_17794_gb300 import synthetic as syn


@pytest.mark.parametrize("m,n,l", [(7, 16, 5), (12, 60, 9), (5, 97, 13)])
def test_sketch_equals_fft_of_rows(m, n, l):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((m, n))
    Om = srft.srft_matrix(n, l, seed=3)
    d = srft.srft_phases(n, 3)
    r = srft.srft_coordinates(n, l, 3)
    ref = np.fft.fft(A * d[None, :], axis=1)[:, r] * np.sqrt(n / l) / np.sqrt(n)
    assert np.abs(A @ Om - ref).max() <= 1e-12 * np.abs(ref).max()


def test_dft_is_unitary():
    n = 48
    F = srft.dft_columns(n, np.arange(n))
    assert np.abs(F.conj().T @ F - np.eye(n)).max() <= 1e-13


def test_phases_unit_modulus_uniform_angle():
    d = srft.srft_phases(20000, seed=7)
    assert np.abs(np.abs(d) - 1.0).max() <= 1e-15
    ang = (np.angle(d) / (2 * np.pi)) % 1.0
    assert stats.kstest(ang, "uniform").pvalue > 1e-3


def test_floyd_sample_distinct_sorted_uniform():
    for n, l in [(10, 1), (10, 10), (1000, 80), (8192, 288)]:
        r = srft.srft_coordinates(n, l, seed=n + l)
        assert r.size == l and np.all(np.diff(r) > 0) and r[0] >= 0 and r[-1] < n
    n, l, runs = 6, 3, 3000
    counts = {c: 0 for c in itertools.combinations(range(n), l)}
    for s in range(runs):
        counts[tuple(srft.srft_coordinates(n, l, seed=s))] += 1
    obs = np.array(list(counts.values()))
    assert stats.chisquare(obs).pvalue > 1e-3


@pytest.mark.parametrize("k,l", [(5, 12), (20, 30)])
def test_exact_capture_of_low_rank(k, l):
    m, n = 200, 150
    sig = np.geomspace(1.0, 1e-3, k)
    A = syn.lowrank_matrix(m, n, sig, seed=k)
    res = srft.fast_range_finder(A, l, seed=1)
    assert np.abs(res.Q.conj().T @ res.Q - np.eye(l)).max() <= 1e-13
    err = np.linalg.norm(A - res.Q @ (res.Q.conj().T @ A), 2)
    assert err <= 1e-13


def test_srft_error_bound():
    m, n = 300, 256
    sig = syn.spectrum("exp", n, r=6.0)
    A = syn.lowrank_matrix(m, n, sig, seed=2)
    for k, l in [(10, 40), (20, 64)]:
        for seed in range(5):
            res = srft.fast_range_finder(A, l, seed=seed)
            err = np.linalg.norm(A - res.Q @ (res.Q.conj().T @ A), 2)
            assert err >= sig[l] * (1 - 1e-12)            # Eckart-Young
            assert err <= np.sqrt(1 + 7 * n / l) * sig[k]


def test_gram_schmidt_phases():
    rng = np.random.default_rng(0)
    Y = rng.standard_normal((30, 6)) + 1j * rng.standard_normal((30, 6))
    Q = srft.gram_schmidt_phases(np.linalg.qr(Y)[0], Y)
    R = Q.conj().T @ Y
    assert np.abs(np.imag(np.diag(R))).max() <= 1e-13 and np.all(np.real(np.diag(R)) > 0)
    assert np.abs(np.tril(R, -1)).max() <= 1e-13


def test_planted_mistake_missing_d():
    """Rows of A made of DFT modes the sample misses: without D the sketch
    sees nothing of A; with D it captures A exactly."""
    m, n, l, seed = 40, 64, 16, 5
    r = set(srft.srft_coordinates(n, l, seed).tolist())
    # modes f whose conjugate n - f is missed too, so a real A stays blind
    missed = [f for f in range(1, n) if f not in r and (n - f) % n not in r][:6]
    assert len(missed) == 6
    F = srft.dft_columns(n, np.array(missed))             # n x 6
    rng = np.random.default_rng(1)
    A = np.real(rng.standard_normal((m, 6)) @ F.conj().T) # real, rank <= 12
    r = np.array(sorted(r))
    good = srft.fast_range_finder(A, l, seed)
    assert np.linalg.norm(A - good.Q @ (good.Q.conj().T @ A), 2) <= 1e-12 * np.linalg.norm(A, 2)
    bad_Y = A @ (np.sqrt(n / l) * srft.dft_columns(n, r))  # D left out
    assert np.linalg.norm(bad_Y) <= 1e-12 * np.linalg.norm(A)


def test_srft_rsvd_stage_b():
    """Stage B on the SRFT range: exact for a matrix of rank <= k, Eckart-Young
    and interlacing otherwise, orthonormal factors, the phase convention, and
    U S V^H reproducing Q Q^H A truncated to rank k."""
    m, n, k, p = 240, 192, 12, 8
    sig = np.geomspace(2.0, 1e-2, 10)
    A = syn.lowrank_matrix(m, n, sig, seed=3)                  # rank 10 <= k
    out = srft.srft_rsvd(A, k, p, seed=2)
    assert np.abs(out.S[:10] - sig).max() <= 1e-12 * sig[0]
    assert np.abs(out.S[10:]).max() <= 1e-12 * sig[0]
    assert np.linalg.norm(A - out.U @ np.diag(out.S) @ out.Vt, 2) <= 1e-12 * sig[0]
    full = syn.spectrum("exp", n, r=5.0)
    A = syn.lowrank_matrix(m, n, full, seed=4)
    out = srft.srft_rsvd(A, k, p, seed=5)
    err = np.linalg.norm(A - out.U @ np.diag(out.S) @ out.Vt, 2)
    assert err >= full[k] * (1 - 1e-12)                        # Eckart-Young
    assert np.all(out.S <= full[:k] * (1 + 1e-12))             # interlacing
    assert np.abs(out.U.conj().T @ out.U - np.eye(k)).max() <= 1e-12
    assert np.abs(out.Vt @ out.Vt.conj().T - np.eye(k)).max() <= 1e-12
    idx = np.argmax(np.abs(out.U), axis=0)
    lead = out.U[idx, np.arange(k)]
    assert np.abs(lead.imag).max() <= 1e-14 and np.all(lead.real > 0)
    # truncating Q Q^H A to rank k gives the same matrix
    P = out.range.Q @ (out.range.Q.conj().T @ A)
    u, s, vh = np.linalg.svd(P, full_matrices=False)
    assert np.abs((u[:, :k] * s[:k]) @ vh[:k] - out.U @ np.diag(out.S) @ out.Vt).max() <= 1e-12
