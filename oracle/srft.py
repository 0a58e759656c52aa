"""Subsampled random Fourier transform (SRFT) test matrix and the fast
randomized range finder built on it (FastRandRF / SRFT of the toolbox,
Section 4's function lists) in plain FP64 / complex128 -- TEST
INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The thesis defines the test matrix (n x l, complex)

    Omega = sqrt(n / l) D F R

  * D: n x n diagonal, independent entries uniform on the complex unit
    circle;
  * F: the n x n unitary DFT, f_pq = n^-1/2 exp(-2 pi i (p-1)(q-1) / n);
  * R: n x l, samples l of the n coordinates uniformly at random;

and FastRandRF (Algorithm 4.5 of Halko, Martinsson and Tropp 2011, which it
names as its source): Y = A Omega, Q = orth(Y), an m x l orthonormal
(complex) basis approximating range(A).  ``srft_rsvd`` adds Stage B of the
prototype (Section 2.2) on that basis: the rank-k SVD B = Q^H A = U~ S V^H,
U = Q U~.

Readings (the thesis is silent on these):
  * the random numbers come from the Philox4x32-10 generator of
    ``philox.py`` (counter words (lo32(t), hi32(t), stream, 0)); the phase
    of D's entry j is 2 pi u_j with u_j the 52-bit uniform of counter t = j
    on stream 2;
  * R samples l distinct coordinates (a subset, no repeats) by Floyd's
    algorithm (Bentley and Floyd, CACM 30(9), 1987): for j = n-l .. n-1,
    draw t uniform on {0..j} and add t, or j when t is already taken; the
    draw of step s = j - (n-l) is t = min(floor(u_s (j+1)), j) with u_s the
    52-bit uniform of counter s on stream 3 (the product rounded once in
    FP64).  The columns of R are the sampled coordinates in ascending order;
  * Q's columns are the Gram-Schmidt vectors of Y's columns in that order
    (unique up to a unit complex factor each).

Library primitives used as steps: numpy's matrix product, exp, and LAPACK's
complex Householder QR.  The DFT is built entry by entry from its definition
(the FFT appears only in the pins, as an independent check).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .philox import _uniform52, philox4x32_10

PHASE_STREAM = 2
SAMPLE_STREAM = 3


def _uniforms(count: int, seed: int, stream: int) -> np.ndarray:
    t = np.arange(count, dtype=np.uint64)
    seed = int(seed)
    w0, w1, _, _ = philox4x32_10(t & np.uint64(0xFFFFFFFF), t >> np.uint64(32),
                                 np.full_like(t, stream), np.zeros_like(t),
                                 seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    return _uniform52(w0, w1)


def srft_phases(n: int, seed: int) -> np.ndarray:
    """Diagonal of D: exp(2 pi i u_j), j = 0..n-1."""
    u = _uniforms(n, seed, PHASE_STREAM)
    return np.exp(2j * np.pi * u)


def srft_coordinates(n: int, l: int, seed: int) -> np.ndarray:
    """The l coordinates R samples (Floyd's algorithm), ascending."""
    if not 1 <= l <= n:
        raise ValueError("need 1 <= l <= n")
    u = _uniforms(l, seed, SAMPLE_STREAM)
    chosen: set[int] = set()
    for s, j in enumerate(range(n - l, n)):
        t = min(int(np.floor(u[s] * float(j + 1))), j)
        chosen.add(j if t in chosen else t)
    return np.array(sorted(chosen), dtype=np.int64)


def dft_columns(n: int, cols: np.ndarray) -> np.ndarray:
    """Columns `cols` (0-based) of the unitary DFT: n^-1/2 exp(-2 pi i p q / n)."""
    p = np.arange(n, dtype=np.float64)[:, None]
    q = np.asarray(cols, dtype=np.float64)[None, :]
    return np.exp(-2j * np.pi * ((p * q) % n) / n) / np.sqrt(n)


def srft_matrix(n: int, l: int, seed: int) -> np.ndarray:
    """Omega = sqrt(n/l) D F R, n x l complex."""
    d = srft_phases(n, seed)
    r = srft_coordinates(n, l, seed)
    return np.sqrt(n / l) * (d[:, None] * dft_columns(n, r))


@dataclass
class SrftRange:
    Q: np.ndarray        # m x l complex, orthonormal columns
    Omega: np.ndarray    # n x l complex
    Y: np.ndarray        # m x l complex, the sample A Omega


def fast_range_finder(A: np.ndarray, l: int, seed: int) -> SrftRange:
    """FastRandRF: Y = A Omega (Omega the SRFT), Q = orth(Y)."""
    A = np.asarray(A)
    m, n = A.shape
    if not 1 <= l <= min(m, n):
        raise ValueError("need 1 <= l <= min(m, n)")
    Om = srft_matrix(n, l, seed)
    Y = A @ Om
    Q, _ = np.linalg.qr(Y, mode="reduced")
    return SrftRange(Q=Q, Omega=Om, Y=Y)


def gram_schmidt_phases(Q: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """Q with each column multiplied by the unit factor that makes
    q_j^H y_j real and positive (the Gram-Schmidt normalisation)."""
    d = np.einsum("ij,ij->j", Q.conj(), Y)
    ph = np.where(np.abs(d) > 0, d / np.where(np.abs(d) > 0, np.abs(d), 1.0), 1.0)
    return Q * ph[None, :]


@dataclass
class SrftSvd:
    U: np.ndarray        # m x k complex, orthonormal columns
    S: np.ndarray        # k, descending
    Vt: np.ndarray       # k x n complex (V^H)
    range: SrftRange


def srft_rsvd(A: np.ndarray, k: int, p: int, seed: int) -> SrftSvd:
    """The rank-k SVD on FastRandRF's range (Stage B of the prototype,
    Section 2.2, on the complex basis): B = Q^H A, B = U~ S V^H, U = Q U~,
    keep the leading k triplets (Section 3.1's truncation).  Each (u_i, v_i)
    is rotated by the unit factor that makes u_i's largest-magnitude entry
    real and positive (the complex form of the real sign convention)."""
    A = np.asarray(A)
    l = k + p
    rf = fast_range_finder(A, l, seed)
    B = rf.Q.conj().T @ A
    Ut, S, Vh = np.linalg.svd(B, full_matrices=False)
    U = rf.Q @ Ut[:, :k]
    Vh = Vh[:k]
    idx = np.argmax(np.abs(U), axis=0)
    ph = U[idx, np.arange(k)]
    ph = np.where(np.abs(ph) > 0, ph / np.abs(ph), 1.0)
    U = U / ph[None, :]
    Vh = Vh / ph[:, None].conj()
    return SrftSvd(U=U, S=S[:k], Vt=Vh, range=rf)
