"""Gaussian test matrix Omega of Algorithm 4, step 1 (Section 3.3) -- oracle side.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The thesis asks for "an n x (k+p) Gaussian test matrix" (Algorithm 1 step 1,
Algorithm 4 step 1) and leaves the generator open.  Both sides of the parity
comparison draw Omega from one counter-based generator so the same seed gives
the same Omega on the CPU and on the GPU; each side implements it from its
published definition:

* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
  as 1, 2, 3", SC'11): a 4 x 32-bit counter and 2 x 32-bit key; each of ten
  rounds multiplies two counter words by fixed odd constants, keeps the high
  and low halves of the 64-bit products, and XORs the high halves with the
  other two words and the round key; the key is bumped by two Weyl constants
  between rounds.
* Box-Muller (Box & Muller 1958): z = sqrt(-2 ln u1) cos(2 pi u2) for u1, u2
  uniform on (0, 1).  One normal per counter; the sine partner is not used.

Counter layout (shared with the CUDA side by specification only): element
(i, j) of the n x l column-major Omega uses the 64-bit linear index
t = j*n + i as counter words (lo32(t), hi32(t), stream, 0) and the key
(lo32(seed), hi32(seed)).  Words 0,1 give u1 and words 2,3 give u2, each as
(x + 1/2) 2^-52 where x is the 52-bit integer (w_a >> 6) 2^26 + (w_b >> 6);
that value is exact in FP64 and lies strictly inside (0, 1).

Pinned by the published known-answer vectors of Philox4x32-10 (the all-zero,
all-ones and pi-digit counter/key cases of Random123's known-answer file).
"""
from __future__ import annotations

import numpy as np

_MASK = np.uint64(0xFFFFFFFF)
# Philox4x32 multipliers and Weyl key increments (SC'11 paper).
_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox4x32 rounds on arrays of counters (uint32 values held in
    uint64 arrays); returns the four output words as uint64 arrays."""
    c0, c1, c2, c3 = (np.asarray(x, dtype=np.uint64) & _MASK for x in (c0, c1, c2, c3))
    k0 = np.uint64(int(k0) & 0xFFFFFFFF)
    k1 = np.uint64(int(k1) & 0xFFFFFFFF)
    for rnd in range(10):
        if rnd:
            k0 = (k0 + _W0) & _MASK
            k1 = (k1 + _W1) & _MASK
        p0 = _M0 * c0          # < 2^64, exact in uint64
        p1 = _M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def _uniform52(wa, wb):
    x = ((wa >> np.uint64(6)) << np.uint64(26)) | (wb >> np.uint64(6))
    return (x.astype(np.float64) + 0.5) * 2.0 ** -52


def philox_words(n: int, l: int, seed: int, stream: int = 0):
    """The four raw 32-bit words for every element of an n x l matrix,
    each as an (n, l) uint64 array (column-major linear counter)."""
    t = np.arange(n * l, dtype=np.uint64)
    seed = int(seed)
    w = philox4x32_10(t & _MASK, t >> np.uint64(32),
                      np.full_like(t, stream & 0xFFFFFFFF), np.zeros_like(t),
                      seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    return tuple(x.reshape(l, n).T for x in w)


def gaussian_matrix(n: int, l: int, seed: int, stream: int = 0) -> np.ndarray:
    """Standard Gaussian n x l matrix (FP64, column-major) for ``seed``."""
    w0, w1, w2, w3 = philox_words(n, l, seed, stream)
    u1 = _uniform52(w0, w1)
    u2 = _uniform52(w2, w3)
    z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    return np.asfortranarray(z)
