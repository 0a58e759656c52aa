"""Seeded synthetic test matrices for the randomized SVD.

This module builds inputs only.  It contains none of the randomized SVD's
arithmetic (no sketch, no orthonormalisation of a sample, no projection, no
small SVD).  Both the CUDA path and the CPU oracle consume what it builds,
which is why it lives in a module of its own.

Every matrix has the form A = U diag(sigma) V^T (+ optional noise), where U
and V have orthonormal columns drawn from the Haar measure (QR of a seeded
Gaussian matrix with the signs of R's diagonal folded into Q, Mezzadri 2007),
so the singular values of A are known exactly by construction.  That is what
lets the tests check the method against closed forms (exact rank-k recovery,
Eckart-Young, the expected-error bounds of Theorems 2, 3 and 6) instead of
against another implementation of the same arithmetic.

Layout: every matrix returned is column-major (Fortran order), the layout
of the thesis' MATLAB setting and of the C ABI.

Spectra of the thesis' workloads and of the ones this library is measured on:
  * ``geometric4``: sigma_i = 2^(-i/4)
  * ``poly``:       sigma_i = i^(-alpha)
  * ``exp``:        sigma_i = exp(-i/r)
  * ``gap``:        the controlled-gap family of Eq. 4.1, sigma_j = gap/j for
                    j <= r and 1/j after (Section 4.2).
"""
from __future__ import annotations

import numpy as np

# Streams of the seeded generator: each random object of a workload draws from
# its own numpy Generator so that, e.g., the noise does not shift U.
_STREAM_U, _STREAM_V, _STREAM_NOISE, _STREAM_SPARSE = 0, 1, 3, 5


def spectrum(kind: str, count: int, *, alpha: float = 1.5, r: float = 40.0,
             gap: float = 1.0, gap_at: int = 15) -> np.ndarray:
    """Return sigma_1 >= ... >= sigma_count for a named decay profile."""
    i = np.arange(1, count + 1, dtype=np.float64)
    if kind == "geometric4":
        return np.exp2(-i / 4.0)
    if kind == "poly":
        return i ** (-alpha)
    if kind == "exp":
        return np.exp(-i / r)
    if kind == "gap":
        # Eq. 4.1: gap/j for the first r terms, 1/j after.
        s = 1.0 / i
        s[:gap_at] *= gap
        return s
    raise ValueError(f"unknown spectrum kind {kind!r}")


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.default_rng([int(seed) & 0xFFFFFFFF, stream])


def haar_columns(rows: int, cols: int, rng: np.random.Generator) -> np.ndarray:
    """First ``cols`` columns of a Haar-distributed orthogonal ``rows x rows``
    matrix: Q of a Gaussian matrix's QR with R's diagonal made positive."""
    g = rng.standard_normal((rows, cols))
    q, r = np.linalg.qr(g, mode="reduced")
    d = np.sign(np.diag(r))
    d[d == 0] = 1.0
    return np.asfortranarray(q * d)


def lowrank_matrix(m: int, n: int, sigma: np.ndarray, seed: int,
                   noise_2norm: float = 0.0) -> np.ndarray:
    """A = U diag(sigma) V^T (+ E), FP64, column-major.

    ``len(sigma)`` <= min(m, n) sets the number of Haar columns of U and V.
    With ``noise_2norm`` > 0, E has i.i.d. N(0, s^2) entries with
    s = noise_2norm / (sqrt(m) + sqrt(n)), so that ||E||_2 is close to
    ``noise_2norm`` (the largest singular value of an m x n Gaussian matrix
    concentrates at s (sqrt(m) + sqrt(n))).
    """
    r = len(sigma)
    if r > min(m, n):
        raise ValueError("more singular values than min(m, n)")
    u = haar_columns(m, r, _rng(seed, _STREAM_U))
    v = haar_columns(n, r, _rng(seed, _STREAM_V))
    a = (u * np.asarray(sigma, dtype=np.float64)) @ v.T
    if noise_2norm > 0.0:
        s = noise_2norm / (np.sqrt(m) + np.sqrt(n))
        a += s * _rng(seed, _STREAM_NOISE).standard_normal((m, n))
    return np.asfortranarray(a)


def symmetric_matrix(n: int, lam: np.ndarray, seed: int) -> np.ndarray:
    """A = U diag(lam) U^T, FP64, column-major: a real symmetric (Hermitian)
    n x n matrix with the prescribed eigenvalues ``lam`` (any signs) and Haar
    eigenvectors, so its eigenvalues are known exactly by construction."""
    r = len(lam)
    if r > n:
        raise ValueError("more eigenvalues than n")
    u = haar_columns(n, r, _rng(seed, _STREAM_U))
    a = (u * np.asarray(lam, dtype=np.float64)) @ u.T
    return np.asfortranarray(0.5 * (a + a.T))


def signed_spectrum(sigma: np.ndarray, seed: int) -> np.ndarray:
    """``sigma`` with seeded random signs: an indefinite spectrum with the
    prescribed magnitudes (the order by magnitude is kept)."""
    sg = np.where(_rng(seed, _STREAM_SPARSE + 1).uniform(size=len(sigma)) < 0.5, -1.0, 1.0)
    return np.asarray(sigma, dtype=np.float64) * sg


def lowrank_factors(m: int, n: int, sigma: np.ndarray, seed: int):
    """The exact factors (U, sigma, V) of :func:`lowrank_matrix` (no noise)."""
    r = len(sigma)
    u = haar_columns(m, r, _rng(seed, _STREAM_U))
    v = haar_columns(n, r, _rng(seed, _STREAM_V))
    return u, np.asarray(sigma, dtype=np.float64), v


def controlled_gap(m: int, n: int, gap: float, seed: int, r: int = 15,
                   vectors: str = "haar") -> np.ndarray:
    """Test matrix of Eq. 4.1 (Section 4.2): sum_j c_j x_j y_j^T with
    c_j = gap/j for j <= r and 1/j for r < j <= n.

    The thesis calls x_j, y_j sparse and nonnegative without saying how they
    are drawn.  ``vectors="haar"`` takes orthonormal Haar columns, which makes
    c_j exactly the singular values; ``vectors="sparse"`` takes nonnegative
    vectors with density 0.1 and uniform entries, normalised to unit length
    (singular values then differ from c_j and are computed by the caller).
    """
    count = min(m, n)
    c = spectrum("gap", count, gap=gap, gap_at=r)
    if vectors == "haar":
        return lowrank_matrix(m, n, c, seed)
    if vectors == "sparse":
        rng = _rng(seed, _STREAM_SPARSE)
        x = rng.uniform(0.0, 1.0, (m, count)) * (rng.uniform(size=(m, count)) < 0.1)
        y = rng.uniform(0.0, 1.0, (n, count)) * (rng.uniform(size=(n, count)) < 0.1)
        x /= np.maximum(np.linalg.norm(x, axis=0), 1e-300)
        y /= np.maximum(np.linalg.norm(y, axis=0), 1e-300)
        return np.asfortranarray((x * c) @ y.T)
    raise ValueError(f"unknown vectors kind {vectors!r}")


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round FP64 values to the nearest BF16 (ties to even) and return them
    as FP64, so a BF16-stored matrix can be handed to an FP64 consumer
    exactly.  Goes through FP32 first; the double rounding FP64 -> FP32 ->
    BF16 matches what a device conversion of an FP32 value does."""
    f = np.asarray(a, dtype=np.float32)
    bits = f.view(np.uint32).astype(np.uint64)
    lsb = (bits >> 16) & 1
    rounded = ((bits + 0x7FFF + lsb) >> 16) << 16
    out = rounded.astype(np.uint32).view(np.float32).astype(np.float64)
    return out.reshape(a.shape, order="A")


# ---------------------------------------------------------------------------
# Device-side generation for the large workloads (torch used as plumbing:
# cuSOLVER/cuBLAS build the input, they are not part of the measured path).
# ---------------------------------------------------------------------------

def lowrank_matrix_torch(m: int, n: int, sigma: np.ndarray, seed: int, *,
                         device="cuda", dtype=None, factor_dtype=None,
                         noise_2norm: float = 0.0, lda: int | None = None):
    """Build A = U diag(sigma) V^T (+ E) on ``device`` with torch and return it
    column-major as a torch tensor of shape (n, lda) (row j holds column j).

    ``factor_dtype`` (default float64) is the precision of the Haar factors
    and of the product; ``dtype`` the stored type of A (default float64).
    The Gaussians of the Haar factors are drawn on the CPU from a seeded
    torch Generator; the noise floor, if any, from a seeded device Generator.
    """
    import torch

    factor_dtype = factor_dtype or torch.float64
    dtype = dtype or torch.float64
    lda = lda or m
    r = len(sigma)

    def haar(rows, cols, stream):
        g = torch.Generator(device="cpu")
        g.manual_seed((int(seed) * 1000003 + stream) & 0x7FFFFFFFFFFFFFFF)
        x = torch.randn(rows, cols, generator=g, dtype=torch.float32)
        x = x.to(device=device, dtype=factor_dtype)
        q, rr = torch.linalg.qr(x, mode="reduced")
        d = torch.sign(torch.diagonal(rr))
        d[d == 0] = 1
        return q * d

    u = haar(m, r, _STREAM_U)
    v = haar(n, r, _STREAM_V)
    s = torch.as_tensor(np.asarray(sigma), dtype=factor_dtype, device=device)
    # Column-major A stored as At (n x m row-major): At = V diag(s) U^T.
    at = (v * s) @ u.T
    del u, v
    if noise_2norm > 0.0:
        # the noise floor is drawn on the device (seeded); at 10^9 entries a
        # host draw would dominate the set-up time
        g = torch.Generator(device=device)
        g.manual_seed((int(seed) * 1000003 + _STREAM_NOISE) & 0x7FFFFFFFFFFFFFFF)
        scale = noise_2norm / (np.sqrt(m) + np.sqrt(n))
        for j0 in range(0, n, 1024):
            j1 = min(n, j0 + 1024)
            e = torch.randn(j1 - j0, m, generator=g, dtype=torch.float32, device=device)
            at[j0:j1] += (scale * e).to(factor_dtype)
    out = torch.zeros(n, lda, dtype=dtype, device=device)
    out[:, :m] = at.to(dtype)
    return out


def symmetric_matrix_torch(n: int, lam: np.ndarray, seed: int, *, device="cuda"):
    """Build A = U diag(lam) U^T (FP64, n x n, Haar U) on ``device`` with
    torch; A is symmetric, so its row-major and column-major storage agree.
    The Gaussians of U are drawn on the CPU from a seeded torch Generator."""
    import torch

    r = len(lam)
    g = torch.Generator(device="cpu")
    g.manual_seed((int(seed) * 1000003 + _STREAM_U) & 0x7FFFFFFFFFFFFFFF)
    x = torch.randn(n, r, generator=g, dtype=torch.float32).to(device=device, dtype=torch.float64)
    q, rr = torch.linalg.qr(x, mode="reduced")
    d = torch.sign(torch.diagonal(rr))
    d[d == 0] = 1
    u = q * d
    lt = torch.as_tensor(np.asarray(lam), dtype=torch.float64, device=device)
    a = (u * lt) @ u.T
    a = 0.5 * (a + a.T)
    return a.contiguous()


# ---------------------------------------------------------------------------
# FP8 E4M3 storage with one power-of-two scale per 128 x 128 tile
# ---------------------------------------------------------------------------

FP8_TILE = 128
FP8_MAX = 448.0


def quantize_e4m3_tiles(at, m: int, lda_q: int | None = None):
    """Stores a column-major matrix as E4M3 codes with per-tile scales.

    ``at``: torch tensor (n, >= m) whose row j is column j of A (any float
    dtype, any device).  Each 128 x 128 tile (I, J) gets the scale
    2^ceil(log2(amax / 448)) (1 for an all-zero tile), a power of two, so
    code * scale is exact in BF16 and FP32; codes are A / scale rounded to
    nearest even.  Returns (codes, scales): codes a uint8 tensor (n, lda_q)
    with lda_q a multiple of 16 (zero padded), scales an FP32 tensor
    (n_tiles, m_tiles) whose row J holds column J of the column-major
    m_tiles x n_tiles scale matrix (ld m_tiles)."""
    import torch

    n = at.shape[0]
    lda_q = lda_q or (m + 15) // 16 * 16
    mt, nt = (m + FP8_TILE - 1) // FP8_TILE, (n + FP8_TILE - 1) // FP8_TILE
    codes = torch.zeros(n, lda_q, dtype=torch.uint8, device=at.device)
    scales = torch.ones(nt, mt, dtype=torch.float32, device=at.device)
    for J in range(nt):
        j0, j1 = J * FP8_TILE, min(n, (J + 1) * FP8_TILE)
        blk = at[j0:j1, :m].to(torch.float64)
        # per-tile amax over the 128-row groups of A
        pad = mt * FP8_TILE - m
        absb = torch.nn.functional.pad(blk.abs(), (0, pad))
        amax = absb.reshape(j1 - j0, mt, FP8_TILE).amax(dim=(0, 2))
        e = torch.ceil(torch.log2(torch.clamp(amax, min=1e-300) / FP8_MAX))
        sc = torch.where(amax > 0, torch.pow(2.0, e), torch.ones_like(amax))
        scales[J] = sc.to(torch.float32)
        rows_scale = sc.repeat_interleave(FP8_TILE)[:m]
        q = (blk / rows_scale).to(torch.float8_e4m3fn)
        codes[j0:j1, :m] = q.view(torch.uint8)
    return codes, scales
