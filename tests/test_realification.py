"""The two facts the GPU's complex steps rest on, checked in numpy (no GPU,
no oracle): the SRFT path orthonormalises and decomposes complex matrices
with the library's real kernels.

1. Interleaved realification (each entry z as [[Re z, -Im z], [Im z, Re z]])
   of the complex Cholesky factor R of an Hermitian positive definite G is
   real, upper triangular with a positive diagonal, and its normal product
   is the realified G -- so it IS the real Cholesky factor of the realified
   G, and the inverse read from its even columns is R^-1 (complex
   CholeskyQR through real kernels).
2. The block realification [[Re M, -Im M], [Im M, Re M]] of a complex
   matrix has every singular value of M twice, and column 2i of either
   real singular factor (after sorting) is [Re x ; Im x] for a singular
   vector x of M up to a unit factor (the complex small SVD of Stage B).
"""
import numpy as np


def _interleave(Z):
    n, m = Z.shape
    out = np.zeros((2 * n, 2 * m))
    out[0::2, 0::2] = Z.real
    out[0::2, 1::2] = -Z.imag
    out[1::2, 0::2] = Z.imag
    out[1::2, 1::2] = Z.real
    return out


def test_complex_cholesky_is_the_real_cholesky_of_the_realification():
    rng = np.random.default_rng(0)
    for l in (1, 5, 17):
        Y = rng.standard_normal((60, l)) + 1j * rng.standard_normal((60, l))
        G = Y.conj().T @ Y
        Rc = np.linalg.cholesky(G).conj().T             # G = Rc^H Rc, Rc upper
        Rr = np.linalg.cholesky(_interleave(G)).T       # real upper factor
        assert np.abs(Rr - _interleave(Rc)).max() <= 1e-12 * np.abs(Rr).max()
        # R^-1 from the even columns of the real inverse
        Xi = np.linalg.inv(Rr)
        S = Xi[0::2, 0::2] + 1j * Xi[1::2, 0::2]
        assert np.abs(S @ Rc - np.eye(l)).max() <= 1e-10
        # Q = Y R^-1 in planar form: [Re Q | Im Q] = [Re Y | Im Y] [[S_re, S_im], [-S_im, S_re]]
        C = np.block([[S.real, S.imag], [-S.imag, S.real]])
        Qp = np.hstack([Y.real, Y.imag]) @ C
        Q = Qp[:, :l] + 1j * Qp[:, l:]
        assert np.abs(Q.conj().T @ Q - np.eye(l)).max() <= 1e-10


def test_block_realification_svd_pairs():
    rng = np.random.default_rng(1)
    l = 12
    M = rng.standard_normal((l, l)) + 1j * rng.standard_normal((l, l))
    MR = np.block([[M.real, -M.imag], [M.imag, M.real]])
    UR, sR, VRt = np.linalg.svd(MR)
    s = np.linalg.svd(M, compute_uv=False)
    assert np.abs(sR[0::2] - s).max() <= 1e-12 * s[0]
    assert np.abs(sR[1::2] - s).max() <= 1e-12 * s[0]
    VR = VRt.T
    for i in range(l):
        x = UR[:l, 2 * i] + 1j * UR[l:, 2 * i]
        w = VR[:l, 2 * i] + 1j * VR[l:, 2 * i]
        assert abs(np.linalg.norm(x) - 1) <= 1e-12
        assert np.abs(M @ w - s[i] * x).max() <= 1e-10 * s[0]
