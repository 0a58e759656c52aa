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
   matrix has every singular value of M twice.  When the singular values of
   M are distinct, column 2i of either real singular factor (after sorting)
   is [Re x ; Im x] for a singular vector x of M up to a unit factor.  When
   they repeat, a real column may be any unit vector of the combined
   subspace, and picking by position can return the same complex vector
   twice (times i).  Stage B therefore picks by structure: real columns in
   order, each orthogonalised as a complex vector against those accepted,
   kept when more than half its norm remains, with the same complex
   coefficients applied to the right vectors.  Both the precondition and
   the structural rule are checked here.
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


def _select_pairs(UR, VR, sR, l, k):
    """The structural pairing rule of Stage B (a test-side restatement)."""
    Z, W, S = [], [], []
    for c in range(2 * l):
        if len(Z) == k:
            break
        x = UR[:l, c] + 1j * UR[l:, c]
        y = VR[:l, c] + 1j * VR[l:, c]
        for _ in range(2):
            if Z:
                Zm, Wm = np.array(Z).T, np.array(W).T
                a = Zm.conj().T @ x
                x = x - Zm @ a
                y = y - Wm @ a
        nrm = np.linalg.norm(x)
        if nrm > 0.5:
            Z.append(x / nrm)
            W.append(y / nrm)
            S.append(sR[c])
    return np.array(Z).T, np.array(W).T, np.array(S)


def _matrix_with_singular_values(sig, seed):
    rng = np.random.default_rng(seed)
    l = len(sig)
    U, _ = np.linalg.qr(rng.standard_normal((l, l)) + 1j * rng.standard_normal((l, l)))
    V, _ = np.linalg.qr(rng.standard_normal((l, l)) + 1j * rng.standard_normal((l, l)))
    return (U * sig) @ V.conj().T


def _realified_svd(M):
    MR = np.block([[M.real, -M.imag], [M.imag, M.real]])
    UR, sR, VRt = np.linalg.svd(MR)
    return UR, sR, VRt.T


def test_structural_pairing_with_repeated_singular_values():
    sig = np.array([3.0, 2.0, 2.0, 1.0, 1.0, 1.0, 0.5, 0.1])
    l = len(sig)
    for seed in range(5):
        M = _matrix_with_singular_values(sig, seed)
        UR, sR, VR = _realified_svd(M)
        Z, W, S = _select_pairs(UR, VR, sR, l, l)
        assert np.abs(S - sig).max() <= 1e-12 * sig[0]
        assert np.abs(Z.conj().T @ Z - np.eye(l)).max() <= 1e-12
        assert np.abs(W.conj().T @ W - np.eye(l)).max() <= 1e-12
        assert np.abs(M @ W - Z * S).max() <= 1e-12 * sig[0]
        assert np.abs((Z * S) @ W.conj().T - M).max() <= 1e-12 * sig[0]


def test_positional_pairing_fails_on_repeated_singular_values():
    """The precondition of picking column 2i: distinct singular values.  A
    real SVD of the realification is free to return, for a repeated value,
    the column pair (z, i z) of one complex vector and then (w, i w) of a
    second one in either real order; a basis in which column 2i and 2i+2 are
    z and i z (as an SVD routine may return) breaks the positional rule,
    while the structural rule recovers an orthonormal pair."""
    sig = np.array([2.0, 2.0, 1.0])
    l = len(sig)
    M = _matrix_with_singular_values(sig, 7)
    UR, sR, VR = _realified_svd(M)
    # reorder the four real columns of sigma = 2 as (z, w, i z, i w): an
    # equally valid real SVD of the realification
    z = UR[:, 0]
    jz = np.concatenate([-z[l:], z[:l]])          # multiplication by i
    a = VR[:, 0]
    ja = np.concatenate([-a[l:], a[:l]])
    rest_u = UR[:, :4] - np.outer(z, z @ UR[:, :4]) - np.outer(jz, jz @ UR[:, :4])
    w = np.linalg.svd(rest_u)[0][:, 0]           # a unit vector of the remaining 2-D part
    jw = np.concatenate([-w[l:], w[:l]])
    # right vectors of w and i w through M_R^T (same sigma)
    MR = np.block([[M.real, -M.imag], [M.imag, M.real]])
    b, jb = MR.T @ w / 2.0, MR.T @ jw / 2.0
    U2 = UR.copy()
    V2 = VR.copy()
    U2[:, :4] = np.stack([z, w, jz, jw], axis=1)
    V2[:, :4] = np.stack([a, b, ja, jb], axis=1)
    assert np.abs(MR @ V2 - U2 * sR).max() <= 1e-12 * sR[0]     # still an SVD of M_R
    picked = U2[:l, 0::2] + 1j * U2[l:, 0::2]                     # positional rule
    assert np.abs(picked.conj().T @ picked - np.eye(l)).max() > 0.5
    Z, W, S = _select_pairs(U2, V2, sR, l, l)                     # structural rule
    assert np.abs(Z.conj().T @ Z - np.eye(l)).max() <= 1e-12
    assert np.abs(M @ W - Z * S).max() <= 1e-12 * sig[0]
