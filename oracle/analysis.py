"""Error measures and the thesis' bounds -- oracle side.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* ``spectral_norm``: ||M||_2 of an explicit or implicit matrix; exact (LAPACK
  singular values) for small matrices, Golub-Kahan-Lanczos bidiagonalisation
  with full reorthogonalisation and a fixed start vector for large ones.
* ``range_error``: ||A - Q Q* A||_2, the quantity bounded in Theorems 2, 3, 6.
* ``lowrank_residual``: ||A - U Sigma V*||_2 of a rank-k factorisation.
* ``sin_canonical_angles``: sines of the canonical angles between two
  subspaces (Eq. 4.3), ascending.
* Bounds: Theorem 2 (Section 3.1), Theorem 3 (Section 3.2), Theorem 6 =
  Eq. 3.4 and its flat-tail form Eq. 3.5 (Section 3.3), and the
  canonical-angle bounds of Theorem 5 under Assumption 4 (Section 3.2).

Readings where the text is silent or garbled:
* Theorem 5 uses gamma_j without defining it (Assumption 4 defines only
  gamma_k = sigma_{k+1}/sigma_k); gamma_j = sigma_{k+1}/sigma_j is taken,
  which reduces to gamma_k at j = k.
* Theorem 5's theta_j are read as the canonical angles between range(U_k)
  and the computed range, sorted ascending so that the j-th bound (which
  grows with j) pairs with the j-th smallest angle.
"""
from __future__ import annotations

import math

import numpy as np


def spectral_norm(matvec, rmatvec, shape, iters: int = 80, seed: int = 12345,
                  tol: float = 1e-12) -> float:
    """Largest singular value of the operator (matvec, rmatvec) of ``shape``
    (m, n) by Golub-Kahan-Lanczos bidiagonalisation with full
    reorthogonalisation; stops when the estimate changes by < tol relative."""
    m, n = shape
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(n)
    v /= np.linalg.norm(v)
    Vs, Us, alphas, betas = [v], [], [], []
    u = matvec(v)
    est_prev = 0.0
    est = 0.0
    for j in range(min(iters, m, n)):
        for w in Us:
            u -= (w @ u) * w
        a = np.linalg.norm(u)
        if a == 0.0:
            break
        u = u / a
        Us.append(u)
        alphas.append(a)
        # singular values of the (j+1) x (j+1) upper bidiagonal matrix
        kk = len(alphas)
        Bm = np.diag(alphas)
        if betas:
            Bm[np.arange(kk - 1), np.arange(1, kk)] = betas[:kk - 1]
        est = float(np.linalg.svd(Bm, compute_uv=False)[0])
        if j > 2 and abs(est - est_prev) <= tol * est:
            break
        est_prev = est
        v = rmatvec(u) - a * Vs[-1]
        for w in Vs:
            v -= (w @ v) * w
        b = np.linalg.norm(v)
        if b == 0.0:
            break
        v = v / b
        Vs.append(v)
        betas.append(b)
        u = matvec(v) - b * u
    return est


def _norm2(M: np.ndarray, exact_limit: int = 4_000_000) -> float:
    if M.size <= exact_limit:
        return float(np.linalg.norm(M, 2))
    return spectral_norm(lambda x: M @ x, lambda y: M.T @ y, M.shape)


def range_error(A: np.ndarray, Q: np.ndarray, exact_limit: int = 4_000_000) -> float:
    """||A - Q Q^T A||_2 (Theorems 2, 3, 6)."""
    A = np.asarray(A, dtype=np.float64)
    if A.size <= exact_limit:
        return float(np.linalg.norm(A - Q @ (Q.T @ A), 2))
    return spectral_norm(lambda x: A @ x - Q @ (Q.T @ (A @ x)),
                         lambda y: A.T @ y - A.T @ (Q @ (Q.T @ y)), A.shape)


def lowrank_residual(A: np.ndarray, U: np.ndarray, S: np.ndarray, Vt: np.ndarray,
                     exact_limit: int = 4_000_000) -> float:
    """||A - U diag(S) Vt||_2."""
    A = np.asarray(A, dtype=np.float64)
    if A.size <= exact_limit:
        return float(np.linalg.norm(A - (U * S) @ Vt, 2))
    return spectral_norm(lambda x: A @ x - U @ (S * (Vt @ x)),
                         lambda y: A.T @ y - Vt.T @ (S * (U.T @ y)), A.shape)


def sin_canonical_angles(X: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """Sines of the canonical angles between range(X) and range(Y) (X, Y with
    orthonormal columns, dim X <= dim Y), ascending (Eq. 4.3)."""
    R = X - Y @ (Y.T @ X)
    s = np.linalg.svd(R, compute_uv=False)
    return np.sort(np.clip(s, 0.0, 1.0))


# ---------------------------------------------------------------------------
# Bounds
# ---------------------------------------------------------------------------

def thm2_bound(sigma: np.ndarray, k: int, p: int, m: int, n: int) -> float:
    """Theorem 2: E||A - QQ*A|| <= [1 + 4 sqrt(k+p)/(p-1) sqrt(min(m,n))] sigma_{k+1}."""
    return (1.0 + 4.0 * math.sqrt(k + p) / (p - 1) * math.sqrt(min(m, n))) * sigma[k]


def thm3_bound(sigma: np.ndarray, k: int, p: int, q: int, m: int, n: int) -> float:
    """Theorem 3: the Theorem 2 factor raised to 1/(2q+1)."""
    fac = 1.0 + 4.0 * math.sqrt((k + p) * min(m, n)) / (p - 1)
    return fac ** (1.0 / (2 * q + 1)) * sigma[k]


def thm6_bound(sigma: np.ndarray, k: int, p: int, q: int) -> float:
    """Theorem 6, Eq. 3.4 (sigma holds all min(m, n) singular values)."""
    e = 2 * q + 1
    tail = math.sqrt(float(np.sum(sigma[k:] ** (2 * e))))
    inner = (1.0 + math.sqrt(k / (p - 1))) * sigma[k] ** e \
        + math.e * math.sqrt(k + p) / p * tail
    return inner ** (1.0 / e)


def eq35_bound(sigma_k1: float, k: int, p: int, q: int, m: int, n: int) -> float:
    """Eq. 3.5: Theorem 6 when sigma_{k+1} = ... = sigma_min(m,n)."""
    e = 2 * q + 1
    fac = (1.0 + math.sqrt(k / (p - 1))) \
        + math.e * math.sqrt(k + p) / p * math.sqrt(min(m, n) - k)
    return fac ** (1.0 / e) * sigma_k1


def thm5_bounds(V: np.ndarray, Omega: np.ndarray, sigma: np.ndarray, k: int, q: int):
    """Theorem 5 bounds on sin theta_j (left) and sin nu_j (right), j = 1..k.

    V holds all right singular vectors of A as columns (n x n, or n x r when
    A has exact rank r -- then V_perp spans the rest and Omega_2 uses the
    orthogonal complement).  Omega_1 = V_k^T Omega, Omega_2 = V_perp^T Omega.
    """
    n = V.shape[0]
    Vk = V[:, :k]
    Om1 = Vk.T @ Omega
    # Omega_2: component of Omega outside range(V_k); its 2-norm structure is
    # that of V_perp^T Omega for any orthonormal completion V_perp.
    R = Omega - Vk @ Om1
    c = float(np.linalg.norm(R @ np.linalg.pinv(Om1), 2))
    j = np.arange(1, k + 1)
    gam = sigma[k] / sigma[j - 1]
    bu = gam ** (2 * q + 1) * c / np.sqrt(1.0 + gam ** (4 * q + 2) * c * c)
    bv = gam ** (2 * q + 2) * c / np.sqrt(1.0 + gam ** (4 * q + 4) * c * c)
    return bu, bv
