"""Randomized SVD, Algorithms 1-4 of the thesis, in plain FP64 -- oracle side.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Steps follow the thesis in its order and notation:

  Algorithm 4 (Section 3.3, RSVD with orthonormalisation):
    1. Omega: n x (k+p) Gaussian test matrix
    2. Y = A Omega
    3. Q = orth(Y)
    4-5. for j = 1..q:  W = orth(A* Q);  Q = orth(A W)
    6. B = Q* A
    7. B = U~ Sigma V*  (SVD of the small matrix)
    8. U = Q U~
  then keep the leading k triplets (Section 3.1: truncate the last p
  components after the small SVD).

  Algorithm 2 (Section 3.1) is Algorithm 4 with q = 0.
  Algorithm 3 (Section 3.2) multiplies by A* and A q times without
  orthonormalising in between, then orthonormalises once.
  Algorithm 1 (Section 2.2) is steps 1-3 alone (the range finder).

Library primitives used as steps: numpy's matrix product, LAPACK's
Householder QR (``orth``; any orthonormal basis of range(Y) is admissible,
the thesis does not fix the method) and LAPACK's SVD for step 7.  Nothing is
blocked, fused or reordered.  The GPU path uses none of these: CholeskyQR2
for orth and a one-sided Jacobi SVD for step 7, so agreement between the two
is evidence about the method, not about a shared routine.

Sign convention (the thesis leaves it open; singular vectors are unique only
up to sign): after sorting sigma descending, each pair (u_i, v_i) is flipped
so that the entry of u_i with the largest magnitude is positive (lowest
index on ties).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .philox import gaussian_matrix


@dataclass
class RsvdResult:
    U: np.ndarray        # m x k, orthonormal columns
    S: np.ndarray        # k, descending
    Vt: np.ndarray       # k x n, orthonormal rows
    Q: np.ndarray        # m x (k+p), the range basis of Stage 1
    Omega: np.ndarray    # n x (k+p), the test matrix of step 1


def orth(Y: np.ndarray) -> np.ndarray:
    """Orthonormal basis of range(Y) (thin Householder QR, LAPACK)."""
    q, _ = np.linalg.qr(Y, mode="reduced")
    return q


def small_svd(B: np.ndarray):
    """Step 7: SVD of the small (k+p) x n matrix B (LAPACK)."""
    return np.linalg.svd(B, full_matrices=False)


def sign_normalise(U: np.ndarray, Vt: np.ndarray):
    """Flip (u_i, v_i) so u_i's largest-magnitude entry is positive."""
    U = U.copy()
    Vt = Vt.copy()
    idx = np.argmax(np.abs(U), axis=0)
    s = np.sign(U[idx, np.arange(U.shape[1])])
    s[s == 0] = 1.0
    return U * s, Vt * s[:, None]


def range_finder(A: np.ndarray, l: int, q: int, seed: int,
                 algorithm: int = 4, Omega: np.ndarray | None = None):
    """Stage 1: returns (Q, Omega).

    algorithm=4: orthonormalise after every product (Algorithm 4, steps 1-5);
    algorithm=3: q plain power steps then one orth (Algorithm 3, steps 1-5);
    algorithm=1 or 2: q is ignored (Algorithm 1 / Algorithm 2 Stage 1).
    """
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    if Omega is None:
        Omega = gaussian_matrix(n, l, seed)              # step 1
    Y = A @ Omega                                        # step 2
    if algorithm in (1, 2):
        return orth(Y), Omega                            # step 3
    if algorithm == 3:
        for _ in range(q):                               # Algorithm 3, step 4
            Z = A.T @ Y
            Y = A @ Z
        return orth(Y), Omega                            # Algorithm 3, step 5
    if algorithm == 4:
        Q = orth(Y)                                      # step 3
        for _ in range(q):                               # steps 4-5
            W = orth(A.T @ Q)
            Q = orth(A @ W)
        return Q, Omega
    raise ValueError(f"unknown algorithm {algorithm}")


def rsvd(A: np.ndarray, k: int, p: int, q: int, seed: int,
         algorithm: int = 4, Omega: np.ndarray | None = None,
         truncate: bool = True) -> RsvdResult:
    """Rank-k randomized SVD of A (Algorithm 4 by default).

    Returns U (m x k), S (k), Vt (k x n) sign-normalised; with
    ``truncate=False`` all k+p triplets are returned.
    """
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    l = k + p
    if not (1 <= k and p >= 0 and l <= min(m, n) and q >= 0):
        raise ValueError("need 1 <= k, p >= 0, k+p <= min(m, n), q >= 0")
    Q, Omega = range_finder(A, l, q, seed, algorithm, Omega)
    B = Q.T @ A                                          # step 6
    Ut, S, Vt = small_svd(B)                             # step 7
    U = Q @ Ut                                           # step 8
    if truncate:                                         # keep rank k
        U, S, Vt = U[:, :k], S[:k], Vt[:k]
    U, Vt = sign_normalise(U, Vt)
    return RsvdResult(U=U, S=S.copy(), Vt=Vt, Q=Q, Omega=Omega)
