"""Single-pass randomized eigendecomposition of a Hermitian matrix
(Algorithm 5, Section 3.4.1) in plain FP64 -- TEST INFRASTRUCTURE ONLY (see
``oracle/__init__.py``).

Steps in the thesis' order and notation, l = k + p, A real symmetric n x n
(the real case of Hermitian):

  Stage 1
    1. Gaussian Omega (n x l, Philox stream 0, as Omega in Algorithm 4)
    2. Y = A Omega                                   (the only pass over A)
    3. Q: the orthonormal matrix formed from Y
  Stage 2
    4. C (k x k): the solution of C (Q* Omega) = Q* Y          (Eq. 3.13)
    5. C = U^ D U^*  (eigendecomposition of the small matrix)
    6. U = Q U^

Readings (the listing is inconsistent on sizes and silent on the rest):
  * step 3 / step 4: C is called k x k, which needs Q to have k columns,
    while orth(Y) has l.  As in Algorithm 6 (whose listing says so), Q is
    the k dominant left singular vectors of Y.  Q* Omega and Q* Y are then
    k x l, and step 4 is an overdetermined system (l equations per row of
    C), solved in least squares: min ||C (Q* Omega) - Q* Y||_F.
  * step 5 names an eigendecomposition U^ D U^*, which needs a Hermitian C.
    The solved C is Hermitian only up to the approximation error of
    Eq. 3.12, so the oracle takes its Hermitian part (C + C*)/2, the nearest
    Hermitian matrix in the Frobenius norm, before the decomposition.
  * order and signs: A may be indefinite; the rank-k output keeps the k
    eigenvalues of C of largest magnitude, sorted by decreasing |lambda|
    (the Hermitian form of the truncation of Section 3.1).  Each
    eigenvector is flipped so that its largest-magnitude entry is positive
    (lowest index on ties), the sign rule of Algorithm 4's oracle.

Library primitives used as steps: matrix products, LAPACK's SVD (step 3),
its least-squares solver (step 4) and its symmetric eigensolver (step 5).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .philox import gaussian_matrix


@dataclass
class HermitianResult:
    U: np.ndarray      # n x k, orthonormal columns
    D: np.ndarray      # k eigenvalues, |D| descending
    C: np.ndarray      # k x k, the least-squares solution of step 4 (before symmetrising)
    Q: np.ndarray      # n x k


def dominant_left(Y: np.ndarray, k: int) -> np.ndarray:
    """Step 3: the k dominant left singular vectors of Y (LAPACK SVD)."""
    u, _, _ = np.linalg.svd(Y, full_matrices=False)
    return u[:, :k]


def solve_step4(Qt_Omega: np.ndarray, Qt_Y: np.ndarray) -> np.ndarray:
    """Step 4: C minimising ||C (Q* Omega) - Q* Y||_F, i.e. the least squares
    of the transposed system (Q* Omega)^T C^T = (Q* Y)^T (LAPACK)."""
    return np.linalg.lstsq(Qt_Omega.T, Qt_Y.T, rcond=None)[0].T


def _sign_columns(U: np.ndarray) -> np.ndarray:
    idx = np.argmax(np.abs(U), axis=0)
    s = np.sign(U[idx, np.arange(U.shape[1])])
    s[s == 0] = 1.0
    return U * s


def hermitian_singlepass(A: np.ndarray, k: int, p: int, seed: int,
                         Omega: np.ndarray | None = None) -> HermitianResult:
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    if A.shape != (n, n):
        raise ValueError("Algorithm 5 takes a square (Hermitian) matrix")
    l = k + p
    if not (1 <= k and p >= 0 and l <= n):
        raise ValueError("need 1 <= k, p >= 0, k+p <= n")
    if Omega is None:
        Omega = gaussian_matrix(n, l, seed, stream=0)       # step 1
    Y = A @ Omega                                            # step 2
    Q = dominant_left(Y, k)                                  # step 3
    C = solve_step4(Q.T @ Omega, Q.T @ Y)                    # step 4
    lam, Uh = np.linalg.eigh(0.5 * (C + C.T))                # step 5
    order = np.argsort(-np.abs(lam), kind="stable")
    lam, Uh = lam[order], Uh[:, order]
    U = _sign_columns(Q @ Uh)                                # step 6
    return HermitianResult(U=U, D=lam, C=C, Q=Q)
