"""Single-pass randomized SVD of a general matrix (Algorithm 6, Section 3.4.2)
in plain FP64 -- TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Steps in the thesis' order and notation, l = k + p:

  1. Gaussian Omega_c (n x l, Philox stream 0) and Omega_r (m x l, stream 1)
  2. Y_c = A Omega_c, Y_r = A* Omega_r
  3. Q_c, Q_r: the k dominant left singular vectors of Y_c and Y_r
  4. C (k x k): least-squares solution of the joint system
         (Omega_r* Q_c) C = Y_r* Q_r   and   C (Q_r* Omega_c) = Q_c* Y_c
  5. C = U^ Sigma V^*  (SVD of the small matrix)
  6. U = Q_c U^, V = Q_r V^

Readings (the thesis' listing is garbled or silent on these):
  * step 2 lists "Y_r = A Omega_r"; Omega_r is m x (k+p) and the text derives
    Y_r = A* Omega_r, the only product the dimensions allow for m != n.
  * step 4 does not weight the two equations; "the least-squares solution of
    the joint system" is read as minimising the sum of both squared
    Frobenius residuals with equal weights, with M = Omega_r* Q_c,
    P = Y_r* Q_r, N = Q_r* Omega_c, R = Q_c* Y_c.  The oracle writes that
    definition out: both equations vectorised (column-major vec, so
    vec(M C) = (I kron M) vec C and vec(C N) = (N^T kron I) vec C), stacked
    into one (2 l k) x k^2 system and handed to LAPACK's least-squares
    solver.  No normal equations are formed.
  * Omega_r comes from Philox stream 1 of the same seed (the thesis draws
    the two matrices independently and names no generator).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .philox import gaussian_matrix
from .randsvd import sign_normalise


@dataclass
class SinglePassResult:
    U: np.ndarray      # m x k
    S: np.ndarray      # k, descending
    Vt: np.ndarray     # k x n
    C: np.ndarray      # k x k, the joint least-squares solution (step 4)
    Qc: np.ndarray     # m x k
    Qr: np.ndarray     # n x k


def dominant_left(Y: np.ndarray, k: int) -> np.ndarray:
    """Step 3: the k dominant left singular vectors of Y (LAPACK SVD)."""
    u, _, _ = np.linalg.svd(Y, full_matrices=False)
    return u[:, :k]


def joint_lstsq(M, P, N, R) -> np.ndarray:
    """Step 4: C minimising ||M C - P||_F^2 + ||C N - R||_F^2 (M: l x k,
    P: l x k, N: k x l, R: k x l), as the stacked least-squares problem
    [I kron M ; N^T kron I] vec C = [vec P ; vec R] (column-major vec)."""
    k = M.shape[1]
    K = np.vstack([np.kron(np.eye(k), M), np.kron(N.T, np.eye(k))])
    rhs = np.concatenate([P.flatten("F"), R.flatten("F")])
    c = np.linalg.lstsq(K, rhs, rcond=None)[0]
    return c.reshape(k, k, order="F")


def singlepass_rsvd(A: np.ndarray, k: int, p: int, seed: int,
                    Omega_c: np.ndarray | None = None,
                    Omega_r: np.ndarray | None = None) -> SinglePassResult:
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    l = k + p
    if not (1 <= k and p >= 0 and l <= min(m, n)):
        raise ValueError("need 1 <= k, p >= 0, k+p <= min(m, n)")
    if Omega_c is None:
        Omega_c = gaussian_matrix(n, l, seed, stream=0)       # step 1
    if Omega_r is None:
        Omega_r = gaussian_matrix(m, l, seed, stream=1)
    Yc = A @ Omega_c                                          # step 2
    Yr = A.T @ Omega_r
    Qc = dominant_left(Yc, k)                                 # step 3
    Qr = dominant_left(Yr, k)
    M = Omega_r.T @ Qc                                        # step 4
    P = Yr.T @ Qr
    N = Qr.T @ Omega_c
    R = Qc.T @ Yc
    C = joint_lstsq(M, P, N, R)
    Uh, S, Vht = np.linalg.svd(C)                             # step 5
    U = Qc @ Uh                                               # step 6
    V = Qr @ Vht.T
    U, Vt = sign_normalise(U, V.T)
    return SinglePassResult(U=U, S=S, Vt=Vt, C=C, Qc=Qc, Qr=Qr)
