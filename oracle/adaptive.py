"""Adaptive randomized range finder (Adaptive_randRF of the toolbox, the
"adaptive" entry of Section 4's function list) in plain FP64 -- TEST
INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The thesis states what the function does: given A (m x n), a tolerance eps
and an integer r, it returns an orthonormal Q with ||(I - Q Q*) A|| <= eps
with probability at least 1 - min(m, n) 10^-r, and it names its source,
Algorithm 4.2 of Halko, Martinsson and Tropp (SIAM Review 53, 2011).  That
published algorithm is restated here, one Gaussian vector at a time, in its
own order:

  * draw r Gaussian vectors omega_1..omega_r, set y_i = A omega_i; j = 0,
    Q_0 empty;
  * while max(||y_{j+1}||, ..., ||y_{j+r}||) > eps / (10 sqrt(2/pi)):
      j = j + 1
      y_j <- (I - Q_{j-1} Q_{j-1}*) y_j           (re-projection)
      q_j = y_j / ||y_j||,  Q_j = [Q_{j-1} q_j]
      draw omega_{j+r},  y_{j+r} = (I - Q_j Q_j*) A omega_{j+r}
      y_i <- y_i - q_j (q_j* y_i)  for i = j+1 .. j+r-1
  * return Q_j.

The threshold eps / (10 sqrt(2/pi)) is the a-posteriori bound behind the
stated probability: for r Gaussian vectors, ||(I - QQ*) A|| <=
10 sqrt(2/pi) max_i ||(I - QQ*) A omega_i|| except with probability
min(m, n) 10^-r (Halko et al., Lemma 4.1).

Readings (the thesis is silent on these):
  * omega_i is column i-1 of the Philox Gaussian of stream 0 (the test
    matrix of every other algorithm here), so the vectors drawn do not
    depend on how many are drawn in the end;
  * the loop also ends when j reaches ``l_max`` (a capacity the caller
    sets, at most min(m, n)); ``converged`` then says whether the
    tolerance was met;
  * the rank-revealing SVD that follows (``adaptive_rsvd``) is Stage B of
    the prototype (Algorithm 1's B = Q* A, its SVD and U = Q U~) with every
    column of Q kept: the tolerance, not k, fixes the rank.

Library primitives used as steps: numpy's matrix-vector products and norms,
LAPACK's SVD for the small matrix.  Nothing is blocked or reordered.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .philox import gaussian_matrix
from .randsvd import sign_normalise

POSTERIOR_FACTOR = 10.0 * np.sqrt(2.0 / np.pi)


@dataclass
class AdaptiveRange:
    Q: np.ndarray            # m x j, orthonormal columns
    rank: int                # j
    converged: bool          # the tolerance test passed (else j hit l_max)
    threshold: float         # eps / (10 sqrt(2/pi))
    lookahead: list = field(default_factory=list)  # the max tested at j = 0, 1, ...


def threshold(eps: float) -> float:
    return eps / POSTERIOR_FACTOR


def adaptive_range_finder(A: np.ndarray, eps: float, r: int, seed: int,
                          l_max: int | None = None,
                          Omega: np.ndarray | None = None) -> AdaptiveRange:
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    cap = min(m, n) if l_max is None else min(l_max, m, n)
    if not (eps > 0 and r >= 1 and cap >= 1):
        raise ValueError("need eps > 0, r >= 1, l_max >= 1")
    if Omega is None:
        Omega = gaussian_matrix(n, cap + r, seed, stream=0)
    thr = threshold(eps)
    ys = [A @ Omega[:, i] for i in range(r)]
    Q = np.zeros((m, 0))
    j = 0
    looks = []
    converged = False
    while True:
        look = max(np.linalg.norm(ys[i]) for i in range(j, j + r))
        looks.append(look)
        if look <= thr:
            converged = True
            break
        if j == cap:
            break
        y = ys[j] - Q @ (Q.T @ ys[j])
        qj = y / np.linalg.norm(y)
        Q = np.column_stack([Q, qj])
        j += 1
        ynew = A @ Omega[:, j - 1 + r]
        ys.append(ynew - Q @ (Q.T @ ynew))
        for i in range(j, j - 1 + r):
            ys[i] = ys[i] - qj * (qj @ ys[i])
    return AdaptiveRange(Q=Q, rank=j, converged=converged, threshold=thr, lookahead=looks)


@dataclass
class AdaptiveSvd:
    U: np.ndarray
    S: np.ndarray
    Vt: np.ndarray
    range: AdaptiveRange


def adaptive_rsvd(A: np.ndarray, eps: float, r: int, seed: int,
                  l_max: int | None = None) -> AdaptiveSvd:
    """The adaptive range followed by Stage B: B = Q* A, B = U~ S V*,
    U = Q U~; rank = the number of columns the range finder kept."""
    A = np.asarray(A, dtype=np.float64)
    rf = adaptive_range_finder(A, eps, r, seed, l_max)
    if rf.rank == 0:
        return AdaptiveSvd(U=rf.Q, S=np.zeros(0), Vt=np.zeros((0, A.shape[1])), range=rf)
    B = rf.Q.T @ A
    Ut, S, Vt = np.linalg.svd(B, full_matrices=False)
    U, Vt = sign_normalise(rf.Q @ Ut, Vt)
    return AdaptiveSvd(U=U, S=S, Vt=Vt, range=rf)
