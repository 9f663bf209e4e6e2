"""Two-stage (successive band) reduction of the skew-symmetric W to tridiagonal
form, FP64 numpy. The first "next" step after Algorithm 3's one-stage reduction
(Section 6 names band reduction as the way to cut the memory-bound SYMV of
Algorithm 3 step 1).

Test infrastructure only (see the package docstring). Plain, unblocked steps;
library primitives used as steps: numpy QR and matmul.

  stage 1 (dense -> band of half-bandwidth b): for the panels of b columns
      k = 0, b, 2b, ...: the block W[k+b:, k:k+b] below the band is QR-factored,
      P = Q_k R, and W <- Q_k^T W Q_k on the rows/columns k+b..m-1, which leaves
      R (upper triangular, inside the band) and zeros below it;
  stage 2 (band -> tridiagonal): Schwarz's bulge chase with plane rotations --
      for each column j, the entries (k, j), k = j+b down to j+2, are annihilated
      by a rotation in the plane (k-1, k); each rotation creates one entry outside
      the band at (k+b, k-1) (and its mirror), which a rotation in the plane
      (k+b-1, k+b) moves b rows further down until it leaves the matrix.

Both stages are orthogonal similarities, so skew symmetry is kept and
W = Q T Q^T with Q = Q1 Q2. Neither touches index 0, so Q e_1 = e_1: by the
implicit-Q theorem the sub-diagonal magnitudes of T equal those of Algorithm 3's
one-stage reduction (unreduced case), which the pins check.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class TwoStage:
    Bw: np.ndarray  # band matrix after stage 1
    Q1: np.ndarray
    T: np.ndarray   # skew tridiagonal after stage 2
    Q2: np.ndarray


def dense_to_band(W: np.ndarray, b: int) -> tuple[np.ndarray, np.ndarray]:
    """Stage 1: B = Q1^T W Q1 with B[i, j] = 0 for |i - j| > b."""
    A = np.array(W, dtype=np.float64)
    m = A.shape[0]
    Q = np.eye(m)
    for k in range(0, m, b):
        r0 = k + b
        if r0 >= m - 1:
            break
        kb = min(b, m - k)
        P = A[r0:, k:k + kb]
        Qk, _ = np.linalg.qr(P, mode="complete")
        A[r0:, :] = Qk.T @ A[r0:, :]
        A[:, r0:] = A[:, r0:] @ Qk
        Q[:, r0:] = Q[:, r0:] @ Qk
    return A, Q


def _rotate(A: np.ndarray, Q: np.ndarray, p: int, q: int, col: int) -> None:
    """Plane rotation G on rows/columns (p, q) with (G^T A G)[q, col] = 0."""
    a, c = A[p, col], A[q, col]
    r = np.hypot(a, c)
    if r == 0.0:
        return
    cs, sn = a / r, c / r
    G = np.array([[cs, -sn], [sn, cs]])  # columns: new basis vectors in the (p, q) plane
    idx = [p, q]
    A[idx, :] = G.T @ A[idx, :]
    A[:, idx] = A[:, idx] @ G
    Q[:, idx] = Q[:, idx] @ G


def band_to_tridiagonal(B: np.ndarray, b: int) -> tuple[np.ndarray, np.ndarray]:
    """Stage 2: T = Q2^T B Q2 tridiagonal, by rotations and bulge chasing."""
    A = np.array(B, dtype=np.float64)
    m = A.shape[0]
    Q = np.eye(m)
    for j in range(m - 2):
        for k in range(min(j + b, m - 1), j + 1, -1):
            _rotate(A, Q, k - 1, k, j)
            p = k
            while p + b < m:  # the rotation in (p-1, p) filled (p+b, p-1)
                q = p + b
                _rotate(A, Q, q - 1, q, p - 1)
                p = q
    return A, Q


def two_stage(W: np.ndarray, b: int) -> TwoStage:
    Bw, Q1 = dense_to_band(W, b)
    T, Q2 = band_to_tridiagonal(Bw, b)
    return TwoStage(Bw=Bw, Q1=Q1, T=T, Q2=Q2)
