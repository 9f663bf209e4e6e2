"""Algorithm 2 (real Bethe--Salpeter problems, Section 3.2, Theorem 5), FP64 numpy.

Test infrastructure only (see the package docstring). The steps in the paper's
order and notation; library primitives used as steps: numpy Cholesky and SVD.

  1. A + B = L1 L1^T,  A - B = L2 L2^T
  2. L2^T L1 = U Lambda+ V^T  (singular value decomposition)
  3. X1 = (L2 U + L1 V),  X2 = (L2 U - L1 V), each times (1/2) Lambda+^{-1/2}

Reading: the algorithm's step 3 prints X1, X2 without the factor
(1/2) Lambda+^{-1/2} that Theorem 5's X carries; with it X1^T X1 - X2^T X2 = I
(the normalization the algorithm promises), without it not, so the factor is
applied. Eigenvalues are returned ascending (the SVD gives them descending).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class RealSolution:
    lam: np.ndarray  # n, ascending
    X1: np.ndarray   # n x n
    X2: np.ndarray   # n x n


def symmetrize_real(A: np.ndarray, B: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Full symmetric A, B from their lower triangles (LAPACK 'L' convention)."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    Af = np.tril(A) + np.tril(A, -1).T
    Bf = np.tril(B) + np.tril(B, -1).T
    return Af, Bf


def step1_cholesky(A: np.ndarray, B: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """A + B = L1 L1^T and A - B = L2 L2^T (both must be positive definite)."""
    return np.linalg.cholesky(A + B), np.linalg.cholesky(A - B)


def step2_svd(L1: np.ndarray, L2: np.ndarray):
    """L2^T L1 = U diag(s) V^T."""
    U, s, Vt = np.linalg.svd(L2.T @ L1)
    return U, s, Vt.T


def step3_vectors(L1, L2, U, s, V) -> tuple[np.ndarray, np.ndarray]:
    """X1 = (1/2)(L2 U + L1 V) Lambda^{-1/2},  X2 = (1/2)(L2 U - L1 V) Lambda^{-1/2}."""
    a, b = L2 @ U, L1 @ V
    f = 0.5 / np.sqrt(s)
    return (a + b) * f[None, :], (a - b) * f[None, :]


def solve_real(A: np.ndarray, B: np.ndarray) -> RealSolution:
    A, B = symmetrize_real(A, B)
    L1, L2 = step1_cholesky(A, B)
    U, s, V = step2_svd(L1, L2)
    X1, X2 = step3_vectors(L1, L2, U, s, V)
    order = np.argsort(s)
    return RealSolution(lam=s[order], X1=X1[:, order], X2=X2[:, order])
