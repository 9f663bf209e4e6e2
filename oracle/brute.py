"""Brute-force eigen-decomposition of H in 50-digit arithmetic (mpmath), n <= 4.

Test infrastructure only (see the package docstring). It builds H of Eq. 1
entry by entry and hands it to mpmath's general (non-Hermitian) eigensolver,
so it shares nothing with the pencil route of :mod:`oracle.definition`.
"""
from __future__ import annotations

import mpmath as mp
import numpy as np


def eig_H(A: np.ndarray, B: np.ndarray, dps: int = 50):
    """All 2n eigenvalues and right eigenvectors of H = [A B; -conj(B) -conj(A)].

    Returns (eigenvalues as a list of mpc sorted by real part, eigenvector matrix
    as an mp.matrix with columns in the same order). The full A, B are used.
    """
    n = A.shape[0]
    if n > 4:
        raise ValueError("brute force is meant for n <= 4")
    with mp.workdps(dps):
        m = 2 * n
        H = mp.matrix(m, m)
        for i in range(n):
            for j in range(n):
                a = mp.mpc(A[i, j].real, A[i, j].imag)
                b = mp.mpc(B[i, j].real, B[i, j].imag)
                H[i, j] = a
                H[i, n + j] = b
                H[n + i, j] = -mp.conj(b)
                H[n + i, n + j] = -mp.conj(a)
        E, ER = mp.eig(H)
        order = sorted(range(m), key=lambda k: mp.re(E[k]))
        Es = [E[k] for k in order]
        V = mp.matrix(m, m)
        for c, k in enumerate(order):
            for r in range(m):
                V[r, c] = ER[r, k]
        return Es, V


def positive_pairs(A: np.ndarray, B: np.ndarray, dps: int = 50):
    """Positive eigenvalues (ascending) and their right eigenvectors scaled so that
    x^H S x = 1, S = diag(I, -I) (Theorem 3 normalization), as numpy complex128."""
    n = A.shape[0]
    Es, V = eig_H(A, B, dps)
    with mp.workdps(dps):
        lam, cols = [], []
        for c in range(n, 2 * n):
            x = [V[r, c] for r in range(2 * n)]
            q = mp.fsum(abs(x[r]) ** 2 for r in range(n)) - mp.fsum(abs(x[r]) ** 2 for r in range(n, 2 * n))
            s = mp.sqrt(q)
            cols.append([complex(xr / s) for xr in x])
            lam.append(Es[c])
        lam_np = np.array([float(mp.re(e)) for e in lam])
        imag_max = max(float(abs(mp.im(e))) for e in Es)
        X = np.array(cols).T
    return lam_np, X, imag_max
