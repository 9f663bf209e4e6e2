"""The Bethe--Salpeter eigenproblem by its definitions (FP64, numpy).

Test infrastructure only (see the package docstring).

What is computed, and where the paper defines it:

* H = [A B; -conj(B) -conj(A)], A = A^H, B = B^T            (Section 1, Eq. 1-2)
* Omega = [A B; conj(B) conj(A)] > 0                         (Eq. cond)
* H = S Omega with S = diag(I, -I), hence H x = lambda x  <=>
  S x = (1/lambda) Omega x, a Hermitian-definite pencil      (Eq. GMG, proof of Thm 3)
* the positive eigenvalues lambda_1..lambda_n, right eigenvectors x_j,
  left eigenvectors y_j = S x_j with y_j^H x_j = 1           (Theorem 3)
* absorption weights (d_r^H x_j)(y_j^H d_l)/(y_j^H x_j)      (Eq. absp)
* the spectral density over all 2n eigenvalues (Eq. DOS) and the absorption
  spectrum (Eq. absp), with the delta function replaced by Section 5's
  Gaussian of standard deviation sigma
* the Tamm-Dancoff eigenvalues: those of A alone (B = 0)     (Section 2, Theorem 4)
* the accuracy metrics of Table 1.

Route: Omega = Lc Lc^H (Cholesky), C = Lc^{-1} S Lc^{-H} is Hermitian with
eigenvalues theta = 1/lambda (Section 3.1, first paragraph); positive theta give
the positive lambda, and x = sqrt(lambda) Lc^{-H} v gives x^H S x = 1.
Library primitives used as steps: numpy Cholesky, triangular solve, eigh.

Input convention: only the lower triangles of A and B are read (LAPACK 'L');
the upper triangles are rebuilt from Hermitian / complex-symmetric symmetry.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla


class NotDefiniteError(ValueError):
    """Omega = [A B; conj(B) conj(A)] is not positive definite (Eq. cond fails)."""


def symmetrize_lower(A: np.ndarray, B: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Rebuild full A (Hermitian) and B (complex symmetric) from their lower triangles (Eq. 2)."""
    A = np.asarray(A)
    B = np.asarray(B)
    Al = np.tril(A, -1)
    Af = Al + Al.conj().T + np.diag(np.diag(A).real)
    Bl = np.tril(B, -1)
    Bf = Bl + Bl.T + np.diag(np.diag(B))
    return Af.astype(np.complex128), Bf.astype(np.complex128)


def build_H(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """H = [A B; -conj(B) -conj(A)] (Eq. 1)."""
    return np.block([[A, B], [-B.conj(), -A.conj()]])


def build_Omega(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Omega = [A B; conj(B) conj(A)] (Eq. cond)."""
    return np.block([[A, B], [B.conj(), A.conj()]])


def S_signs(n: int) -> np.ndarray:
    """Diagonal of S = diag(I_n, -I_n) (Eq. GMG)."""
    return np.concatenate([np.ones(n), -np.ones(n)])


def build_M(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """M = [Re(A+B) Im(A-B); -Im(A+B) Re(A-B)] (Theorem 2, Eq. embedding)."""
    return np.block([[(A + B).real, (A - B).imag], [-(A + B).imag, (A - B).real]])


def build_Q(n: int) -> np.ndarray:
    """Q = (1/sqrt 2) [I -iI; I iI] (proof of Theorem 2)."""
    I = np.eye(n)
    return np.block([[I, -1j * I], [I, 1j * I]]) / np.sqrt(2.0)


def build_J(n: int) -> np.ndarray:
    """J_n = [0 I; -I 0] (Eq. J)."""
    I = np.eye(n)
    Z = np.zeros((n, n))
    return np.block([[Z, I], [-I, Z]])


@dataclass
class OracleSolution:
    lam: np.ndarray  # (n,) positive eigenvalues, ascending
    X: np.ndarray  # (2n, n) right eigenvectors, column j <-> lam[j]
    Y: np.ndarray  # (2n, n) left eigenvectors, Y = S X
    lam_all: np.ndarray  # (2n,) all eigenvalues of H from the pencil, ascending


def solve(A: np.ndarray, B: np.ndarray) -> OracleSolution:
    """All positive eigenpairs of H with y_j^H x_j = 1 (Theorem 3, Eq. normalization)."""
    A, B = symmetrize_lower(A, B)
    n = A.shape[0]
    Omega = build_Omega(A, B)
    try:
        Lc = np.linalg.cholesky(Omega)
    except np.linalg.LinAlgError as exc:
        raise NotDefiniteError(str(exc)) from exc
    s = S_signs(n)
    # C = Lc^{-1} S Lc^{-H}
    Linv_S = sla.solve_triangular(Lc, np.diag(s).astype(np.complex128), lower=True)
    C = sla.solve_triangular(Lc, Linv_S.conj().T, lower=True).conj().T
    C = (C + C.conj().T) / 2
    theta, V = np.linalg.eigh(C)
    lam_all = np.sort(1.0 / theta)
    pos = theta > 0
    if int(pos.sum()) != n:
        raise NotDefiniteError("pencil inertia is not (n, n)")
    lam = 1.0 / theta[pos]
    Xv = sla.solve_triangular(Lc.conj().T, V[:, pos], lower=False)
    X = Xv * np.sqrt(lam)[None, :]
    order = np.argsort(lam)
    lam = lam[order]
    X = X[:, order]
    Y = s[:, None] * X
    return OracleSolution(lam=lam, X=X, Y=Y, lam_all=lam_all)


def weights(X: np.ndarray, Y: np.ndarray, d_r: np.ndarray, d_l: np.ndarray) -> np.ndarray:
    """w_j = (d_r^H x_j)(y_j^H d_l) / (y_j^H x_j) (Eq. absp); complex in general."""
    a = d_r.conj() @ X
    b = Y.conj().T @ d_l
    c = np.einsum("ij,ij->j", Y.conj(), X)
    return a * b / c


def gaussian_delta(t, sigma: float):
    """Section 5: delta(t) ~ exp(-t^2 / (2 sigma^2)) / (sqrt(2 pi) sigma)."""
    t = np.asarray(t, dtype=np.float64)
    return np.exp(-(t * t) / (2.0 * sigma * sigma)) / (np.sqrt(2.0 * np.pi) * sigma)


def dos(lam: np.ndarray, omega: np.ndarray, sigma: float) -> np.ndarray:
    """Eq. DOS: phi(omega) = 1/(2n) sum over the 2n eigenvalues of H, which are
    +-lambda_j (Theorem 1), of delta(omega - lambda)."""
    eigs = np.concatenate([lam, -lam])
    return gaussian_delta(omega[:, None] - eigs[None, :], sigma).sum(axis=1) / eigs.shape[0]


def absorption(lam: np.ndarray, w: np.ndarray, omega: np.ndarray, sigma: float) -> np.ndarray:
    """Eq. absp: eps+(omega) = sum_j w_j delta(omega - lambda_j) over the positive half."""
    return (w[None, :] * gaussian_delta(omega[:, None] - lam[None, :], sigma)).sum(axis=1)


def tda_eigenvalues(A: np.ndarray) -> np.ndarray:
    """Tamm-Dancoff approximation: B dropped, the eigenvalues of the Hermitian A
    (library eigvalsh as the step), ascending."""
    Af, _ = symmetrize_lower(A, np.zeros_like(A))
    return np.linalg.eigvalsh(Af)


def negative_half(X: np.ndarray) -> np.ndarray:
    """Right eigenvectors for -lambda_j: [conj(X2); conj(X1)] (Theorem 3, Eq. eigvec_r-)."""
    n = X.shape[0] // 2
    return np.concatenate([X[n:].conj(), X[:n].conj()], axis=0)


def full_pairs(lam: np.ndarray, X: np.ndarray):
    """(Lambda_full, X_full, Y_full) with the negative half from Theorem 3.

    Theorem 3: X = [X1 conj(X2); X2 conj(X1)], Y = [X1 -conj(X2); -X2 conj(X1)],
    i.e. y = S x on the positive half and y = -S x on the negative half.
    """
    n = X.shape[0] // 2
    Xn = negative_half(X)
    s = S_signs(n)[:, None]
    Xf = np.concatenate([X, Xn], axis=1)
    Yf = np.concatenate([s * X, -s * Xn], axis=1)
    return np.concatenate([lam, -lam]), Xf, Yf


def table1_metrics(A: np.ndarray, B: np.ndarray, lam: np.ndarray, X: np.ndarray) -> dict:
    """The two accuracy metrics of Table 1 plus the max scaled residual.

    res_F   = ||Y^H H X - Lambda||_F / ||H||_F
    biorth  = ||Y^H X - I_2n||_F / sqrt(2n)
    scaled  = max_j ||H x_j - lambda_j x_j||_2 / (||H||_F ||x_j||_2)
    """
    A, B = symmetrize_lower(A, B)
    H = build_H(A, B)
    n = A.shape[0]
    Lf, Xf, Yf = full_pairs(lam, X)
    normH = np.linalg.norm(H)
    res_F = np.linalg.norm(Yf.conj().T @ H @ Xf - np.diag(Lf)) / normH
    biorth = np.linalg.norm(Yf.conj().T @ Xf - np.eye(2 * n)) / np.sqrt(2 * n)
    R = H @ X - X * lam[None, :]
    scaled = np.max(np.linalg.norm(R, axis=0) / (normH * np.linalg.norm(X, axis=0)))
    return {"res_F": float(res_F), "biorth": float(biorth), "scaled_residual": float(scaled)}


def scaled_residuals(A: np.ndarray, B: np.ndarray, lam: np.ndarray, X: np.ndarray, cols=None) -> np.ndarray:
    """||H x_j - lambda_j x_j|| / (||H||_F ||x_j||) for the chosen columns; O(n^2) per column."""
    A, B = symmetrize_lower(A, B)
    n = A.shape[0]
    if cols is None:
        cols = np.arange(lam.shape[0])
    cols = np.asarray(cols)
    x = X[:, cols]
    x1, x2 = x[:n], x[n:]
    Hx = np.concatenate([A @ x1 + B @ x2, -B.conj() @ x1 - A.conj() @ x2], axis=0)
    normH = np.sqrt(2.0 * (np.linalg.norm(A) ** 2 + np.linalg.norm(B) ** 2))
    r = Hx - x * lam[cols][None, :]
    return np.linalg.norm(r, axis=0) / (normH * np.linalg.norm(x, axis=0))


def eig_count_below(A: np.ndarray, B: np.ndarray, sigma: float) -> int:
    """Number of eigenvalues of H in (0, sigma) for sigma > 0, by Sylvester inertia.

    For the definite pencil S x = theta Omega x (theta = 1/lambda), the eigenvalues
    with theta > 1/sigma are exactly the lambda in (0, sigma); their count is the
    number of positive eigenvalues of S - Omega/sigma (Sylvester's law of inertia).
    Used to check single eigenvalues at sizes where a full solve is too slow.
    """
    A, B = symmetrize_lower(A, B)
    n = A.shape[0]
    K = np.diag(S_signs(n)).astype(np.complex128) - build_Omega(A, B) / sigma
    _, D, _ = sla.ldl(K, lower=True, hermitian=True)
    # D is block diagonal with 1x1 and 2x2 Hermitian blocks: count their positive eigenvalues.
    m = D.shape[0]
    count = 0
    i = 0
    while i < m:
        if i + 1 < m and D[i + 1, i] != 0:
            a, b, c = D[i, i].real, D[i + 1, i], D[i + 1, i + 1].real
            count += int(np.sum(np.linalg.eigvalsh(np.array([[a, np.conj(b)], [b, c]])) > 0))
            i += 2
        else:
            count += int(D[i, i].real > 0)
            i += 1
    return count


def eig_count_below_schur(A: np.ndarray, B: np.ndarray, sigma: float) -> int:
    """Number of eigenvalues of H in (0, sigma), sigma > 0, by Sylvester inertia of
    S - Omega/sigma reduced to an n x n Hermitian matrix.

    With Omega = [A B; conj(B) conj(A)] (Eq. cond) and S = diag(I, -I),
    K = S - Omega/sigma = [I - A/sigma, -B/sigma; -conj(B)/sigma, -(I + conj(A)/sigma)].
    Its (2,2) block is negative definite whenever conj(A)/sigma + I is (A > 0 holds
    for every problem with Omega > 0), so by the additivity of inertia over a
    Schur complement (Haynsworth) the positive eigenvalues of K -- the lambda in
    (0, sigma), see eig_count_below -- are those of
        Sc = K11 - K12 K22^{-1} K21 = I - A/sigma + (B/sigma) (I + conj(A)/sigma)^{-1} (conj(B)/sigma).
    Same count as eig_count_below at an eighth of the indefinite factorization's
    cost (a Cholesky and two triangular solves do the rest). Library routines as
    steps: Cholesky, triangular solve, LDL^H.
    """
    A, B = symmetrize_lower(A, B)
    n = A.shape[0]
    I = np.eye(n)
    G = I + A.conj() / sigma
    try:
        Lg = np.linalg.cholesky(G)
    except np.linalg.LinAlgError as exc:
        raise NotDefiniteError("I + conj(A)/sigma is not positive definite") from exc
    # (B/sigma) G^{-1} (conj(B)/sigma) = Z^H Z with Z = Lg^{-1} conj(B) / sigma (B^T = B)
    Z = sla.solve_triangular(Lg, B.conj() / sigma, lower=True)
    Sc = I - A / sigma + Z.conj().T @ Z
    Sc = (Sc + Sc.conj().T) / 2
    _, D, _ = sla.ldl(Sc, lower=True, hermitian=True)
    count = 0
    i = 0
    while i < n:
        if i + 1 < n and D[i + 1, i] != 0:
            a, b, c = D[i, i].real, D[i + 1, i], D[i + 1, i + 1].real
            count += int(np.sum(np.linalg.eigvalsh(np.array([[a, np.conj(b)], [b, c]])) > 0))
            i += 2
        else:
            count += int(D[i, i].real > 0)
            i += 1
    return count
