"""Algorithm 1 and Algorithm 3 restated step by step (FP64, numpy).

Test infrastructure only (see the package docstring). Each function is one step
in the paper's order and notation; nothing is blocked, fused or reordered.
Library primitives used as steps: numpy Cholesky, matmul, eigh.

Algorithm 1 (complex BSE, Section 3.1):
  1. M = [Re(A+B) Im(A-B); -Im(A+B) Re(A-B)]
  2. M = L L^T
  3. W = L^T J L
  4. -iW = [Z+ Z-] diag(Lambda+, -Lambda+) [Z+ Z-]^H
  5. [X1; X2] = diag(I, -I) Q L Z+ Lambda+^{-1/2}

Algorithm 3 (steps 4-5 of Algorithm 1, Section 3.3):
  1. W = U T U^T by Householder reflections (skew-symmetric tridiagonal T)
  2. -i D^H T D = [V+ V-] diag(Lambda+, -Lambda+) [V+ V-]^T,  D = diag(1, i, i^2, ...)
  3. Phi = L U
  4. Yhat = Q Phi D
  5. Y+ = Yhat V+
  6. [X1; X2] = diag(I, -I) Y+   (times Lambda+^{-1/2}, as in step 5 of Algorithm 1)

Readings of the text:
* D has 2n entries, D = diag(i^k), k = 0..2n-1 (the printed list runs to i^{2n}).
* Algorithm 3's last step carries the Lambda+^{-1/2} factor of Algorithm 1 step 5;
  without it y_j^H x_j = lambda_j instead of 1 (Theorem 3 normalization).
* The Householder reflector for column j is H_j = I - tau_j v_j v_j^T with
  v_j(j+1) = 1 and beta_j = -sign(alpha) ||(alpha, x)|| (LAPACK dlarfg convention);
  T's sub-diagonal holds beta_j, its super-diagonal -beta_j, so the alpha_k of
  remark 2 (the super-diagonal) is -beta_k.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .definition import build_M, build_J, build_Q, symmetrize_lower


def step1_M(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Algorithm 1 step 1 (lower triangles of A, B are read)."""
    A, B = symmetrize_lower(A, B)
    return build_M(A, B)


def step2_cholesky(M: np.ndarray) -> np.ndarray:
    """Algorithm 1 step 2: lower-triangular L with M = L L^T."""
    return np.linalg.cholesky(M)


def step3_W(L: np.ndarray) -> np.ndarray:
    """Algorithm 1 step 3: W = L^T J L (real skew-symmetric)."""
    n = L.shape[0] // 2
    return L.T @ build_J(n) @ L


def householder(x: np.ndarray) -> tuple[np.ndarray, float, float]:
    """Reflector H = I - tau v v^T with v[0] = 1 and H x = beta e_1 (dlarfg convention)."""
    alpha = x[0]
    sigma = float(np.dot(x[1:], x[1:]))
    v = np.zeros_like(x)
    v[0] = 1.0
    if sigma == 0.0:
        return v, 0.0, float(alpha)
    norm = np.sqrt(alpha * alpha + sigma)
    beta = -norm if alpha >= 0 else norm
    tau = (beta - alpha) / beta
    v[1:] = x[1:] / (alpha - beta)
    return v, float(tau), float(beta)


@dataclass
class Tridiag:
    T: np.ndarray  # (m, m) skew-symmetric tridiagonal
    beta: np.ndarray  # (m-1,) sub-diagonal T[k+1, k]
    vs: list  # reflector vectors (length m, zero above row j+1)
    taus: np.ndarray  # (m-1,)
    U: np.ndarray  # (m, m) orthogonal, W = U T U^T


def alg3_step1_tridiagonalize(W: np.ndarray) -> Tridiag:
    """Algorithm 3 step 1: reduce W to skew tridiagonal T = U^T W U, one column at a time.

    Each H_j is applied literally as A <- H_j A H_j (two rank-1 products), without
    using skew symmetry.
    """
    m = W.shape[0]
    A = W.astype(np.float64).copy()
    vs, taus, betas = [], [], []
    U = np.eye(m)
    for j in range(m - 1):
        v_loc, tau, beta = householder(A[j + 1 :, j].copy())
        v = np.zeros(m)
        v[j + 1 :] = v_loc
        # A <- H A H,  H = I - tau v v^T
        A = A - tau * np.outer(v, v @ A)
        A = A - tau * np.outer(A @ v, v)
        U = U - tau * np.outer(U @ v, v)
        vs.append(v)
        taus.append(tau)
        betas.append(beta)
    T = np.zeros((m, m))
    b = np.array(betas)
    idx = np.arange(m - 1)
    T[idx + 1, idx] = b
    T[idx, idx + 1] = -b
    return Tridiag(T=T, beta=b, vs=vs, taus=np.array(taus), U=U)


def D_matrix(m: int) -> np.ndarray:
    """D = diag(i^k), k = 0..m-1 (Algorithm 3 step 2, reading noted above)."""
    return np.diag(1j ** np.arange(m))


def alg3_step2_tridiag_eig(T: np.ndarray) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Algorithm 3 step 2: positive spectral decomposition of -i D^H T D.

    Returns (Lambda+, V+, Tsym) with Lambda+ ascending and V+ real (m, n).
    """
    m = T.shape[0]
    D = D_matrix(m)
    Tc = -1j * D.conj().T @ T @ D
    Tsym = Tc.real
    w, V = np.linalg.eigh(Tsym)
    n = m // 2
    return w[n:], V[:, n:], Tsym


def alg3_backtransform(L, U, Vp, lam):
    """Algorithm 3 steps 3-6 (with Lambda+^{-1/2}); returns (X, Y, Yplus)."""
    m = L.shape[0]
    n = m // 2
    Phi = L @ U  # step 3
    Yhat = build_Q(n) @ Phi @ D_matrix(m)  # step 4
    Yplus = Yhat @ Vp  # step 5
    s = np.concatenate([np.ones(n), -np.ones(n)])
    X = s[:, None] * Yplus / np.sqrt(lam)[None, :]  # step 6 (+ Alg. 1 step 5 scaling)
    Y = s[:, None] * X
    return X, Y, Yplus


@dataclass
class Alg1Result:
    M: np.ndarray
    L: np.ndarray
    W: np.ndarray
    tri: Tridiag
    Tsym: np.ndarray
    lam: np.ndarray
    Vp: np.ndarray
    X: np.ndarray
    Y: np.ndarray


def run(A: np.ndarray, B: np.ndarray) -> Alg1Result:
    """Algorithm 1 with steps 4-5 done by Algorithm 3 (small sizes only: O(m^3) numpy loops)."""
    M = step1_M(A, B)
    L = step2_cholesky(M)
    W = step3_W(L)
    tri = alg3_step1_tridiagonalize(W)
    lam, Vp, Tsym = alg3_step2_tridiag_eig(tri.T)
    X, Y, _ = alg3_backtransform(L, tri.U, Vp, lam)
    return Alg1Result(M=M, L=L, W=W, tri=tri, Tsym=Tsym, lam=lam, Vp=Vp, X=X, Y=Y)
