"""Eigenpairs of a symmetric tridiagonal matrix by a representation tree (the MRRR
idea: Dhillon and Parlett, Linear Algebra Appl. 387, 2004), FP64 numpy.

Test infrastructure only (see the package docstring). It restates, for the
tridiagonal step of Algorithm 3 (Section 3.3, remark 2, which calls for
reorthogonalization when high accuracy is wanted), the way to get orthogonal eigenvectors
without reorthogonalization; the device tree is tested against it. Plain scalar
loops (vectorized over shifts where the recurrence allows), small sizes only.

  root       T - sigma I = L D L^T with sigma below the spectrum (positive
             definite, hence a relatively robust representation)
  values     bisection on the representation: the number of eigenvalues of
             L D L^T below x is the number of negative pivots of
             L D L^T - x I = L+ D+ L+^T (stationary qd transform)
  tree       eigenvalues whose relative gap to both neighbours is >= gaptol are
             singletons; runs of closer ones form clusters. A cluster gets a
             child representation L D L^T - tau I = L' D' L'^T with tau just
             left of it (the cluster's eigenvalues shrink to distances from tau,
             which enlarges their relative gaps), its eigenvalues are refined on
             the child, and the classification repeats there. A cluster of more
             than 1/gaptol members (a dense spectrum) gets tau within a quarter
             of (mean gap / gaptol) of its first eigenvalue, so that the first
             ~1/gaptol of them separate in the child and the rest form a smaller
             cluster there ("peeling")
  vectors    a singleton's vector comes from the twisted factorization of its
             representation shifted by the eigenvalue: the stationary transform
             from the top, the progressive one from the bottom, twist index r
             where |gamma_r| is smallest, z_r = 1 and the two bidiagonal
             recurrences outward; the eigenvalue is then corrected by the
             Rayleigh quotient gamma_r / ||z||^2 and the vector recomputed
"""
from __future__ import annotations

import numpy as np

EPS = 2.0 ** -52
TINY = 2.0 ** -1000  # stands in for an exactly zero pivot (the transforms stay finite)


def _nz(x: float) -> float:
    return x if x != 0.0 else -TINY


def ldl_root(a: np.ndarray, b: np.ndarray, sigma: float):
    """L D L^T = T - sigma I for T = tridiag(b, a, b): D (n), l (n - 1)."""
    n = a.shape[0]
    D = np.zeros(n)
    l = np.zeros(max(n - 1, 0))
    D[0] = a[0] - sigma
    for i in range(n - 1):
        l[i] = b[i] / D[i]
        D[i + 1] = a[i + 1] - sigma - l[i] * b[i]
    return D, l


def stqds(D, l, tau):
    """Stationary transform: L D L^T - tau I = L+ D+ L+^T; also returns s."""
    n = D.shape[0]
    Dp = np.zeros(n)
    lp = np.zeros(max(n - 1, 0))
    s = np.zeros(n)
    s[0] = -tau
    for i in range(n - 1):
        Dp[i] = _nz(s[i] + D[i])
        lp[i] = D[i] * l[i] / Dp[i]
        s[i + 1] = lp[i] * l[i] * s[i] - tau
    Dp[n - 1] = _nz(s[n - 1] + D[n - 1])
    return Dp, lp, s


def pqds(D, l, tau):
    """Progressive transform: L D L^T - tau I = U- D- U-^T (U- unit upper
    bidiagonal, superdiagonal u); also returns p."""
    n = D.shape[0]
    Dm = np.zeros(n)
    u = np.zeros(max(n - 1, 0))
    p = np.zeros(n)
    p[n - 1] = D[n - 1] - tau
    for i in range(n - 2, -1, -1):
        Dm[i + 1] = _nz(D[i] * l[i] * l[i] + p[i + 1])
        t = D[i] / Dm[i + 1]
        u[i] = l[i] * t
        p[i] = p[i + 1] * t - tau
    Dm[0] = p[0]
    return Dm, u, p


def negcount(D, l, x) -> int:
    """Eigenvalues of L D L^T below x (negative pivots of the shifted factor)."""
    Dp, _, _ = stqds(D, l, x)
    return int(np.sum(Dp < 0))


def negcounts(D, l, xs: np.ndarray) -> np.ndarray:
    """negcount for every shift in xs at once: the stationary transform of
    stqds with a vector of shifts (the same recurrence, elementwise)."""
    xs = np.asarray(xs, dtype=np.float64)
    n = D.shape[0]
    cnt = np.zeros(xs.shape, dtype=np.int64)
    s = -xs
    for i in range(n - 1):
        dp = s + D[i]
        dp = np.where(dp == 0.0, -TINY, dp)
        cnt += dp < 0
        s = (D[i] * l[i] / dp) * l[i] * s - xs
    dp = s + D[n - 1]
    dp = np.where(dp == 0.0, -TINY, dp)
    cnt += dp < 0
    return cnt


def bisect(D, l, lo, hi, k, tol=4 * EPS):
    """The k-th smallest eigenvalue (0-based) of L D L^T in [lo, hi], to relative
    accuracy tol."""
    return float(bisect_all(D, l, np.array([lo]), np.array([hi]), np.array([k]), tol)[0])


def bisect_all(D, l, lo, hi, ks, tol=4 * EPS):
    """bisect for several eigenvalues at once (eigenvalue ks[i] in [lo[i], hi[i]]);
    each interval is halved on its own until it meets the same stopping rule."""
    lo = np.array(lo, dtype=np.float64)
    hi = np.array(hi, dtype=np.float64)
    ks = np.asarray(ks)
    active = hi - lo > tol * np.maximum(np.abs(lo), np.abs(hi))
    while np.any(active):
        mid = 0.5 * (lo + hi)
        active &= (mid != lo) & (mid != hi)
        if not np.any(active):
            break
        idx = np.nonzero(active)[0]
        up = negcounts(D, l, mid[idx]) > ks[idx]
        hi[idx[up]] = mid[idx[up]]
        lo[idx[~up]] = mid[idx[~up]]
        active = hi - lo > tol * np.maximum(np.abs(lo), np.abs(hi))
    return 0.5 * (lo + hi)


def twisted_vector(D, l, lam):
    """Twisted factorization of L D L^T - lam I: (z with z_r = 1, gamma_r, r)."""
    n = D.shape[0]
    Dp, lp, s = stqds(D, l, lam)
    Dm, u, p = pqds(D, l, lam)
    gamma = s + p + lam
    r = int(np.argmin(np.abs(gamma)))
    z = np.zeros(n)
    z[r] = 1.0
    for i in range(r - 1, -1, -1):
        z[i] = -lp[i] * z[i + 1]
    for i in range(r, n - 1):
        z[i + 1] = -u[i] * z[i]
    return z, gamma[r], r


def _vector(D, l, lam, iters=3):
    for _ in range(iters):
        z, g, _ = twisted_vector(D, l, lam)
        lam = lam + g / float(z @ z)
    z, _, _ = twisted_vector(D, l, lam)
    return z / np.linalg.norm(z), lam


def _eigvals(D, l, idx, lo, hi):
    return bisect_all(D, l, np.full(len(idx), lo), np.full(len(idx), hi), np.array(idx))


MAX_DEPTH = 8    # levels of child representations for clusters of <= 1/gaptol members
MAX_PEELS = 64   # levels that peel a larger cluster


def _solve(D, l, shift, idx, lo, hi, gaptol, depth, out_lam, out_z, tree, peels=0):
    """Eigenpairs idx of L D L^T (whose eigenvalues lie in [lo, hi]); the
    matrix's eigenvalues are these plus `shift`."""
    lam = _eigvals(D, l, idx, lo, hi)
    k = 0
    m = len(idx)
    while k < m:
        # extend a cluster while the relative gap to the next value is small
        e = k
        while e + 1 < m and (lam[e + 1] - lam[e]) < gaptol * max(abs(lam[e]), abs(lam[e + 1])):
            e += 1
        size = e - k + 1
        large = size * gaptol > 1.0
        if e == k or (depth >= MAX_DEPTH and not large) or (large and peels >= MAX_PEELS):
            for t in range(k, e + 1):
                z, lt = _vector(D, l, lam[t])
                out_lam[idx[t]] = lt + shift
                out_z[:, idx[t]] = z
            tree.append((depth, 1 if e == k else size))
        else:
            # child representation just left of the cluster
            left = lam[k - 1] if k > 0 else lam[k] - (lam[e] - lam[k]) - abs(lam[k]) * 1e-3
            width = lam[e] - lam[k]
            off = min(lam[k] - left, width + abs(lam[k]) * 1e-3)
            if large:
                # more than 1/gaptol members: a shift at the scale of the whole width
                # would leave every relative gap below gaptol; at a quarter of (mean
                # gap / gaptol) the first ~1/gaptol members separate in the child and
                # the rest form a smaller cluster there
                off = min(off, width / (size - 1) / gaptol)
            tau = lam[k] - max(0.25 * off, abs(lam[k]) * 8 * EPS)
            Dc, lc, _ = stqds(D, l, tau)
            tree.append((depth, size))
            lo_c = (lam[k] - tau) * (1 - 1e-6)
            hi_c = (lam[e] - tau) * (1 + 1e-6) + abs(lam[e]) * 4 * EPS
            _solve(Dc, lc, shift + tau, [idx[t] for t in range(k, e + 1)], lo_c, hi_c, gaptol,
                   depth if large else depth + 1, out_lam, out_z, tree, peels + 1 if large else peels)
        k = e + 1


def eigh_tridiagonal(a: np.ndarray, b: np.ndarray, gaptol: float = 1e-3):
    """All eigenpairs of T = tridiag(b, a, b) (ascending). Returns (lam, Z, tree):
    tree lists (depth, size) for every singleton (size 1), every cluster that got
    a child representation, and every group left at the depth limit (MAX_DEPTH,
    or MAX_PEELS for the peeling levels of clusters of more than 1/gaptol)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    n = a.shape[0]
    if n == 1:
        return a.copy(), np.ones((1, 1)), [(0, 1)]
    r = np.concatenate([np.abs(b), [0.0]]) + np.concatenate([[0.0], np.abs(b)])
    glo, ghi = float(np.min(a - r)), float(np.max(a + r))
    sigma = glo - 1e-3 * (ghi - glo) - 1e-300
    D, l = ldl_root(a, b, sigma)
    lam = np.zeros(n)
    Z = np.zeros((n, n))
    tree = []
    _solve(D, l, sigma, list(range(n)), 0.0, (ghi - sigma) * (1 + 1e-12), gaptol, 0, lam, Z, tree)
    order = np.argsort(lam)
    return lam[order], Z[:, order], tree
