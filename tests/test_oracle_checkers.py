"""Pins for the oracle's yardsticks: the scaled residual and Table 1's metrics.

`oracle.definition.scaled_residuals` expands H x block by block (it never forms
H) and `table1_metrics` forms the full pairs of Theorem 3; every full-size parity
claim is measured with them. Here they are tied to things outside the oracle:

* H of Eq. 1 written out entry by entry in plain Python from the lower triangles
  of A and B (no numpy block assembly, no `symmetrize_lower`), and residual norms
  summed with math.fsum, on vectors and eigenvalue guesses that are NOT eigenpairs;
* closed forms: rescaling exact eigenvectors by known real factors c_j changes
  Table 1's two metrics by amounts fixed by Theorem 3's normalization;
* n = 1 by hand.

The planted-mistake tests at the end patch the checkers themselves (a dropped
conjugate in the bottom block, ||H||_F taken from A alone, the negative half's
left vectors with the wrong sign) and show that a pin here catches each.
"""
import math

import numpy as np
import pytest

from oracle import definition as D
from paper_1501_03830_gb300.synth import make_problem


def _entry(M, i, j, hermitian):
    """Entry (i, j) of the full matrix whose lower triangle is stored (Eq. 2)."""
    if i >= j:
        v = complex(M[i, j])
        if i == j and hermitian:
            v = complex(v.real, 0.0)
        return v
    v = complex(M[j, i])
    return v.conjugate() if hermitian else v


def _H_entrywise(A, B):
    """H = [A B; -conj(B) -conj(A)] (Eq. 1) as a list of rows of Python complex."""
    n = A.shape[0]
    H = [[0j] * (2 * n) for _ in range(2 * n)]
    for i in range(n):
        for j in range(n):
            a = _entry(A, i, j, True)
            b = _entry(B, i, j, False)
            H[i][j] = a
            H[i][n + j] = b
            H[n + i][j] = -b.conjugate()
            H[n + i][n + j] = -a.conjugate()
    return H


def _frob(H):
    return math.sqrt(math.fsum(abs(h) ** 2 for row in H for h in row))


def _resid_entrywise(H, lam, x):
    """||H x - lam x||_2 / (||H||_F ||x||_2) by the definition (reading 9)."""
    m = len(H)
    r = []
    for i in range(m):
        re = math.fsum((H[i][k] * x[k]).real for k in range(m)) - (lam * x[i]).real
        im = math.fsum((H[i][k] * x[k]).imag for k in range(m)) - (lam * x[i]).imag
        r.append(re * re + im * im)
    rn = math.sqrt(math.fsum(r))
    xn = math.sqrt(math.fsum(abs(v) ** 2 for v in x))
    return rn / (_frob(H) * xn)


def _random_pairs(n, seed, k):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((2 * n, k)) + 1j * rng.standard_normal((2 * n, k))
    lam = rng.uniform(0.5, 3.0, size=k)
    return lam, X


@pytest.mark.parametrize("n,seed", [(1, 11), (5, 12), (37, 13)])
def test_scaled_residuals_match_entrywise_definition(n, seed):
    """scaled_residuals on arbitrary (non-eigen) vectors equals the entry-by-entry
    ||H x - lam x|| / (||H||_F ||x||) of Eq. 1 (all columns and a chosen subset)."""
    p = make_problem(n, seed)
    k = min(4, n + 1)
    lam, X = _random_pairs(n, seed + 100, k)
    H = _H_entrywise(p.A, p.B)
    want = np.array([_resid_entrywise(H, lam[j], X[:, j]) for j in range(k)])
    got = D.scaled_residuals(p.A, p.B, lam, X)
    assert np.max(np.abs(got - want) / want) <= 1e-12
    cols = [k - 1, 0]
    got_sub = D.scaled_residuals(p.A, p.B, lam, X, cols=cols)
    assert np.max(np.abs(got_sub - want[cols]) / want[cols]) <= 1e-12


@pytest.mark.parametrize("n,seed", [(5, 21), (37, 22)])
def test_table1_scaled_residual_matches_entrywise(n, seed):
    """table1_metrics' max scaled residual equals the entry-by-entry definition's
    maximum over the columns, on non-eigen vectors."""
    p = make_problem(n, seed)
    lam, X = _random_pairs(n, seed + 100, n)
    H = _H_entrywise(p.A, p.B)
    want = max(_resid_entrywise(H, lam[j], X[:, j]) for j in range(n))
    got = D.table1_metrics(p.A, p.B, lam, X)["scaled_residual"]
    assert abs(got - want) <= 1e-12 * want


def test_scaled_residual_n1_by_hand():
    """n = 1: H = [[a, b], [-conj b, -a]], ||H||_F^2 = 2a^2 + 2|b|^2."""
    a, b = 2.0, 0.5 - 0.25j
    x1, x2, lam = 0.3 + 0.4j, -0.2 + 0.1j, 1.7
    r1 = a * x1 + b * x2 - lam * x1
    r2 = -b.conjugate() * x1 - a * x2 - lam * x2
    want = math.sqrt(abs(r1) ** 2 + abs(r2) ** 2) / (
        math.sqrt(2 * a * a + 2 * abs(b) ** 2) * math.sqrt(abs(x1) ** 2 + abs(x2) ** 2))
    got = D.scaled_residuals(np.array([[a + 0j]]), np.array([[b]]), np.array([lam]), np.array([[x1], [x2]]))
    assert abs(got[0] - want) <= 1e-15 * want


@pytest.mark.parametrize("n,seed", [(6, 31), (20, 32)])
def test_table1_metrics_closed_form_under_rescaling(n, seed):
    """Theorem 3 normalizes y_j^H x_j = 1 with y = S x (and y = -S x on the negative
    half). Scaling each exact x_j by a real c_j (and its negative-half partner with
    it) makes Y^H X = diag(c^2, c^2) and Y^H H X = diag(c^2 lam, -c^2 lam), so
    biorth = sqrt(2 sum (c_j^2 - 1)^2) / sqrt(2n) and
    res_F = sqrt(2 sum ((c_j^2 - 1) lam_j)^2) / ||H||_F, with ||H||_F from Eq. 1's
    entries. The residual is scale-invariant and stays at rounding level."""
    p = make_problem(n, seed)
    s = D.solve(p.A, p.B)
    c = np.random.default_rng(seed).uniform(0.5, 1.5, size=n)
    m = D.table1_metrics(p.A, p.B, s.lam, s.X * c[None, :])
    normH = _frob(_H_entrywise(p.A, p.B))
    d = c * c - 1.0
    biorth = math.sqrt(2.0 * math.fsum(d * d)) / math.sqrt(2 * n)
    res_F = math.sqrt(2.0 * math.fsum((d * s.lam) ** 2)) / normH
    assert abs(m["biorth"] - biorth) <= 1e-13 + 1e-12 * biorth
    assert abs(m["res_F"] - res_F) <= 1e-13 + 1e-12 * res_F
    assert m["scaled_residual"] <= 1e-14
    # exact pairs: both metrics at rounding level
    m0 = D.table1_metrics(p.A, p.B, s.lam, s.X)
    assert m0["biorth"] <= 1e-13 and m0["res_F"] <= 1e-13


# --- planted mistakes in the checkers themselves ---------------------------------


def _bad_conj_bottom(A, B, lam, X, cols=None):
    A, B = D.symmetrize_lower(A, B)
    n = A.shape[0]
    cols = np.arange(lam.shape[0]) if cols is None else np.asarray(cols)
    x = X[:, cols]
    Hx = np.concatenate([A @ x[:n] + B @ x[n:], -B @ x[:n] - A @ x[n:]], axis=0)  # conjugates dropped
    normH = np.sqrt(2.0 * (np.linalg.norm(A) ** 2 + np.linalg.norm(B) ** 2))
    return np.linalg.norm(Hx - x * lam[cols][None, :], axis=0) / (normH * np.linalg.norm(x, axis=0))


def _bad_norm_A_only(A, B, lam, X, cols=None):
    A, B = D.symmetrize_lower(A, B)
    n = A.shape[0]
    cols = np.arange(lam.shape[0]) if cols is None else np.asarray(cols)
    x = X[:, cols]
    Hx = np.concatenate([A @ x[:n] + B @ x[n:], -B.conj() @ x[:n] - A.conj() @ x[n:]], axis=0)
    normH = np.linalg.norm(A)  # ||H||_F of A alone
    return np.linalg.norm(Hx - x * lam[cols][None, :], axis=0) / (normH * np.linalg.norm(x, axis=0))


@pytest.mark.parametrize("bad", [_bad_conj_bottom, _bad_norm_A_only])
def test_planted_mistake_in_scaled_residuals_is_caught(monkeypatch, bad):
    monkeypatch.setattr(D, "scaled_residuals", bad)
    with pytest.raises(AssertionError):
        test_scaled_residuals_match_entrywise_definition(5, 12)


def test_planted_mistake_in_table1_pairs_is_caught(monkeypatch):
    """Negative-half left vectors taken as +S x instead of -S x (Theorem 3)."""

    def bad_full_pairs(lam, X):
        n = X.shape[0] // 2
        Xn = D.negative_half(X)
        s = D.S_signs(n)[:, None]
        return np.concatenate([lam, -lam]), np.concatenate([X, Xn], axis=1), np.concatenate([s * X, s * Xn], axis=1)

    monkeypatch.setattr(D, "full_pairs", bad_full_pairs)
    with pytest.raises(AssertionError):
        test_table1_metrics_closed_form_under_rescaling(6, 31)


def test_planted_mistake_in_table1_norm_is_caught(monkeypatch):
    """res_F divided by ||A||_F instead of ||H||_F."""
    orig = D.table1_metrics

    def bad_table1(A, B, lam, X):
        m = orig(A, B, lam, X)
        Af, Bf = D.symmetrize_lower(A, B)
        normH = np.linalg.norm(D.build_H(Af, Bf))
        m["res_F"] *= normH / np.linalg.norm(Af)
        return m

    monkeypatch.setattr(D, "table1_metrics", bad_table1)
    with pytest.raises(AssertionError):
        test_table1_metrics_closed_form_under_rescaling(6, 31)


def test_planted_mistake_in_table1_residual_is_caught(monkeypatch):
    """Table 1's column residual with H's bottom block unconjugated."""

    def bad_table1(A, B, lam, X):
        Af, Bf = D.symmetrize_lower(A, B)
        H = np.block([[Af, Bf], [-Bf, -Af]])
        R = H @ X - X * lam[None, :]
        normH = np.linalg.norm(H)
        return {"res_F": 0.0, "biorth": 0.0,
                "scaled_residual": float(np.max(np.linalg.norm(R, axis=0) / (normH * np.linalg.norm(X, axis=0))))}

    monkeypatch.setattr(D, "table1_metrics", bad_table1)
    with pytest.raises(AssertionError):
        test_table1_scaled_residual_matches_entrywise(5, 21)
