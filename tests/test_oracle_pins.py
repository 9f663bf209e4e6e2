"""Pins that tie the CPU oracle to the paper and to mathematics, not to itself.

Each test names the passage (section, equation, theorem) whose fact it checks.
A plausible mistake anywhere in the oracle (a dropped term, a wrong sign, a
transposed operand, a wrong normalization) fails at least one of them; the
"planted mistake" tests at the end show this for a few such mistakes.
"""
import json
import os

import numpy as np
import pytest

from oracle import alg1, alg2, brute
from oracle import definition as D
from paper_1501_03830_gb300.synth import make_problem

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "brute_force_eigs.json")


def _rel(a, b):
    return np.max(np.abs(a - b) / np.abs(b))


@pytest.mark.parametrize("n,seed", [(1, 5), (37, 6), (300, 7)])
def test_eig_count_below_schur(n, seed):
    """Sylvester inertia through the Schur complement of S - Omega/sigma (Eq. cond):
    exactly k eigenvalues below lambda_k (1 - 1e-10) and k + 1 below lambda_k (1 + 1e-10),
    the same counts as the full indefinite factorization."""
    p = make_problem(n, seed)
    s = D.solve(p.A, p.B)
    for k in sorted({0, n // 3, n - 1}):
        for f, want in ((1 - 1e-10, k), (1 + 1e-10, k + 1)):
            sig = s.lam[k] * f
            assert D.eig_count_below_schur(p.A, p.B, sig) == want
            assert D.eig_count_below(p.A, p.B, sig) == want


def test_planted_mistake_schur_sign_is_caught(monkeypatch):
    """Subtracting the Schur term instead of adding it (K12 K22^{-1} K21 has two minus
    signs) miscounts and fails the inertia pin."""
    import scipy.linalg as sla

    def bad(A, B, sigma):
        A, B = D.symmetrize_lower(A, B)
        n = A.shape[0]
        Lg = np.linalg.cholesky(np.eye(n) + A.conj() / sigma)
        Z = sla.solve_triangular(Lg, B.conj() / sigma, lower=True)
        Sc = np.eye(n) - A / sigma - Z.conj().T @ Z
        return int(np.sum(np.linalg.eigvalsh((Sc + Sc.conj().T) / 2) > 0))

    monkeypatch.setattr(D, "eig_count_below_schur", bad)
    with pytest.raises(AssertionError):
        test_eig_count_below_schur(37, 6)


# --- closed forms -------------------------------------------------------------


@pytest.mark.parametrize("a,b", [(2.0, 0.5 + 0.3j), (1.0, 0.0), (3.0, -1.2j), (1.5, 1.4)])
def test_n1_closed_form(a, b):
    """n = 1: H = [a b; -conj(b) -a], lambda = sqrt(a^2 - |b|^2) (Eq. 1 with Eq. cond)."""
    A = np.array([[a]], dtype=complex)
    B = np.array([[b]], dtype=complex)
    s = D.solve(A, B)
    lam = np.sqrt(a * a - abs(b) ** 2)
    assert abs(s.lam[0] - lam) <= 1e-14 * lam
    x1, x2 = s.X[0, 0], s.X[1, 0]
    # first row of (H - lambda) x = 0 and the Theorem 3 normalization |x1|^2 - |x2|^2 = 1
    assert abs((a - lam) * x1 + b * x2) <= 1e-13
    assert abs(abs(x1) ** 2 - abs(x2) ** 2 - 1.0) <= 1e-13
    # Eq. absp with d_r = d_l = e_1: w = |x1|^2 / (|x1|^2 - |x2|^2) = |x1|^2
    d = np.array([1.0, 0.0], dtype=complex)
    w = D.weights(s.X, s.Y, d, d)
    assert abs(w[0] - abs(x1) ** 2) <= 1e-13


def test_n1_not_definite():
    """Eq. cond fails when |b| >= a: the oracle must refuse, not return garbage."""
    with pytest.raises(D.NotDefiniteError):
        D.solve(np.array([[1.0 + 0j]]), np.array([[1.5 + 0j]]))


# --- brute force (50 digits) ------------------------------------------------


def test_golden_brute_force():
    """Stored 50-digit eigenvalues of H (tests/golden, written by oracle.brute)."""
    with open(GOLDEN) as f:
        gold = json.load(f)
    for case in gold["cases"]:
        p = make_problem(case["n"], case["seed"], real=case["real"])
        s = D.solve(p.A, p.B)
        ref = np.array([float(x) for x in case["eig_re"]])
        assert _rel(s.lam_all, ref) <= 5e-14
        n = case["n"]
        assert _rel(s.lam, ref[n:]) <= 5e-14


@pytest.mark.parametrize("n,seed", [(1, 3), (2, 4), (3, 5), (4, 6)])
def test_brute_force_eigvecs(n, seed):
    """Right eigenvectors agree with mpmath up to phase: compare the rank-1 projectors
    x_j y_j^H, which are phase free (Theorem 3, y = S x)."""
    p = make_problem(n, seed)
    s = D.solve(p.A, p.B)
    lb, Xb, imag = brute.positive_pairs(p.A, p.B)
    assert imag <= 1e-40
    assert _rel(s.lam, lb) <= 1e-14
    S = D.S_signs(n)[:, None]
    for j in range(n):
        P1 = np.outer(s.X[:, j], (S * s.X)[:, j].conj())
        P2 = np.outer(Xb[:, j], (S * Xb)[:, j].conj())
        assert np.max(np.abs(P1 - P2)) <= 1e-12


# --- invariants -----------------------------------------------------------------


@pytest.mark.parametrize("n,seed", [(16, 1), (64, 0)])
def test_zgeev_crosscheck_and_realness(n, seed):
    """A general eigensolver on H (the paper's ZGEEV comparator, Section 4) gives real,
    +/- paired eigenvalues equal to the oracle's (Theorem 1, Eq. GMG)."""
    p = make_problem(n, seed)
    A, B = D.symmetrize_lower(p.A, p.B)
    ev = np.linalg.eigvals(D.build_H(A, B))
    assert np.max(np.abs(ev.imag)) <= 1e-10
    evs = np.sort(ev.real)
    s = D.solve(p.A, p.B)
    assert _rel(evs[n:], s.lam) <= 1e-11
    assert _rel(-evs[:n][::-1], s.lam) <= 1e-11


@pytest.mark.parametrize("n,seed", [(8, 2), (64, 0), (200, 9)])
def test_pairing(n, seed):
    """All 2n pencil eigenvalues come in +/- pairs (Theorem 1); the pencil route does not
    enforce this, so it is a real check (Section 3.1 on ZHEGV)."""
    s = D.solve(make_problem(n, seed).A, make_problem(n, seed).B)
    neg = -s.lam_all[:n][::-1]
    assert _rel(neg, s.lam) <= 1e-12


@pytest.mark.parametrize("n,seed", [(8, 2), (64, 0), (150, 4)])
def test_tda_upper_bound(n, seed):
    """Theorem 4: lambda_j(H) <= lambda_j(A) for every j (both sorted the same way)."""
    p = make_problem(n, seed)
    s = D.solve(p.A, p.B)
    A, _ = D.symmetrize_lower(p.A, p.B)
    la = np.linalg.eigvalsh(A)
    assert np.all(s.lam <= la * (1 + 1e-13))


@pytest.mark.parametrize("n,seed", [(5, 1), (64, 3)])
def test_real_case_product_eigenproblem(n, seed):
    """Real case (Eq. H-real): lambda^2 are the eigenvalues of (A-B)(A+B), computed here as
    eig(L1^T (A-B) L1) with A+B = L1 L1^T (Section 2.1)."""
    p = make_problem(n, seed, real=True)
    s = D.solve(p.A.astype(complex), p.B.astype(complex))
    A = np.tril(p.A) + np.tril(p.A, -1).T
    B = np.tril(p.B) + np.tril(p.B, -1).T
    L1 = np.linalg.cholesky(A + B)
    mu = np.linalg.eigvalsh(L1.T @ (A - B) @ L1)
    assert _rel(np.sqrt(np.sort(mu)), s.lam) <= 1e-13


@pytest.mark.parametrize("n,seed", [(32, 7), (64, 0)])
def test_table1_metrics_small(n, seed):
    """Table 1's residual and biorthogonality metrics are at FP64 level (1e-15 in the paper)."""
    p = make_problem(n, seed)
    s = D.solve(p.A, p.B)
    m = D.table1_metrics(p.A, p.B, s.lam, s.X)
    assert m["res_F"] <= 2e-14
    assert m["biorth"] <= 2e-14
    assert m["scaled_residual"] <= 1e-14


def test_theorem3_structure():
    """Theorem 3: X1^H X1 - X2^H X2 = I, conj(X1)^H X2 = conj(X2)^H X1, and
    [conj(X2); conj(X1)] are eigenvectors for -lambda."""
    n = 24
    p = make_problem(n, 8)
    s = D.solve(p.A, p.B)
    X1, X2 = s.X[:n], s.X[n:]
    assert np.max(np.abs(X1.conj().T @ X1 - X2.conj().T @ X2 - np.eye(n))) <= 1e-13
    assert np.max(np.abs(X1.T @ X2 - X2.T @ X1)) <= 1e-13
    A, B = D.symmetrize_lower(p.A, p.B)
    H = D.build_H(A, B)
    Xn = D.negative_half(s.X)
    assert np.max(np.abs(H @ Xn + Xn * s.lam[None, :])) <= 1e-12


def test_weights_phase_invariant_and_complex():
    """Eq. absp is invariant to x_j -> e^{i phi} x_j; with y != x the weights are complex."""
    n = 16
    p = make_problem(n, 5)
    s = D.solve(p.A, p.B)
    w = D.weights(s.X, s.Y, p.d_r, p.d_l)
    ph = np.exp(1j * np.linspace(0, 6, n))
    w2 = D.weights(s.X * ph[None, :], s.Y * ph[None, :], p.d_r, p.d_l)
    assert np.max(np.abs(w - w2)) <= 1e-13
    assert np.max(np.abs(w.imag)) > 1e-8


def test_lower_triangle_convention():
    """Only the lower triangles of A and B are read (Eq. 2 defines the rest)."""
    p = make_problem(12, 3)
    A2 = p.A.copy()
    B2 = p.B.copy()
    iu = np.triu_indices(12, 1)
    A2[iu] = 99.0 + 7j
    B2[iu] = -5.0
    s1 = D.solve(p.A, p.B)
    s2 = D.solve(A2, B2)
    assert np.max(np.abs(s1.lam - s2.lam)) == 0.0


def test_eig_count_below():
    """Sylvester inertia count agrees with the sorted spectrum."""
    p = make_problem(20, 2)
    s = D.solve(p.A, p.B)
    for k in (0, 5, 19):
        assert D.eig_count_below(p.A, p.B, s.lam[k] * (1 - 1e-9)) == k
        assert D.eig_count_below(p.A, p.B, s.lam[k] * (1 + 1e-9)) == k + 1


# --- Algorithm 1 / 3 stage restatement ----------------------------------------


def test_theorem2_embedding():
    """Theorem 2: Q^H H Q = -i J M with M real symmetric (pins build_M)."""
    n = 7
    p = make_problem(n, 1)
    A, B = D.symmetrize_lower(p.A, p.B)
    Q = D.build_Q(n)
    lhs = Q.conj().T @ D.build_H(A, B) @ Q
    M = D.build_M(A, B)
    assert np.max(np.abs(lhs - (-1j) * D.build_J(n) @ M)) <= 1e-14
    assert np.max(np.abs(M - M.T)) == 0.0
    # and the Theorem 4 proof: Q^H Omega Q = Atilde + Btilde, i.e. M (it is positive definite)
    assert np.max(np.abs(Q.conj().T @ D.build_Omega(A, B) @ Q - M)) <= 1e-14


@pytest.mark.parametrize("n,seed", [(6, 1), (32, 2)])
def test_alg1_stages(n, seed):
    """Algorithm 1/3 intermediates have the properties the text states or implies."""
    p = make_problem(n, seed)
    r = alg1.run(p.A, p.B)
    m = 2 * n
    assert np.max(np.abs(r.L @ r.L.T - r.M)) <= 1e-14 * np.abs(r.M).max() * m
    # W = L^T J L is skew; its (2,2) block is exactly zero (L = [L11 0; L21 L22])
    assert np.max(np.abs(r.W + r.W.T)) <= 1e-14
    assert np.max(np.abs(r.W[n:, n:])) == 0.0
    # Householder: U orthogonal, U^T W U = T tridiagonal
    U = r.tri.U
    assert np.max(np.abs(U.T @ U - np.eye(m))) <= 1e-13
    assert np.max(np.abs(U.T @ r.W @ U - r.tri.T)) <= 1e-12
    # remark 2: -i D^H T D is real symmetric, zero diagonal, off-diagonal = T's super-diagonal
    Tc = -1j * alg1.D_matrix(m).conj().T @ r.tri.T @ alg1.D_matrix(m)
    assert np.max(np.abs(Tc.imag)) <= 1e-15
    assert np.max(np.abs(np.diag(Tc.real))) == 0.0
    assert np.allclose(np.diag(Tc.real, 1), -r.tri.beta, rtol=0, atol=1e-15)
    # its positive eigenvalues are the singular values of the bidiagonal half (Golub-Kahan)
    a = -r.tri.beta
    Bd = np.diag(a[0::2]) + np.diag(a[1::2], 1)
    sv = np.sort(np.linalg.svd(Bd, compute_uv=False))
    assert _rel(sv, r.lam) <= 1e-13
    # and they equal the pencil route's eigenvalues
    s = D.solve(p.A, p.B)
    assert _rel(r.lam, s.lam) <= 1e-13
    # eigenvectors: phase-free comparison through the weights (Eq. absp)
    w1 = D.weights(r.X, r.Y, p.d_r, p.d_l)
    w2 = D.weights(s.X, s.Y, p.d_r, p.d_l)
    assert np.max(np.abs(w1 - w2)) <= 1e-11 * np.max(np.abs(w2))


def test_alg1_minus_iW_spectrum():
    """Algorithm 1 step 4: -iW is Hermitian with eigenvalues +/- lambda."""
    n = 10
    p = make_problem(n, 4)
    r = alg1.run(p.A, p.B)
    ev = np.linalg.eigvalsh(-1j * r.W)
    s = D.solve(p.A, p.B)
    assert _rel(ev[n:], s.lam) <= 1e-13
    assert _rel(-ev[:n][::-1], s.lam) <= 1e-13


# --- spectra (Eq. DOS, Eq. absp, Section 5's Gaussian) -----------------------


def test_gaussian_delta_closed_forms():
    """Section 5's Gaussian: peak 1/(sqrt(2 pi) sigma), unit integral, half
    maximum at t = sigma sqrt(2 ln 2)."""
    sig = 5e-4
    assert abs(D.gaussian_delta(0.0, sig) - 1.0 / (np.sqrt(2 * np.pi) * sig)) <= 1e-12 / sig
    t = np.linspace(-12 * sig, 12 * sig, 48001)
    assert abs(np.trapezoid(D.gaussian_delta(t, sig), t) - 1.0) <= 1e-12
    half = sig * np.sqrt(2 * np.log(2))
    assert abs(D.gaussian_delta(half, sig) / D.gaussian_delta(0.0, sig) - 0.5) <= 1e-14


def test_dos_normalization_symmetry_and_peaks():
    """Eq. DOS counts all 2n eigenvalues +-lambda_j with weight 1/(2n): the density
    integrates to 1 over the real line, is even in omega, and an isolated
    eigenvalue gives a peak of height g(0)/(2n)."""
    lam = np.array([1.0, 1.7, 2.9])
    sig = 0.01
    om = np.linspace(-3.5, 3.5, 140001)
    phi = D.dos(lam, om, sig)
    assert abs(np.trapezoid(phi, om) - 1.0) <= 1e-10
    assert np.allclose(phi, phi[::-1], rtol=0, atol=1e-12 * phi.max())
    peak = D.dos(lam, np.array([1.7]), sig)[0]
    assert abs(peak - D.gaussian_delta(0.0, sig) / 6.0) <= 1e-12 * peak


@pytest.mark.parametrize("n,seed", [(3, 1), (6, 2)])
def test_absorption_sum_rule(n, seed):
    """Completeness of the biorthonormal pairs (Theorem 3, Y^H X = I over all 2n):
    sum over +-lambda of (d_r^H x)(y^H d_l) = d_r^H d_l. The broadened spectra of
    both halves therefore integrate to d_r^H d_l, and the positive half alone to
    sum_j w_j (Eq. absp, unit-integral Gaussians)."""
    p = make_problem(n, seed)
    s = D.solve(p.A, p.B)
    rng = np.random.default_rng(seed)
    dr = rng.standard_normal(2 * n) + 1j * rng.standard_normal(2 * n)
    dl = rng.standard_normal(2 * n) + 1j * rng.standard_normal(2 * n)
    lf, Xf, Yf = D.full_pairs(s.lam, s.X)
    wf = D.weights(Xf, Yf, dr, dl)
    assert abs(wf.sum() - dr.conj() @ dl) <= 1e-12 * np.linalg.norm(dr) * np.linalg.norm(dl)
    w = D.weights(s.X, s.Y, dr, dl)
    sig = 0.02
    om = np.linspace(0.0, s.lam.max() + 12 * sig, 200001)
    eps = D.absorption(s.lam, w, om, sig)
    assert abs(np.trapezoid(eps, om) - w.sum()) <= 1e-9 * np.abs(w).sum()
    om2 = np.linspace(-s.lam.max() - 12 * sig, s.lam.max() + 12 * sig, 400001)
    both = D.absorption(lf, wf, om2, sig)
    assert abs(np.trapezoid(both, om2) - dr.conj() @ dl) <= 1e-9 * np.abs(wf).sum()


@pytest.mark.parametrize("n,seed", [(5, 3), (12, 4)])
def test_tda_eigenvalues(n, seed):
    """B = 0 makes H block diagonal (Eq. 1): its positive eigenvalues are those of
    A exactly, the Tamm-Dancoff values; with B != 0 every lambda_j(H) lies below
    lambda_j(A) (Theorem 4)."""
    p = make_problem(n, seed)
    tda = D.tda_eigenvalues(p.A)
    s0 = D.solve(p.A, np.zeros_like(p.B))
    assert _rel(s0.lam, tda) <= 1e-13
    s = D.solve(p.A, p.B)
    assert np.all(s.lam <= tda * (1 + 1e-14))


# --- Algorithm 2 (real problems, Theorem 5) --------------------------------------


@pytest.mark.parametrize("n,seed", [(1, 3), (6, 4), (40, 5)])
def test_alg2_against_definition(n, seed):
    """Algorithm 2's outputs satisfy the definitions: H [X1; X2] = [X1; X2] Lambda
    with H = [A B; -B -A] built literally (Eq. H-real), X1^T X1 - X2^T X2 = I
    (Theorem 5 normalization), and Lambda equals the positive eigenvalues from
    the Hermitian-definite route of the complex oracle."""
    p = make_problem(n, seed, real=True)
    s = alg2.solve_real(p.A, p.B)
    A, B = alg2.symmetrize_real(p.A, p.B)
    H = np.block([[A, B], [-B, -A]])
    X = np.concatenate([s.X1, s.X2], axis=0)
    assert np.max(np.abs(H @ X - X * s.lam[None, :])) <= 1e-12 * np.abs(H).sum(axis=1).max()
    assert np.max(np.abs(s.X1.T @ s.X1 - s.X2.T @ s.X2 - np.eye(n))) <= 1e-12
    ref = D.solve(p.A.astype(complex), p.B.astype(complex))
    assert _rel(s.lam, ref.lam) <= 1e-13


def test_alg2_n1_closed_form():
    """n = 1: lambda = sqrt((a + b)(a - b)) = sqrt(a^2 - b^2) (Section 2's real case)."""
    a, b = 2.5, 0.7
    s = alg2.solve_real(np.array([[a]]), np.array([[b]]))
    assert abs(s.lam[0] - np.sqrt(a * a - b * b)) <= 1e-15 * s.lam[0]
    assert abs(s.X1[0, 0] ** 2 - s.X2[0, 0] ** 2 - 1.0) <= 1e-14


def test_planted_mistake_alg2_factor_is_caught(monkeypatch):
    """Dropping the (1/2) Lambda^{-1/2} factor (the printed step 3) breaks the
    normalization pin; swapping L1 and L2 breaks the residual pin."""

    def no_factor(L1, L2, U, s, V):
        return L2 @ U + L1 @ V, L2 @ U - L1 @ V

    monkeypatch.setattr(alg2, "step3_vectors", no_factor)
    with pytest.raises(AssertionError):
        test_alg2_against_definition(6, 4)
    monkeypatch.undo()

    orig = alg2.step1_cholesky

    def swapped(A, B):
        L1, L2 = orig(A, B)
        return L2, L1

    monkeypatch.setattr(alg2, "step1_cholesky", swapped)
    with pytest.raises(AssertionError):
        test_alg2_against_definition(6, 4)


# --- planted mistakes: each must be caught by a pin -----------------------------


def test_planted_mistake_in_M_is_caught(monkeypatch):
    """Sign error in M's (1,2) block breaks the Theorem 2 identity."""
    n = 5
    p = make_problem(n, 1)
    A, B = D.symmetrize_lower(p.A, p.B)

    def bad_M(A, B):
        return np.block([[(A + B).real, -(A - B).imag], [-(A + B).imag, (A - B).real]])

    Q = D.build_Q(n)
    lhs = Q.conj().T @ D.build_H(A, B) @ Q
    assert np.max(np.abs(lhs - (-1j) * D.build_J(n) @ bad_M(A, B))) > 1e-3


def test_planted_mistake_transpose_is_caught(monkeypatch):
    """Rebuilding B's upper triangle with ^H instead of ^T (B is complex symmetric, Eq. 2)
    is caught by the brute-force eigenvectors. (A's upper triangle is never read by the
    pencil route: its Cholesky reads Omega's lower triangle only.)"""
    n = 3
    p = make_problem(n, 12)
    lb, Xb, _ = brute.positive_pairs(p.A, p.B)

    def bad_sym(A, B):
        Al = np.tril(A, -1)
        Bl = np.tril(B, -1)
        return (Al + Al.conj().T + np.diag(np.diag(A).real)).astype(complex), (
            Bl + Bl.conj().T + np.diag(np.diag(B))
        ).astype(complex)

    monkeypatch.setattr(D, "symmetrize_lower", bad_sym)
    s = D.solve(p.A, p.B)
    S = D.S_signs(n)[:, None]
    worst = 0.0
    for j in range(n):
        P1 = np.outer(s.X[:, j], (S * s.X)[:, j].conj())
        P2 = np.outer(Xb[:, j], (S * Xb)[:, j].conj())
        worst = max(worst, np.max(np.abs(P1 - P2)))
    assert worst > 1e-4


def test_planted_mistake_normalization_is_caught():
    """Using y = x instead of y = S x breaks Table 1's biorthogonality metric."""
    n = 8
    p = make_problem(n, 2)
    s = D.solve(p.A, p.B)
    Xf = np.concatenate([s.X, D.negative_half(s.X)], axis=1)
    bad = np.linalg.norm(Xf.conj().T @ Xf - np.eye(2 * n)) / np.sqrt(2 * n)
    assert bad > 1e-3


def test_planted_mistake_dos_half_spectrum_is_caught(monkeypatch):
    """A density summed over the positive half only (dropping Theorem 1's -lambda_j)
    fails the normalization and symmetry pins."""

    def bad_dos(lam, omega, sigma):
        return D.gaussian_delta(omega[:, None] - lam[None, :], sigma).sum(axis=1) / (2 * lam.shape[0])

    monkeypatch.setattr(D, "dos", bad_dos)
    with pytest.raises(AssertionError):
        test_dos_normalization_symmetry_and_peaks()
