"""Pins of the representation-tree tridiagonal eigensolver in oracle/mrrr.py:
eigenvalues against a library symmetric eigensolver (a special case it reduces
to), orthogonality and residuals on the classic hard cases (Wilkinson's W21+ and
glued copies of it, whose eigenvalues agree in pairs to ~1e-14), the BSE
eigenvalues through the tridiagonal form of Algorithm 3 (Section 3.3), and the
role of the tree: without child representations the vectors of a tight cluster
are not orthogonal."""
import numpy as np
import pytest

from oracle import alg1, mrrr
from oracle import definition as D
from paper_1501_03830_gb300.synth import make_problem


def _check(a, b, gaptol=1e-3):
    lam, Z, tree = mrrr.eigh_tridiagonal(a, b, gaptol)
    T = np.diag(a) + np.diag(b, 1) + np.diag(b, -1)
    nrm = np.abs(T).sum(axis=1).max()
    ref = np.linalg.eigvalsh(T)
    n = len(a)
    return (np.max(np.abs(lam - ref)) / nrm, np.max(np.abs(Z.T @ Z - np.eye(n))),
            np.max(np.linalg.norm(T @ Z - Z * lam, axis=0)) / nrm, tree)


def _glued(copies, glue):
    a = np.tile(np.abs(np.arange(21) - 10.0), copies)
    b = np.tile(np.concatenate([np.ones(20), [glue]]), copies)[:-1]
    return a, b


def test_wilkinson_w21():
    ev, orth, res, tree = _check(np.abs(np.arange(21) - 10.0), np.ones(20))
    assert ev <= 1e-14 and orth <= 1e-12 and res <= 1e-14
    assert max(d for d, _ in tree) >= 1  # its close pairs need child representations


@pytest.mark.parametrize("glue", [1e-10, 1e-14])
def test_glued_wilkinson(glue):
    ev, orth, res, _ = _check(*_glued(5, glue))
    assert ev <= 1e-14 and orth <= 1e-12 and res <= 1e-14


def test_random_tridiagonal():
    rng = np.random.default_rng(0)
    ev, orth, res, _ = _check(rng.standard_normal(150), rng.standard_normal(149))
    assert ev <= 1e-14 and orth <= 1e-12 and res <= 1e-14


@pytest.mark.parametrize("n,seed", [(12, 3), (30, 4)])
def test_bse_tridiagonal_form(n, seed):
    """-i D^H T D of Algorithm 3 step 2 is the real tridiagonal with zero diagonal
    and off-diagonal -beta; its positive eigenvalues are the BSE eigenvalues."""
    p = make_problem(n, seed)
    W = alg1.step3_W(alg1.step2_cholesky(alg1.step1_M(p.A, p.B)))
    t = alg1.alg3_step1_tridiagonalize(W)
    lam, Z, _ = mrrr.eigh_tridiagonal(np.zeros(2 * n), -t.beta)
    ref = D.solve(p.A, p.B).lam
    assert np.max(np.abs(lam[n:] - ref) / ref) <= 1e-12
    assert np.max(np.abs(lam[:n] + ref[::-1]) / ref[::-1]) <= 1e-12
    assert np.max(np.abs(Z.T @ Z - np.eye(2 * n))) <= 1e-12


def test_without_tree_cluster_vectors_are_not_orthogonal():
    """gaptol = 0 makes every eigenvalue a singleton of the root representation:
    on glued W21+ the vectors of the near-coincident pairs then collapse onto
    each other, which the tree prevents."""
    _, orth0, _, _ = _check(*_glued(5, 1e-10), gaptol=0.0)
    _, orth, _, _ = _check(*_glued(5, 1e-10))
    assert orth0 > 1e-3 and orth <= 1e-12


def test_peeling_a_cluster_larger_than_one_over_gaptol():
    """With gaptol = 0.05, the positive half of a BSE tridiagonal of n = 100 is one
    cluster of more than 1/gaptol members at the root; the tree peels it (child
    shifts within a quarter of mean gap / gaptol of its first member) and still
    gives eigenvalues to 1e-14 and orthogonal vectors."""
    n = 100
    p = make_problem(n, 5)
    W = alg1.step3_W(alg1.step2_cholesky(alg1.step1_M(p.A, p.B)))
    t = alg1.alg3_step1_tridiagonalize(W)
    ev, orth, res, tree = _check(np.zeros(2 * n), -t.beta, gaptol=0.05)
    # residual bar: O(m eps ||T||), the twisted-factorization bound, with m = 2n
    assert ev <= 1e-14 and orth <= 1e-12 and res <= 2 * (2 * n) * 2.0 ** -52
    assert max(s for _, s in tree) * 0.05 > 1.0  # a cluster of more than 1/gaptol members
