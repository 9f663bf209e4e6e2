"""Pins of the two-stage (band) reduction restatement in oracle/sbr.py against
facts that do not come from it: the band and tridiagonal structure, orthogonal
similarity W = Q T Q^T, Q e_1 = e_1, and -- by the implicit-Q theorem -- the
sub-diagonal magnitudes of Algorithm 3's one-stage reduction (oracle/alg1.py, a
different algorithm reaching the same unique result)."""
import numpy as np
import pytest

from oracle import alg1, sbr
from paper_1501_03830_gb300.synth import make_problem


def _W(n, seed):
    p = make_problem(n, seed)
    return alg1.step3_W(alg1.step2_cholesky(alg1.step1_M(p.A, p.B)))


@pytest.mark.parametrize("n,seed,b", [(8, 1, 2), (20, 2, 4), (32, 3, 8), (17, 4, 3), (6, 5, 1)])
def test_two_stage_structure_and_similarity(n, seed, b):
    W = _W(n, seed)
    m = W.shape[0]
    r = sbr.two_stage(W, b)
    i, j = np.indices((m, m))
    scale = np.abs(W).max()
    assert np.max(np.abs(r.Bw[np.abs(i - j) > b]), initial=0.0) <= 1e-13 * scale
    assert np.max(np.abs(r.T[np.abs(i - j) > 1]), initial=0.0) <= 1e-13 * scale
    assert np.max(np.abs(r.T + r.T.T)) <= 1e-13 * scale  # skew kept
    Q = r.Q1 @ r.Q2
    assert np.max(np.abs(Q.T @ Q - np.eye(m))) <= 1e-13
    assert np.max(np.abs(Q @ r.T @ Q.T - W)) <= 1e-13 * scale
    assert np.array_equal(Q[:, 0], np.eye(m)[:, 0])


@pytest.mark.parametrize("n,seed,b", [(16, 6, 4), (24, 7, 6)])
def test_two_stage_matches_one_stage_subdiagonal(n, seed, b):
    """Q e_1 = e_1 in both reductions, so |T[k+1, k]| agree (implicit-Q theorem)."""
    W = _W(n, seed)
    r = sbr.two_stage(W, b)
    t = alg1.alg3_step1_tridiagonalize(W)
    scale = np.abs(W).max()
    assert np.max(np.abs(np.abs(np.diag(r.T, -1)) - np.abs(t.beta))) <= 1e-11 * scale


def test_two_stage_spectrum():
    """The eigenvalues +-i sigma of the skew tridiagonal equal those of W."""
    rng = np.random.default_rng(9)
    X = rng.standard_normal((30, 30))
    W = X - X.T
    r = sbr.two_stage(W, 5)
    ew = np.sort(np.linalg.eigvals(W).imag)
    et = np.sort(np.linalg.eigvals(r.T).imag)
    assert np.max(np.abs(ew - et)) <= 1e-12 * np.abs(ew).max()


def test_planted_mistake_one_sided_panel_is_caught(monkeypatch):
    """A stage-1 panel transform applied from one side only is not a similarity:
    the reconstruction pin fails."""

    def bad(W, b):
        A = np.array(W, dtype=np.float64)
        m = A.shape[0]
        Q = np.eye(m)
        for k in range(0, m, b):
            r0 = k + b
            if r0 >= m - 1:
                break
            Qk, _ = np.linalg.qr(A[r0:, k:k + b], mode="complete")
            A[r0:, :] = Qk.T @ A[r0:, :]
            Q[:, r0:] = Q[:, r0:] @ Qk
        return A, Q

    monkeypatch.setattr(sbr, "dense_to_band", bad)
    with pytest.raises(AssertionError):
        test_two_stage_structure_and_similarity(8, 1, 2)
