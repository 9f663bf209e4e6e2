"""Algorithm 2 (real Bethe-Salpeter problems, Theorem 5) on the GPU: bse_solve_real
against the oracle's Algorithm 2 and against the definitions."""
import numpy as np
import pytest

from oracle import alg2
from paper_1501_03830_gb300.synth import make_problem
from tests.helpers import torch_cuda

pytestmark = pytest.mark.gpu

EPS = 2.0 ** -52


def _ctx():
    from paper_1501_03830_gb300 import bse

    return bse, bse.Context(0)


def _H(p):
    A, B = alg2.symmetrize_real(p.A, p.B)
    return np.block([[A, B], [-B, -A]])


@pytest.mark.parametrize("n,seed,precision", [(64, 21, "fp64"), (300, 22, "fp64"), (64, 23, "mixed_refined"),
                                              (333, 24, "mixed_refined"), (1, 25, "fp64")])
def test_solve_real_matches_oracle(n, seed, precision):
    torch_cuda()
    bse, ctx = _ctx()
    p = make_problem(n, seed, real=True)
    try:
        lam, X1, X2, info = ctx.solve_real(p.A, p.B, precision=precision)
    finally:
        ctx.close()
    assert info.status == 0
    ref = alg2.solve_real(p.A, p.B)
    tol = 1e-12 if precision == "fp64" else 1e-10
    assert np.max(np.abs(lam - ref.lam) / ref.lam) <= tol
    X = np.concatenate([X1, X2], axis=0)
    H = _H(p)
    r = np.linalg.norm(H @ X - X * lam[None, :], axis=0) / (np.linalg.norm(H) * np.linalg.norm(X, axis=0))
    assert np.max(r) <= 100 * n * EPS
    assert np.max(np.abs(X1.T @ X1 - X2.T @ X2 - np.eye(n))) <= 1e-10
    # column convention: the largest-modulus entry is positive
    idx = np.argmax(np.abs(X), axis=0)
    assert np.all(X[idx, np.arange(n)] > 0)
    # same vectors as the oracle's up to the column sign
    Xr = np.concatenate([ref.X1, ref.X2], axis=0)
    sgn = np.sign(np.sum(X * Xr, axis=0))
    assert np.max(np.abs(X - Xr * sgn[None, :])) <= 1e-8 * np.max(np.abs(Xr))


def test_solve_real_device_inputs_and_outputs():
    torch = torch_cuda()
    bse, ctx = _ctx()
    p = make_problem(128, 26, real=True)
    dA = torch.from_numpy(np.ascontiguousarray(np.asfortranarray(p.A).T)).cuda()
    dB = torch.from_numpy(np.ascontiguousarray(np.asfortranarray(p.B).T)).cuda()
    lam = torch.empty(128, dtype=torch.float64, device="cuda")
    X1 = torch.empty(128 * 128, dtype=torch.float64, device="cuda")
    X2 = torch.empty(128 * 128, dtype=torch.float64, device="cuda")
    try:
        ctx.solve_real(dA, dB, precision="fp64", out={"lambda": lam, "X1": X1, "X2": X2})
        torch.cuda.synchronize()
        lam_h, X1_h, X2_h, _ = ctx.solve_real(p.A, p.B, precision="fp64")
    finally:
        ctx.close()
    assert np.array_equal(lam.cpu().numpy(), lam_h)
    assert np.array_equal(X1.cpu().numpy().reshape(128, 128).T, X1_h)
    assert np.array_equal(X2.cpu().numpy().reshape(128, 128).T, X2_h)


def test_solve_real_not_definite():
    """A - B indefinite: the second factorization meets a non-positive pivot; the
    reported column is counted from n."""
    torch_cuda()
    bse, ctx = _ctx()
    n = 40
    p = make_problem(n, 27, real=True)
    B = p.B.copy()
    B[5, 5] = p.A[5, 5] + 1.0  # (A - B)[5, 5] < 0
    try:
        with pytest.raises(bse.BSEError) as e:
            ctx.solve_real(p.A, B, precision="fp64")
    finally:
        ctx.close()
    assert e.value.code == bse.BSE_ERR_NOT_DEFINITE


def test_solve_real_n2048_product_eigenvalues():
    """Eq. H-real at n = 2048: lambda^2 are the eigenvalues of (A - B)(A + B),
    computed through the Cholesky factor of A + B as a symmetric problem."""
    import scipy.linalg as sla

    torch_cuda()
    bse, ctx = _ctx()
    p = make_problem(2048, 2049, real=True)
    try:
        lam, X1, X2, _ = ctx.solve_real(p.A, p.B, precision="fp64")
    finally:
        ctx.close()
    A, B = alg2.symmetrize_real(p.A, p.B)
    L = np.linalg.cholesky(A + B)
    ref = np.sqrt(np.sort(sla.eigh(L.T @ (A - B) @ L, eigvals_only=True)))
    assert np.max(np.abs(lam - ref) / ref) <= 1e-11
    cols = np.linspace(0, 2047, 24).astype(int)
    G = X1[:, cols].T @ X1[:, cols] - X2[:, cols].T @ X2[:, cols]
    assert np.max(np.abs(G - np.eye(len(cols)))) <= 1e-10
