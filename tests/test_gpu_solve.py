"""End-to-end parity of bse_solve / bse_spectrum (through the C ABI) with the
oracle's definition route, on seeded inputs of the paper's shape.

Bars (the benchmark spec): relative eigenvalue error <= 1e-10 and scaled residual
max_j ||H x_j - lambda_j x_j|| / (||H||_F ||x_j||) <= 100 n eps for the FP64 and
refined paths; the unrefined FP32 path is reported and held to a loose bound.
Eigenvectors are compared phase-free (projectors x y^H and the weights).
"""
import numpy as np
import pytest

from oracle import definition as D
from paper_1501_03830_gb300.synth import make_problem
from tests.helpers import dev_c128, host_colmajor, projector_gap, rel_err, torch_cuda

pytestmark = pytest.mark.gpu

EPS = 2.220446049250313e-16


def _ctx():
    from paper_1501_03830_gb300 import bse

    return bse, bse.Context(0)


def _check(p, lam, X, ref, tol_lam, n):
    assert rel_err(lam, ref.lam) <= tol_lam
    res = D.scaled_residuals(p.A, p.B, lam, X)
    assert np.max(res) <= 100 * n * EPS
    return res


@pytest.mark.parametrize("n", [1, 2, 3, 5, 16, 33, 64, 100, 257])
def test_fp64_vs_oracle(n):
    torch_cuda()
    bse, ctx = _ctx()
    p = make_problem(n, 1000 + n)
    ref = D.solve(p.A, p.B)
    lam, X, Y, info, sol = ctx.solve(p.A, p.B, precision="fp64", want_Y=True, keep=True)
    _check(p, lam, X, ref, 1e-12, n)
    assert np.array_equal(Y[:n], X[:n]) and np.array_equal(Y[n:], -X[n:])
    m = D.table1_metrics(p.A, p.B, lam, X)
    # Table 1 metrics (the paper's are ~1e-15): the reorthogonalized tridiagonal
    # eigenvectors (remark 2) keep the FP64 path at that level
    assert m["res_F"] <= 1e-13 and m["biorth"] <= 1e-13, m
    if n <= 64:
        assert projector_gap(X, ref.X, n) <= 1e-9
    w = ctx.spectrum(sol, p.d_r, p.d_l)
    wref = D.weights(ref.X, ref.Y, p.d_r, p.d_l)
    assert np.max(np.abs(w - wref)) <= 1e-9 * np.max(np.abs(wref))
    sol.free()
    ctx.close()


@pytest.mark.parametrize("n", [1, 7, 64, 150, 600])
def test_mixed_and_refined(n):
    torch_cuda()
    bse, ctx = _ctx()
    p = make_problem(n, 2000 + n)
    ref = D.solve(p.A, p.B)
    lam32, X32, _, info32, _ = ctx.solve(p.A, p.B, precision="mixed")
    err32 = rel_err(lam32, ref.lam)
    assert err32 <= 1e-4  # FP32 bulk: reported, not hidden
    lam, X, _, info, _ = ctx.solve(p.A, p.B, precision="mixed_refined")
    _check(p, lam, X, ref, 1e-10, n)
    assert info.sweeps >= 1
    m = D.table1_metrics(p.A, p.B, lam, X)
    # Table 1's Frobenius metrics over all 2n pairs: the couplings of the positive
    # half with the negative half sit at the rounding of the last sweep's FP32 update
    assert m["biorth"] <= 1e-11 and m["res_F"] <= 1e-11, m
    ctx.close()


def test_device_pointers_and_lower_triangle():
    """Device inputs/outputs give the same result as host ones; upper triangles are ignored."""
    torch = torch_cuda()
    bse, ctx = _ctx()
    n = 48
    p = make_problem(n, 77)
    lam_h, X_h, _, _, _ = ctx.solve(p.A, p.B, precision="fp64")
    Ag = p.A.copy()
    Bg = p.B.copy()
    iu = np.triu_indices(n, 1)
    Ag[iu] = 5.0 - 3.0j
    Bg[iu] = np.nan
    A = dev_c128(torch, Ag)
    B = dev_c128(torch, Bg)
    lam = torch.empty(n, dtype=torch.float64, device="cuda")
    X = torch.empty(2 * n * n, dtype=torch.complex128, device="cuda")
    ctx.solve(A, B, precision="fp64", out={"lambda": lam, "X": X})
    torch.cuda.synchronize()
    assert np.array_equal(lam.cpu().numpy(), lam_h)
    assert np.array_equal(host_colmajor(X, (2 * n, n)), X_h)
    ctx.close()


def test_not_definite_reports_column():
    torch_cuda()
    bse, ctx = _ctx()
    n = 20
    p = make_problem(n, 5)
    B = p.B.copy()
    B[3, 3] = 10.0  # |b_33| > a_33: Omega indefinite
    with pytest.raises(bse.BSEError) as ei:
        ctx.solve(p.A, B, precision="fp64")
    assert ei.value.code == bse.BSE_ERR_NOT_DEFINITE
    # the context stays usable afterwards
    lam, X, _, _, _ = ctx.solve(p.A, p.B, precision="fp64")
    assert rel_err(lam, D.solve(p.A, p.B).lam) <= 1e-12
    ctx.close()


def test_real_case_config():
    """Real special case (A, B real symmetric): lambda^2 = eig((A-B)(A+B)) (Section 2.1)."""
    torch_cuda()
    bse, ctx = _ctx()
    n = 96
    p = make_problem(n, 31, real=True)
    lam, X, _, _, _ = ctx.solve(p.A.astype(complex), p.B.astype(complex), precision="fp64")
    A = np.tril(p.A) + np.tril(p.A, -1).T
    B = np.tril(p.B) + np.tril(p.B, -1).T
    L1 = np.linalg.cholesky(A + B)
    mu = np.sort(np.linalg.eigvalsh(L1.T @ (A - B) @ L1))
    assert rel_err(lam, np.sqrt(mu)) <= 1e-12
    ctx.close()


def test_invalid_arguments():
    torch_cuda()
    bse, ctx = _ctx()
    L = bse.lib()
    A = np.zeros((4, 4), dtype=complex, order="F")
    lam = np.zeros(4)
    assert L.bse_solve(ctx.handle, 0, bse.ptr(A), 4, bse.ptr(A), 4, 0, bse.ptr(lam), None, None, None, None) == bse.BSE_ERR_ARG
    assert L.bse_solve(ctx.handle, 4, bse.ptr(A), 3, bse.ptr(A), 4, 0, bse.ptr(lam), None, None, None, None) == bse.BSE_ERR_ARG
    assert L.bse_solve(ctx.handle, 4, bse.ptr(A), 4, bse.ptr(A), 4, 7, bse.ptr(lam), None, None, None, None) == bse.BSE_ERR_ARG
    ctx.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_refined"])
@pytest.mark.parametrize("n", [3, 64, 300])
def test_eigenvector_phase_convention(precision, n):
    """The returned x_j have a fixed phase: the largest-modulus entry of the top
    half (the first of equal ones) is real and positive, with y_j = diag(I, -I) x_j
    exactly and the solution otherwise as before (residuals, projectors)."""
    torch_cuda()
    bse, ctx = _ctx()
    p = make_problem(n, 3000 + n)
    lam, X, Y, _, _ = ctx.solve(p.A, p.B, precision=precision, want_Y=True)
    # an entry of (within rounding) the largest modulus of the top half is exactly
    # real and positive in every column (which of two near-equal entries the kernel
    # took is not re-derived here: a one-ulp tie could go either way)
    top = X[:n]
    mx = np.max(np.abs(top), axis=0)
    lead = (top.imag == 0.0) & (top.real > 0.0) & (np.abs(top) >= mx * (1 - 1e-12))
    assert np.all(lead.any(axis=0))
    assert np.array_equal(Y[:n], X[:n]) and np.array_equal(Y[n:], -X[n:])
    ref = D.solve(p.A, p.B)
    tol = 1e-4 if precision == "mixed" else 1e-10
    assert rel_err(lam, ref.lam) <= tol
    if precision != "mixed":
        assert np.max(D.scaled_residuals(p.A, p.B, lam, X)) <= 100 * n * EPS
        if n <= 64:
            assert projector_gap(X, ref.X, n) <= 1e-8
    ctx.close()
