"""Spectral density (Eq. DOS) and broadened absorption spectrum (Eq. absp) on the
GPU, against the oracle's plain sums, and the Tamm-Dancoff comparison of
Section 5 (B = 0 gives the eigenvalues of A; with B the BSE eigenvalues lie
below them, Theorem 4)."""
import numpy as np
import pytest

from oracle import definition as D
from paper_1501_03830_gb300.synth import make_problem
from tests.helpers import torch_cuda

pytestmark = pytest.mark.gpu


def _lib():
    from paper_1501_03830_gb300 import bse

    return bse.lib(), bse


@pytest.mark.parametrize("n,k,sigma", [(1, 1, 0.1), (700, 2001, 5e-3), (5000, 300, 5e-4), (257, 513, 2.0)])
def test_stage_broaden_matches_oracle(n, k, sigma):
    """Random positive eigenvalues and complex weights; the grid spans both signs
    and runs past the spectrum (pure zeros there); k not a multiple of the block."""
    torch = torch_cuda()
    L, bse = _lib()
    rng = np.random.default_rng(n + k)
    lam = np.sort(rng.uniform(0.5, 3.0, n))
    w = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    om = np.linspace(-3.5, 4.0, k)
    dl = torch.from_numpy(lam).cuda()
    dw = torch.from_numpy(w).cuda()
    dom = torch.from_numpy(om).cuda()
    dos = torch.empty(k, dtype=torch.float64, device="cuda")
    eps = torch.empty(k, dtype=torch.complex128, device="cuda")
    bse.check(L.bse_stage_broaden(n, dl.data_ptr(), dw.data_ptr(), k, dom.data_ptr(), sigma, dos.data_ptr(),
                                  eps.data_ptr(), None), "broaden")
    torch.cuda.synchronize()
    ref_d = D.dos(lam, om, sigma)
    ref_e = D.absorption(lam, w, om, sigma)
    got_d = dos.cpu().numpy()
    got_e = eps.cpu().numpy()
    assert np.max(np.abs(got_d - ref_d)) <= 1e-13 * max(ref_d.max(), 1e-300) + 1e-300
    assert np.max(np.abs(got_e - ref_e)) <= 1e-13 * np.abs(w).sum() * D.gaussian_delta(0.0, sigma)
    # DOS alone (no weights) gives the same density
    dos2 = torch.empty(k, dtype=torch.float64, device="cuda")
    bse.check(L.bse_stage_broaden(n, dl.data_ptr(), None, k, dom.data_ptr(), sigma, dos2.data_ptr(), None, None),
              "broaden")
    torch.cuda.synchronize()
    assert torch.equal(dos, dos2)


def test_stage_broaden_rejects_bad_arguments():
    torch = torch_cuda()
    L, _ = _lib()
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    assert L.bse_stage_broaden(1, x.data_ptr(), None, 1, x.data_ptr(), 0.0, x.data_ptr(), None, None) < 0
    assert L.bse_stage_broaden(1, x.data_ptr(), None, 1, x.data_ptr(), 0.1, x.data_ptr(), x.data_ptr(), None) < 0
    assert L.bse_stage_broaden(0, x.data_ptr(), None, 1, x.data_ptr(), 0.1, x.data_ptr(), None, None) < 0


@pytest.mark.parametrize("precision", ["fp64", "mixed_refined"])
def test_absorption_of_a_solve_matches_oracle(precision):
    """Solve n = 96, keep the solution, broaden on the host grid with the
    problem's dipoles; compare with the oracle's spectra of its own solve. The
    eigenvalues agree to ~1e-14 relative, so the Gaussians (sigma = 5e-3) agree
    to ~1e-11 of their peak."""
    torch_cuda()
    _, bse = _lib()
    p = make_problem(96, 5)
    ctx = bse.Context(0)
    try:
        lam, _, _, info, sol = ctx.solve(p.A, p.B, precision=precision, keep=True)
        om = np.linspace(0.0, 12.0, 3001)
        sig = 5e-3
        dos, eps = ctx.absorption(sol, om, sig, p.d_r, p.d_l)
        dos_only, none = ctx.absorption(sol, om, sig)
        sol.free()
    finally:
        ctx.close()
    assert none is None and np.array_equal(dos, dos_only)
    ref = D.solve(p.A, p.B)
    w = D.weights(ref.X, ref.Y, p.d_r, p.d_l)
    g0 = D.gaussian_delta(0.0, sig)
    assert np.max(np.abs(dos - D.dos(ref.lam, om, sig))) <= 1e-9 * g0 / (2 * p.n)
    assert np.max(np.abs(eps - D.absorption(ref.lam, w, om, sig))) <= 1e-9 * g0 * np.abs(w).sum()


@pytest.mark.parametrize("n,seed", [(64, 11), (300, 12)])
def test_tda_comparison(n, seed):
    """Section 5's comparison: the solver with B = 0 returns the eigenvalues of A
    (the TDA values); with B every BSE eigenvalue is below its TDA value."""
    torch_cuda()
    _, bse = _lib()
    p = make_problem(n, seed)
    ctx = bse.Context(0)
    try:
        lam_tda = ctx.solve(p.A, np.zeros_like(p.B), precision="fp64")[0]
        lam = ctx.solve(p.A, p.B, precision="fp64")[0]
    finally:
        ctx.close()
    ref = D.tda_eigenvalues(p.A)
    assert np.max(np.abs(lam_tda - ref) / ref) <= 1e-12
    assert np.all(lam <= lam_tda * (1 + 1e-13))
