"""The representation-tree (MRRR) tridiagonal eigensolver on the device
(bse_stage_tdeig_mrrr, k_mrrr.cu) against the oracle's tree (oracle/mrrr.py) and a
library symmetric eigensolver, on the classic hard cases (Wilkinson's W21+ and
glued copies of it, whose eigenvalues agree in pairs to ~1e-14), random
tridiagonals, tight clusters, a dense BSE tridiagonal that needs the peeling
levels, and the BSE form of Algorithm 3 step 2 (Section 3.3, remark 2), then whole
FP64 solves with the tree's vectors in place of the reorthogonalized ones."""
import numpy as np
import pytest

from oracle import alg1, mrrr
from oracle import definition as D
from paper_1501_03830_gb300.synth import make_problem
from tests.helpers import rel_err, torch_cuda

pytestmark = pytest.mark.gpu

EPS = 2.0 ** -52


def _lib():
    from paper_1501_03830_gb300 import bse

    return bse.lib(), bse


def _device_mrrr(torch, a, b, il, iu, gaptol=1e-3, bse_form=0, bse_signs=0):
    L, bse = _lib()
    m = len(b) + 1
    nz = iu - il
    da = None if a is None else torch.tensor(np.asarray(a, dtype=np.float64), device="cuda")
    db = torch.tensor(np.concatenate([np.asarray(b, dtype=np.float64), [0.0]]), device="cuda")
    lam = torch.empty(nz, dtype=torch.float64, device="cuda")
    Z = torch.empty(m * nz, dtype=torch.float64, device="cuda")
    work = torch.empty(L.bse_stage_tdeig_mrrr_worksize(m, il, iu), dtype=torch.uint8, device="cuda")
    st = torch.zeros(4, dtype=torch.int32, device="cuda")
    bse.check(L.bse_stage_tdeig_mrrr(m, None if da is None else da.data_ptr(), db.data_ptr(), bse_form, il, iu,
                                     gaptol, lam.data_ptr(), Z.data_ptr(), nz, bse_signs, work.data_ptr(),
                                     st.data_ptr(), None), "tdeig_mrrr")
    torch.cuda.synchronize()
    assert st.cpu().numpy()[0] == 0
    return lam.cpu().numpy(), Z.cpu().numpy().reshape(m, nz)


def _glued(copies, glue):
    a = np.tile(np.abs(np.arange(21) - 10.0), copies)
    b = np.tile(np.concatenate([np.ones(20), [glue]]), copies)[:-1]
    return a, b


def _cases():
    rng = np.random.default_rng(0)
    return {
        "w21": (np.abs(np.arange(21) - 10.0), np.ones(20)),
        "glued_1e-10": _glued(5, 1e-10),
        "glued_1e-14": _glued(5, 1e-14),
        "random_150": (rng.standard_normal(150), rng.standard_normal(149)),
    }


@pytest.mark.parametrize("case", ["w21", "glued_1e-10", "glued_1e-14", "random_150"])
def test_mrrr_general_tridiagonal_matches_oracle(case):
    """All eigenpairs: eigenvalues to 1e-14 ||T|| of a library solver and of the
    oracle's tree, vectors orthogonal to 1e-12 with residuals at rounding level --
    the oracle's own pins, met by the device."""
    torch = torch_cuda()
    a, b = _cases()[case]
    m = len(a)
    lam, Z = _device_mrrr(torch, a, b, 0, m)
    T = np.diag(a) + np.diag(b, 1) + np.diag(b, -1)
    nrm = np.abs(T).sum(axis=1).max()
    ref = np.linalg.eigvalsh(T)
    lam_o, Z_o, _ = mrrr.eigh_tridiagonal(a, b)
    assert np.max(np.abs(lam - ref)) / nrm <= 1e-14
    assert np.max(np.abs(lam - lam_o)) / nrm <= 1e-14
    assert np.max(np.abs(Z.T @ Z - np.eye(m))) <= 1e-12
    assert np.max(np.linalg.norm(T @ Z - Z * lam, axis=0)) / nrm <= 1e-14
    # the oracle's tree gives the same vectors (up to sign) where an eigenvalue is
    # well separated from the others
    gaps = np.minimum(np.abs(np.diff(ref, prepend=-np.inf)), np.abs(np.diff(ref, append=np.inf)))
    sep = gaps > 1e-3 * nrm
    dots = np.abs(np.sum(Z[:, sep] * Z_o[:, sep], axis=0))
    assert np.all(np.abs(dots - 1.0) <= 1e-10)


def test_mrrr_subset_and_tight_clusters():
    """Ten eigenvalues 1e-9 apart in each of twenty groups (the zero-diagonal
    Golub-Kahan form of a bidiagonal with those singular values): the positive
    half alone, to FP64 accuracy and orthogonal without reorthogonalization
    (twisted factorizations on the root matrix leave them ~1e-6 off)."""
    torch = torch_cuda()
    rng = np.random.default_rng(11)
    sig = np.concatenate([1.0 + 0.4 * g + 1e-9 * np.arange(10) for g in range(20)])
    n = sig.shape[0]
    m = 2 * n
    Qa, _ = np.linalg.qr(rng.standard_normal((n, n)))
    Qb, _ = np.linalg.qr(rng.standard_normal((n, n)))
    from tests.test_gpu_stages import _bidiagonalize

    d, f = _bidiagonalize(Qa @ np.diag(sig) @ Qb.T)
    alpha = np.zeros(m - 1)
    alpha[0::2] = d
    alpha[1::2] = f
    lam, Z = _device_mrrr(torch, None, alpha, n, m)
    assert np.max(np.abs(lam - np.sort(sig))) <= 1e-13
    T = np.diag(alpha, 1) + np.diag(alpha, -1)
    assert np.max(np.abs(Z.T @ Z - np.eye(n))) <= 1e-12
    assert np.max(np.linalg.norm(T @ Z - Z * lam, axis=0)) <= 1e-13 * sig.max()


def _bse_beta(n, seed):
    p = make_problem(n, seed)
    W = alg1.step3_W(alg1.step2_cholesky(alg1.step1_M(p.A, p.B)))
    return p, alg1.alg3_step1_tridiagonalize(W).beta


def test_mrrr_peeling_dense_bse_tridiagonal():
    """gaptol = 0.05 makes the positive half of a BSE tridiagonal at n = 100 one
    cluster of more than 1/gaptol members: the device tree peels it as the oracle's
    does, and the eigenvalues (BSE form, positive half) match the oracle's and the
    definition route's."""
    torch = torch_cuda()
    n = 100
    p, beta = _bse_beta(n, 5)
    m = 2 * n
    lam, Z = _device_mrrr(torch, None, beta, n, m, gaptol=0.05, bse_form=1)
    lam_o, _, tree = mrrr.eigh_tridiagonal(np.zeros(m), -beta, 0.05)
    assert max(s for _, s in tree) * 0.05 > 1.0
    T = np.diag(-beta, 1) + np.diag(-beta, -1)
    nrm = np.abs(T).sum(axis=1).max()
    # each level of the tree perturbs its representation by a few eps relative,
    # so a leaf's eigenvalue carries O(levels x eps ||T||); the two trees differ (the
    # device works on the positive half only, the oracle on all of them), so their
    # values agree to that order, and both agree with a library solver to it
    ref = np.linalg.eigvalsh(T)[n:]
    assert np.max(np.abs(lam - lam_o[n:])) <= 32 * EPS * nrm
    assert np.max(np.abs(lam - ref)) <= 32 * EPS * nrm
    assert rel_err(lam, D.solve(p.A, p.B).lam) <= 1e-12
    assert np.max(np.abs(Z.T @ Z - np.eye(n))) <= 1e-12
    assert np.max(np.linalg.norm(T @ Z - Z * lam, axis=0)) <= 2 * m * EPS * nrm


def test_mrrr_bse_form_matches_tdeig_layout():
    """bse_form = 1, the positive half and bse_signs = 1 give bse_stage_tdeig's
    outputs: the same eigenvalues (1e-13) and the same sign-folded vectors up to a
    sign per column."""
    torch = torch_cuda()
    L, bse = _lib()
    n = 150
    _, beta = _bse_beta(n, 7)
    m = 2 * n
    lam, Z = _device_mrrr(torch, None, beta, n, m, bse_form=1, bse_signs=1)
    e = torch.tensor(beta.tolist() + [0.0], dtype=torch.float64, device="cuda")
    lam_t = torch.empty(n, dtype=torch.float64, device="cuda")
    Vs = torch.empty(m * n, dtype=torch.float64, device="cuda")
    work = torch.empty(L.bse_stage_tdeig_worksize(m), dtype=torch.uint8, device="cuda")
    st = torch.zeros(4, dtype=torch.int32, device="cuda")
    bse.check(L.bse_stage_tdeig(m, e.data_ptr(), lam_t.data_ptr(), Vs.data_ptr(), work.data_ptr(), st.data_ptr(),
                                None), "tdeig")
    torch.cuda.synchronize()
    assert rel_err(lam, lam_t.cpu().numpy()) <= 1e-13
    V = Vs.cpu().numpy().reshape(m, n)
    assert np.max(np.abs(np.abs(np.sum(Z * V, axis=0)) - 1.0)) <= 1e-8


@pytest.mark.parametrize("n", [64, 257, 600])
def test_fp64_solve_with_mrrr_vectors(n):
    """bse_set_tdeig_method(1): the FP64 path takes the tree's vectors instead of
    reorthogonalized twisted ones: eigenvalues to 1e-12 and scaled residuals within
    100 n eps as before; the Table 1 metrics follow the tree's orthogonality,
    O(m eps / gaptol) (Dhillon-Parlett), measured at ~1/50 of that bound on these
    spectra and held to 1/20 of it (the reorthogonalized vectors reach 1e-13)."""
    torch_cuda()
    L, bse = _lib()
    p = make_problem(n, 1000 + n)
    ref = D.solve(p.A, p.B)
    assert L.bse_set_tdeig_method(1) == 0
    try:
        with bse.Context(0) as ctx:
            lam, X, _, _, _ = ctx.solve(p.A, p.B, precision="fp64")
            lam2, X2, _, _, _ = ctx.solve(p.A, p.B, precision="mixed_refined")
    finally:
        assert L.bse_set_tdeig_method(0) == 0
    assert rel_err(lam, ref.lam) <= 1e-12
    assert np.max(D.scaled_residuals(p.A, p.B, lam, X)) <= 100 * n * EPS
    met = D.table1_metrics(p.A, p.B, lam, X)
    bar = (2 * n) * EPS / 1e-3 / 20
    assert met["res_F"] <= bar and met["biorth"] <= bar, met
    assert rel_err(lam2, ref.lam) <= 1e-10
    assert np.max(D.scaled_residuals(p.A, p.B, lam2, X2)) <= 100 * n * EPS
