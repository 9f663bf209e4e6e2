"""Two-stage (band) reduction on the GPU (bse_stage_sbr, Section 3.3's closing
remark), against the oracle:

* |T[k+1, k]| equals the one-stage reduction's (oracle.alg1, Algorithm 3 step 1):
  both are orthogonal similarities with Q e_1 = e_1, so by the implicit-Q theorem
  the sub-diagonal magnitudes of the (unreduced) tridiagonal are the same;
* the reflectors reconstruct W: with Q1 rebuilt on the host from the stored
  stage-1 vectors and Q2 from bse_stage_sbr_apply_q2 on the identity,
  (Q1 Q2) T (Q1 Q2)^T = W to FP32 level, and Q1 Q2 is orthogonal;
* whole solves through bse_solve with the two-stage path forced at small orders
  match the oracle (mixed: FP32 level; mixed + refinement: 1e-10) and the
  one-stage path.
Orders span one to several 64-wide panels with ragged tails.
"""
import numpy as np
import pytest

from oracle import alg1
from oracle import definition as D
from paper_1501_03830_gb300.synth import make_problem
from tests.helpers import dev_f, host_colmajor, torch_cuda

pytestmark = pytest.mark.gpu

B = 64


def _lib():
    from paper_1501_03830_gb300 import bse

    return bse.lib(), bse


def _W_input(n, seed):
    p = make_problem(n, seed)
    return alg1.step3_W(alg1.step2_cholesky(alg1.step1_M(p.A, p.B)))


def _ld32(m):
    return (m + 31) // 32 * 32


def _run_sbr(torch, L, bse, W):
    m = W.shape[0]
    ld = _ld32(m)
    Wp = np.full((ld, m), np.nan)
    Wp[:m, :] = np.tril(W, -1)
    Wp[:m, :][np.triu_indices(m)] = np.nan  # the upper triangle is not read
    Wd = dev_f(torch, Wp, "float32")
    e = torch.empty(m, dtype=torch.float64, device="cuda")
    tau = torch.empty(m, dtype=torch.float32, device="cuda")
    work = torch.empty(L.bse_stage_sbr_worksize(m), dtype=torch.uint8, device="cuda")
    st = torch.zeros(4, dtype=torch.int32, device="cuda")
    bse.check(L.bse_stage_sbr(m, Wd.data_ptr(), ld, e.data_ptr(), tau.data_ptr(), work.data_ptr(), st.data_ptr(),
                              None), "sbr")
    torch.cuda.synchronize()
    assert int(st[0].item()) == 0
    return Wd, e.cpu().numpy(), tau.cpu().numpy().astype(np.float64), work, ld


@pytest.mark.parametrize("n", [2, 33, 65, 100, 150, 257])
def test_sbr_subdiagonal_matches_one_stage(n):
    torch = torch_cuda()
    L, bse = _lib()
    W = _W_input(n, 700 + n)
    m = 2 * n
    _, e, _, _, _ = _run_sbr(torch, L, bse, W)
    ref = alg1.alg3_step1_tridiagonalize(W)
    scale = np.max(np.abs(W))
    assert np.max(np.abs(np.abs(e[: m - 1]) - np.abs(ref.beta))) <= 1e-3 * scale
    # the eigenvalues +-i sigma of T equal those of W (FP32 level)
    T = np.zeros((m, m))
    T[np.arange(1, m), np.arange(m - 1)] = e[: m - 1]
    T = T - T.T
    sw = np.sort(np.linalg.svd(W, compute_uv=False))
    st = np.sort(np.linalg.svd(T, compute_uv=False))
    assert np.max(np.abs(sw - st)) <= 2e-5 * sw[-1]


@pytest.mark.parametrize("m", [130, 200, 300])
def test_sbr_reflectors_reconstruct_W(m):
    """W = (Q1 Q2) T (Q1 Q2)^T with Q1 from the stage-1 reflectors (unit entry at
    row k + 64 of column k, scalar tau[k]) and Q2 = apply_q2(I)."""
    torch = torch_cuda()
    L, bse = _lib()
    rng = np.random.default_rng(m)
    X = rng.standard_normal((m, m))
    W = X - X.T
    Wd, e, tau, work, ld = _run_sbr(torch, L, bse, W)
    Wg = host_colmajor(Wd, (ld, m)).astype(np.float64)[:m]
    Q1 = np.eye(m)
    for k in range(m):
        if k + B >= m or tau[k] == 0.0:
            continue
        v = np.zeros(m)
        v[k + B:] = Wg[k + B:, k]
        assert v[k + B] == 1.0
        Q1 = Q1 - tau[k] * np.outer(Q1 @ v, v)
    Phi = dev_f(torch, np.eye(m), "float32")
    bse.check(L.bse_stage_sbr_apply_q2(m, Phi.data_ptr(), m, work.data_ptr(), None), "q2")
    torch.cuda.synchronize()
    Q2 = host_colmajor(Phi, (m, m)).astype(np.float64)
    Q = Q1 @ Q2
    T = np.zeros((m, m))
    T[np.arange(1, m), np.arange(m - 1)] = e[: m - 1]
    T = T - T.T
    scale = np.max(np.abs(W))
    assert np.max(np.abs(Q.T @ Q - np.eye(m))) <= 2e-5
    assert np.max(np.abs(Q[:, 0] - np.eye(m)[:, 0])) <= 1e-6  # Q e_1 = e_1
    assert np.max(np.abs(Q @ T @ Q.T - W)) <= 5e-5 * scale


@pytest.mark.parametrize("n", [40, 97, 150, 300])
def test_solve_with_band_reduction(n):
    """bse_solve with the two-stage reduction forced: the eigenvalues of the mixed path
    at FP32 level and of the refined path within 1e-10 of the oracle, residuals at the
    bar, Theorem 3's normalization, and the same refined eigenvalues as the one-stage
    path."""
    torch_cuda()
    L, bse = _lib()
    p = make_problem(n, 900 + n)
    ref = D.solve(p.A, p.B)
    eps = 2.0 ** -52
    try:
        assert L.bse_set_band_reduction(4) == 0
        with bse.Context(0) as ctx:
            lam_m, _, _, info_m, _ = ctx.solve(p.A, p.B, precision="mixed")
            lam, X, _, info, _ = ctx.solve(p.A, p.B, precision="mixed_refined")
    finally:
        L.bse_set_band_reduction(0)
    assert info_m.status == 0 and info.status == 0
    assert np.max(np.abs(lam_m - ref.lam) / ref.lam) <= 1e-4
    assert np.max(np.abs(lam - ref.lam) / ref.lam) <= 1e-10
    assert np.max(D.scaled_residuals(p.A, p.B, lam, X)) <= 100 * n * eps
    s = np.concatenate([np.ones(n), -np.ones(n)])[:, None]
    assert np.max(np.abs(np.einsum("ij,ij->j", (s * X).conj(), X) - 1.0)) <= 1e-12
    with bse.Context(0) as ctx:
        lam1, _, _, _, _ = ctx.solve(p.A, p.B, precision="mixed_refined")
    assert np.max(np.abs(lam - lam1) / lam1) <= 1e-12
