"""Stage-by-stage parity of the CUDA kernels against the oracle's Algorithm 1/3
restatement (oracle.alg1), through the stage C ABI (include/bse_stages.h).

Each stage is fed the GPU's own output of the previous stage, so a mismatch
points at one kernel. Sizes span several tiles and ragged tails.
"""
import ctypes as C

import numpy as np
import pytest

from oracle import alg1
from oracle import definition as D
from paper_1501_03830_gb300.synth import make_problem
from tests.helpers import dev_c128, dev_f, host_colmajor, torch_cuda

pytestmark = pytest.mark.gpu

SIZES = [1, 3, 33, 100]


def _lib():
    from paper_1501_03830_gb300 import bse

    return bse.lib(), bse


def _status(torch):
    return torch.zeros(4, dtype=torch.int32, device="cuda")


@pytest.mark.parametrize("n", SIZES)
def test_form_M(n):
    torch = torch_cuda()
    L, bse = _lib()
    p = make_problem(n, 100 + n)
    m = 2 * n
    A = dev_c128(torch, p.A)
    B = dev_c128(torch, p.B)
    M = torch.empty(m * m, dtype=torch.float64, device="cuda")
    Mf = torch.empty(m * m, dtype=torch.float32, device="cuda")
    bse.check(L.bse_stage_form_M(n, A.data_ptr(), n, B.data_ptr(), n, M.data_ptr(), m, Mf.data_ptr(), m, None), "form_M")
    torch.cuda.synchronize()
    ref = alg1.step1_M(p.A, p.B)
    got = host_colmajor(M, (m, m))
    assert np.array_equal(got, ref)  # same FP64 additions: bit-exact
    gotf = host_colmajor(Mf, (m, m))
    assert np.array_equal(gotf, ref.astype(np.float32))


@pytest.mark.parametrize("n", SIZES + [200])
@pytest.mark.parametrize("fp32", [0, 1])
def test_potrf(n, fp32):
    torch = torch_cuda()
    L, bse = _lib()
    p = make_problem(n, 200 + n)
    m = 2 * n
    Mref = alg1.step1_M(p.A, p.B)
    dt = "float32" if fp32 else "float64"
    Md = dev_f(torch, Mref, dt)
    work = torch.empty(L.bse_stage_potrf_worksize(m, fp32), dtype=torch.uint8, device="cuda")
    st = _status(torch)
    bse.check(L.bse_stage_potrf(m, Md.data_ptr(), m, fp32, work.data_ptr(), st.data_ptr(), None), "potrf")
    torch.cuda.synchronize()
    assert st.cpu().numpy()[0] == 0
    got = np.tril(host_colmajor(Md, (m, m)).astype(np.float64))
    Lref = alg1.step2_cholesky(Mref)
    tol = 2e-5 if fp32 else 1e-13
    assert np.max(np.abs(got - Lref)) <= tol * np.max(np.abs(Lref))


def test_potrf_not_definite():
    """Eq. cond violated: the status word carries BSE_ERR_NOT_DEFINITE and a 1-based column."""
    torch = torch_cuda()
    L, bse = _lib()
    m = 150
    Mref = np.eye(m) * 2.0
    Mref[97, 97] = -1.0
    Md = dev_f(torch, Mref)
    work = torch.empty(L.bse_stage_potrf_worksize(m, 0), dtype=torch.uint8, device="cuda")
    st = _status(torch)
    bse.check(L.bse_stage_potrf(m, Md.data_ptr(), m, 0, work.data_ptr(), st.data_ptr(), None), "potrf")
    torch.cuda.synchronize()
    s = st.cpu().numpy()
    assert s[0] == bse.BSE_ERR_NOT_DEFINITE and s[1] == 98


@pytest.mark.parametrize("n", SIZES + [130])
@pytest.mark.parametrize("fp32", [0, 1])
def test_form_W(n, fp32):
    torch = torch_cuda()
    L, bse = _lib()
    p = make_problem(n, 300 + n)
    m = 2 * n
    Lref = alg1.step2_cholesky(alg1.step1_M(p.A, p.B))
    dt = "float32" if fp32 else "float64"
    # garbage in L's strict upper triangle must be ignored
    Lg = Lref + np.triu(np.full((m, m), 7.0), 1)
    Ld = dev_f(torch, Lg, dt)
    Wd = dev_f(torch, np.full((m, m), np.nan), dt)
    bse.check(L.bse_stage_form_W(n, Ld.data_ptr(), m, Wd.data_ptr(), m, fp32, None), "form_W")
    torch.cuda.synchronize()
    got = np.tril(host_colmajor(Wd, (m, m)).astype(np.float64))
    Lin = Lref.astype(np.float32).astype(np.float64) if fp32 else Lref
    Wref = np.tril(alg1.step3_W(Lin))
    tol = 1e-5 if fp32 else 1e-13
    assert np.max(np.abs(got - Wref)) <= tol * max(1.0, np.max(np.abs(Wref)))
    assert np.all(np.diag(got) == 0.0)
    assert np.all(got[n:, n:] == 0.0)


def _W_input(n, seed):
    p = make_problem(n, seed)
    return alg1.step3_W(alg1.step2_cholesky(alg1.step1_M(p.A, p.B)))


@pytest.mark.parametrize("n", [1, 3, 33, 70, 100, 129, 257])
@pytest.mark.parametrize("fp32", [0, 1])
def test_tridiag(n, fp32):
    """Blocked skew reduction reproduces the unblocked literal H A H reduction (same
    reflector convention, so beta_k match with their signs) and U^T W U = T."""
    torch = torch_cuda()
    L, bse = _lib()
    m = 2 * n
    W = _W_input(n, 400 + n)
    dt = "float32" if fp32 else "float64"
    Wd = dev_f(torch, np.tril(W, -1) + np.triu(np.full((m, m), np.nan)), dt)
    e = torch.empty(m, dtype=torch.float64, device="cuda")
    tau = torch.empty(m, dtype=torch.float32 if fp32 else torch.float64, device="cuda")
    work = torch.empty(L.bse_stage_tridiag_worksize(m, fp32), dtype=torch.uint8, device="cuda")
    st = _status(torch)
    bse.check(L.bse_stage_tridiag(m, Wd.data_ptr(), m, e.data_ptr(), tau.data_ptr(), fp32, work.data_ptr(),
                                  st.data_ptr(), None), "tridiag")
    torch.cuda.synchronize()
    assert st.cpu().numpy()[0] == 0
    ref = alg1.alg3_step1_tridiagonalize(W)
    eg = e.cpu().numpy()[: m - 1]
    scale = np.max(np.abs(W))
    # FP32: beta and tau carry the rounding of ~m FP32 reflector steps
    tol = 1e-3 if fp32 else 1e-11
    assert np.max(np.abs(eg - ref.beta)) <= tol * scale
    taug = tau.cpu().numpy()[: m - 1].astype(np.float64)
    assert np.max(np.abs(taug - ref.taus)) <= (2e-3 if fp32 else 1e-10)
    # reflectors stored in W's strict lower part: rebuild U and check U^T W U = T
    Wg = host_colmajor(Wd, (m, m)).astype(np.float64)
    U = np.eye(m)
    for j in range(m - 1):
        v = np.zeros(m)
        v[j + 1:] = Wg[j + 1:, j]
        assert v[j + 1] == 1.0
        U = U - taug[j] * np.outer(U @ v, v)
    T = np.zeros((m, m))
    idx = np.arange(m - 1)
    T[idx + 1, idx] = eg
    T[idx, idx + 1] = -eg
    assert np.max(np.abs(U.T @ W @ U - T)) <= (1e-4 if fp32 else 1e-12) * scale


@pytest.mark.parametrize("n", [1, 2, 33, 100, 256])
def test_tdeig(n):
    """Bisection + twisted vectors vs a library eigensolver on Tsym (remark 2)."""
    torch = torch_cuda()
    L, bse = _lib()
    m = 2 * n
    rng = np.random.default_rng(n)
    beta = rng.uniform(0.3, 3.0, m - 1) * np.where(rng.random(m - 1) < 0.5, -1.0, 1.0)
    e = torch.from_numpy(beta).cuda()
    lam = torch.empty(n, dtype=torch.float64, device="cuda")
    Vs = torch.empty(m * n, dtype=torch.float64, device="cuda")
    work = torch.empty(L.bse_stage_tdeig_worksize(m), dtype=torch.uint8, device="cuda")
    st = _status(torch)
    bse.check(L.bse_stage_tdeig(m, e.data_ptr(), lam.data_ptr(), Vs.data_ptr(), work.data_ptr(), st.data_ptr(), None),
              "tdeig")
    torch.cuda.synchronize()
    assert st.cpu().numpy()[0] == 0
    Tsym = np.diag(-beta, 1) + np.diag(-beta, -1)
    w, V = np.linalg.eigh(Tsym)
    lg = lam.cpu().numpy()
    # eigh is accurate to eps*||T|| absolutely (not relatively for tiny eigenvalues)
    assert np.max(np.abs(lg - w[n:])) <= 1e-14 * np.max(np.abs(w))
    # bisection itself is relatively accurate: compare with the bidiagonal's singular
    # values from the Golub-Kahan form for the well-separated part of the spectrum
    big = w[n:] > 1e-3 * np.max(w)
    assert np.max(np.abs(lg[big] - w[n:][big]) / w[n:][big]) <= 1e-13
    # Vs is row-major m x n with the D signs folded in
    Vg = Vs.cpu().numpy().reshape(m, n)
    sgn = np.array([1.0, 1.0, -1.0, -1.0])[np.arange(m) % 4]
    Vg = Vg * sgn[:, None]
    ov = np.abs(Vg.T @ V[:, n:])
    assert np.max(np.abs(ov - np.eye(n))) <= 1e-10
    # residual of each computed pair
    r = Tsym @ Vg - Vg * lg[None, :]
    assert np.max(np.linalg.norm(r, axis=0)) <= 1e-13 * np.max(np.abs(w))


@pytest.mark.parametrize("n", [1, 3, 33, 70])
@pytest.mark.parametrize("fp32", [0, 1])
def test_backtransform(n, fp32):
    """Steps 3-6 of Algorithm 3 on the oracle's L, reflectors and V+ vs the oracle."""
    torch = torch_cuda()
    L, bse = _lib()
    m = 2 * n
    p = make_problem(n, 500 + n)
    Lref = alg1.step2_cholesky(alg1.step1_M(p.A, p.B))
    W = alg1.step3_W(Lref)
    tri = alg1.alg3_step1_tridiagonalize(W)
    lam, Vp, _ = alg1.alg3_step2_tridiag_eig(tri.T)
    Xref, Yref, _ = alg1.alg3_backtransform(Lref, tri.U, Vp, lam)
    # reflectors in the storage convention of the stage ABI
    Wst = np.full((m, m), np.nan)
    taus = np.zeros(m)
    for j in range(m - 1):
        Wst[j + 1:, j] = tri.vs[j][j + 1:]
        taus[j] = tri.taus[j]
    dt = "float32" if fp32 else "float64"
    Ld = dev_f(torch, Lref + np.triu(np.full((m, m), 3.0), 1), dt)
    Wd = dev_f(torch, Wst, dt)
    taud = torch.from_numpy(taus.astype(dt)).cuda()
    sgn = np.array([1.0, 1.0, -1.0, -1.0])[np.arange(m) % 4]
    Vs = torch.from_numpy(np.ascontiguousarray(Vp * sgn[:, None])).cuda()
    lamd = torch.from_numpy(lam).cuda()
    X = torch.empty(m * n, dtype=torch.complex128, device="cuda")
    Y = torch.empty(m * n, dtype=torch.complex128, device="cuda")
    work = torch.empty(L.bse_stage_backtransform_worksize(m, fp32), dtype=torch.uint8, device="cuda")
    bse.check(L.bse_stage_backtransform(m, Ld.data_ptr(), m, Wd.data_ptr(), m, taud.data_ptr(), Vs.data_ptr(),
                                        lamd.data_ptr(), X.data_ptr(), Y.data_ptr(), m, fp32, work.data_ptr(), None),
              "backtransform")
    torch.cuda.synchronize()
    Xg = host_colmajor(X, (m, n))
    Yg = host_colmajor(Y, (m, n))
    tol = 1e-4 if fp32 else 1e-12
    scale = np.max(np.abs(Xref))
    assert np.max(np.abs(Xg - Xref)) <= tol * scale
    assert np.max(np.abs(Yg - Yref)) <= tol * scale


@pytest.mark.parametrize("n", [1, 40, 257])
def test_weights(n):
    torch = torch_cuda()
    L, bse = _lib()
    m = 2 * n
    p = make_problem(n, 600 + n)
    s = D.solve(p.A, p.B)
    Xd = dev_c128(torch, s.X)
    dr = torch.from_numpy(p.d_r).cuda()
    dl = torch.from_numpy(p.d_l).cuda()
    w = torch.empty(n, dtype=torch.complex128, device="cuda")
    bse.check(L.bse_stage_weights(n, Xd.data_ptr(), m, dr.data_ptr(), dl.data_ptr(), w.data_ptr(), None), "weights")
    torch.cuda.synchronize()
    ref = D.weights(s.X, s.Y, p.d_r, p.d_l)
    assert np.max(np.abs(w.cpu().numpy() - ref)) <= 1e-12 * np.max(np.abs(ref))


def _bidiagonalize(X):
    """Golub-Kahan Householder bidiagonalization of a square X (test helper):
    returns the diagonal d and superdiagonal f of B = U^T X V."""
    A = np.array(X, dtype=np.float64)
    n = A.shape[0]
    for k in range(n):
        x = A[k:, k]
        v = x.copy()
        v[0] += np.copysign(np.linalg.norm(x), x[0])
        if np.linalg.norm(v) > 0:
            v /= np.linalg.norm(v)
            A[k:, k:] -= 2.0 * np.outer(v, v @ A[k:, k:])
        if k < n - 2:
            x = A[k, k + 1:]
            v = x.copy()
            v[0] += np.copysign(np.linalg.norm(x), x[0])
            if np.linalg.norm(v) > 0:
                v /= np.linalg.norm(v)
                A[k:, k + 1:] -= 2.0 * np.outer(A[k:, k + 1:] @ v, v)
    return np.diag(A).copy(), np.diag(A, 1).copy()


def test_tdeig_clustered_and_reorth():
    """Tight clusters (ten eigenvalues 1e-9 apart, twenty groups): multisection keeps
    every eigenvalue to FP64 accuracy; the twisted vectors of a cluster are far from
    orthogonal (eps ||T|| / gap ~ 1e-6), and the reorthogonalization of remark 2 takes
    them to rounding level without spoiling the residuals. Tsym is the zero-diagonal
    tridiagonal of a bidiagonal with these singular values (Golub-Kahan form)."""
    torch = torch_cuda()
    L, bse = _lib()
    rng = np.random.default_rng(11)
    sig = np.concatenate([1.0 + 0.4 * g + 1e-9 * np.arange(10) for g in range(20)])
    n = sig.shape[0]
    m = 2 * n
    Qa, _ = np.linalg.qr(rng.standard_normal((n, n)))
    Qb, _ = np.linalg.qr(rng.standard_normal((n, n)))
    d, f = _bidiagonalize(Qa @ np.diag(sig) @ Qb.T)
    alpha = np.zeros(m - 1)
    alpha[0::2] = d
    alpha[1::2] = f
    e = torch.tensor((-alpha).tolist() + [0.0], dtype=torch.float64, device="cuda")
    lam = torch.empty(n, dtype=torch.float64, device="cuda")
    Vs = torch.empty(m * n, dtype=torch.float64, device="cuda")
    work = torch.empty(L.bse_stage_tdeig_worksize(m), dtype=torch.uint8, device="cuda")
    st = _status(torch)
    bse.check(L.bse_stage_tdeig(m, e.data_ptr(), lam.data_ptr(), Vs.data_ptr(), work.data_ptr(), st.data_ptr(), None),
              "tdeig")
    torch.cuda.synchronize()
    assert st.cpu().numpy()[0] == 0
    assert np.max(np.abs(np.sort(lam.cpu().numpy()) - np.sort(sig))) <= 1e-13
    signs = np.array([1.0 if (k & 2) == 0 else -1.0 for k in range(m)])[:, None]
    Tsym = np.diag(alpha, 1) + np.diag(alpha, -1)

    def vectors():
        return Vs.cpu().numpy().reshape(m, n) * signs

    V0 = vectors()
    before = np.max(np.abs(V0.T @ V0 - np.eye(n)))
    rw = torch.empty(L.bse_stage_tdeig_reorth_worksize(m), dtype=torch.uint8, device="cuda")
    bse.check(L.bse_stage_tdeig_reorth(m, Vs.data_ptr(), rw.data_ptr(), None), "reorth")
    torch.cuda.synchronize()
    V = vectors()
    lg = lam.cpu().numpy()
    assert before >= 1e-9  # the clusters do need it
    assert np.max(np.abs(V.T @ V - np.eye(n))) <= 1e-13
    assert np.max(np.linalg.norm(Tsym @ V - V * lg[None, :], axis=0)) <= 1e-13 * sig.max()
