"""Failure detection on the device without a GPU fault: a bounded wait that runs out.

The tridiagonal panel kernel's blocks meet at grid barriers whose waits give up
after a fixed number of polls and report BSE_ERR_TIMEOUT instead of hanging. A
test hook lowers that number so the waits of one launch run out on purpose;
nothing faults, traps or spins without bound. The context stays usable: the next
reduction and the next solve on it are correct once the default is restored.
"""
import numpy as np
import pytest

from oracle import definition as D
from paper_1501_03830_gb300.synth import make_problem
from tests.helpers import dev_f, torch_cuda

pytestmark = pytest.mark.gpu


def test_panel_barrier_timeout_is_reported_and_recovers():
    torch = torch_cuda()
    from paper_1501_03830_gb300 import bse

    L = bse.lib()
    m = 1200  # above the one-CTA size limit, so the cooperative panel kernel runs
    rng = np.random.default_rng(5)
    W = np.tril(rng.standard_normal((m, m)), -1)
    W = W - W.T
    work = torch.empty(L.bse_stage_tridiag_worksize(m, 1), dtype=torch.uint8, device="cuda")
    e = torch.empty(m, dtype=torch.float64, device="cuda")
    tau = torch.empty(m, dtype=torch.float32, device="cuda")

    def reduce():
        Wd = dev_f(torch, np.tril(W, -1), "float32")
        st = torch.zeros(4, dtype=torch.int32, device="cuda")
        rc = L.bse_stage_tridiag(m, Wd.data_ptr(), m, e.data_ptr(), tau.data_ptr(), 1, work.data_ptr(),
                                 st.data_ptr(), None)
        torch.cuda.synchronize()
        return rc, int(st[0].item())

    try:
        assert L.bse_debug_barrier_spin(1) == 0
        rc, code = reduce()
        assert rc in (bse.BSE_OK, bse.BSE_ERR_TIMEOUT)
        assert code == bse.BSE_ERR_TIMEOUT
    finally:
        assert L.bse_debug_barrier_spin(0) == 0
    # the same buffers and process: a normal reduction again
    rc, code = reduce()
    assert rc == bse.BSE_OK and code == 0
    # |sub-diagonal| of T: its singular values are those of W (skew: eigenvalues +-i sigma)
    T = np.zeros((m, m))
    b = e.cpu().numpy()[: m - 1]
    T[np.arange(1, m), np.arange(m - 1)] = b
    T = T - T.T
    sv_T = np.sort(np.linalg.svd(T, compute_uv=False))
    sv_W = np.sort(np.linalg.svd(W, compute_uv=False))
    assert np.max(np.abs(sv_T - sv_W)) <= 1e-4 * sv_W[-1]
    # and a whole solve on a fresh context
    p = make_problem(300, 77)
    ref = D.solve(p.A, p.B)
    with bse.Context(0) as ctx:
        lam, X, _, info, _ = ctx.solve(p.A, p.B, precision="mixed_refined")
    assert info.status == 0
    assert np.max(np.abs(lam - ref.lam) / ref.lam) <= 1e-10
