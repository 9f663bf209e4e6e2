"""The allocation-free tridiagonal eigensolver entry point (bse_stage_tdeig_noalloc)
against the workspace-taking one (bse_stage_tdeig), through the C ABI.

Callers that cannot allocate device memory use the no-alloc variant, whose scratch
is a fixed array inside the library. Two calls in a row (a larger problem, then a
smaller one that lands on the first call's leftover scratch) must both match the
regular entry point. This file is collected last on purpose.
"""
import numpy as np
import pytest

from tests.helpers import torch_cuda

pytestmark = pytest.mark.gpu


def _run(torch, L, bse, fn_name, m, beta, with_work):
    n = m // 2
    e = torch.from_numpy(beta).cuda()
    lam = torch.empty(n, dtype=torch.float64, device="cuda")
    Vs = torch.empty(m * n, dtype=torch.float64, device="cuda")
    st = torch.zeros(4, dtype=torch.int32, device="cuda")
    if with_work:
        work = torch.empty(L.bse_stage_tdeig_worksize(m), dtype=torch.uint8, device="cuda")
        rc = L.bse_stage_tdeig(m, e.data_ptr(), lam.data_ptr(), Vs.data_ptr(), work.data_ptr(), st.data_ptr(), None)
    else:
        rc = L.bse_stage_tdeig_noalloc(m, e.data_ptr(), lam.data_ptr(), Vs.data_ptr(), st.data_ptr(), None)
    bse.check(rc, fn_name)
    torch.cuda.synchronize()
    assert st.cpu().numpy()[0] == 0
    return lam.cpu().numpy(), Vs.cpu().numpy().reshape(m, n)


def test_noalloc_matches_workspace_entry_point_twice():
    torch = torch_cuda()
    from paper_1501_03830_gb300 import bse

    L = bse.lib()
    rng = np.random.default_rng(2024)
    for m in (1024, 300):
        beta = rng.uniform(0.3, 3.0, m - 1) * np.where(rng.random(m - 1) < 0.5, -1.0, 1.0)
        lam_ref, V_ref = _run(torch, L, bse, "bse_stage_tdeig", m, beta, True)
        lam, V = _run(torch, L, bse, "bse_stage_tdeig_noalloc", m, beta, False)
        assert np.max(np.abs(lam - lam_ref)) <= 1e-14 * np.max(np.abs(lam_ref))
        assert np.max(np.abs(V - V_ref)) <= 1e-12


def test_noalloc_rejects_oversize():
    torch_cuda()
    from paper_1501_03830_gb300 import bse

    L = bse.lib()
    rc = L.bse_stage_tdeig_noalloc(65538, 1, 1, None, 1, None)
    assert rc == bse.BSE_ERR_ARG
    assert "65536" in bse.last_error()
