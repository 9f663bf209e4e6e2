"""Batched solves (many independent problems of uneven size in one call).

Each problem of the batch runs the kernels of a single solve on one of several
streams, so the batched results must be bit-for-bit those of solving the
problems one by one, and every problem must meet the parity bar against the
oracle (refined path: eigenvalues to 1e-10 relative, scaled residual <= 100 n eps).
"""
import numpy as np
import pytest

from oracle import definition as D
from paper_1501_03830_gb300.synth import batch_sizes, make_problem
from tests.helpers import rel_err, torch_cuda

pytestmark = pytest.mark.gpu


def _ctx():
    from paper_1501_03830_gb300 import bse

    return bse, bse.Context(0)


def test_batched_matches_single_and_oracle():
    torch_cuda()
    bse, ctx = _ctx()
    ns = [int(v) for v in batch_sizes(24, 32, 192, seed=3)]
    probs = [make_problem(n, 300 + i) for i, n in enumerate(ns)]
    res, st = ctx.solve_batched([(p.A, p.B) for p in probs], precision="mixed_refined")
    assert np.all(st == 0)
    for i, p in enumerate(probs):
        lam, X = res[i]
        ref = D.solve(p.A, p.B)
        assert rel_err(lam, ref.lam) <= 1e-10, (ns[i], rel_err(lam, ref.lam))
        r = D.scaled_residuals(p.A, p.B, lam, X)
        assert np.max(r) <= 100 * p.n * 2.0 ** -52
        if i % 6 == 0:  # bit-for-bit the single-solve result
            lam1, X1, _, _, _ = ctx.solve(p.A, p.B, precision="mixed_refined")
            assert np.array_equal(lam1, lam) and np.array_equal(X1, X)
    ctx.close()


def test_batched_device_buffers_and_fp64():
    torch = torch_cuda()
    bse, ctx = _ctx()
    ns = [40, 97, 64, 33]
    probs = [make_problem(n, 500 + n) for n in ns]
    dev = []
    outs = []
    for p in probs:
        A = torch.from_numpy(np.ascontiguousarray(np.asfortranarray(p.A).T)).cuda()
        B = torch.from_numpy(np.ascontiguousarray(np.asfortranarray(p.B).T)).cuda()
        dev.append((A, B))
        outs.append((torch.empty(p.n, dtype=torch.float64, device="cuda"),
                     torch.empty(2 * p.n * p.n, dtype=torch.complex128, device="cuda")))
    res, st = ctx.solve_batched(dev, precision="fp64", outs=outs)
    torch.cuda.synchronize()
    assert np.all(st == 0)
    for p, (lam, X) in zip(probs, outs):
        ref = D.solve(p.A, p.B)
        assert rel_err(lam.cpu().numpy(), ref.lam) <= 1e-12
    ctx.close()


def test_batched_reports_per_problem_failure():
    """A problem that violates Eq. cond fails alone; the others are solved."""
    torch_cuda()
    bse, ctx = _ctx()
    good = [make_problem(n, 700 + n) for n in (48, 80)]
    bad = make_problem(64, 9)
    Abad = bad.A.copy()
    Abad[5, 5] = -50.0  # M loses positive definiteness
    problems = [(good[0].A, good[0].B), (Abad, bad.B), (good[1].A, good[1].B)]
    res, st = ctx.solve_batched(problems, precision="mixed_refined")
    assert st[0] == 0 and st[2] == 0 and st[1] == -2
    for g, (lam, _) in zip(good, (res[0], res[2])):
        assert rel_err(lam, D.solve(g.A, g.B).lam) <= 1e-10
    ctx.close()
