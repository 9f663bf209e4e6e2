"""The request loop (bse_submit / bse_poll): continuous batching of uneven solves.

Requests that arrive while others run are admitted as slots and HBM free up and
their kernels overlap on the device; each request still runs exactly the kernels
of a single solve, so every result must be bit-for-bit the result of solving the
problem alone, and meet the parity bar against the oracle.
"""
import time

import numpy as np
import pytest

from oracle import definition as D
from paper_1501_03830_gb300.synth import make_problem
from tests.helpers import rel_err, torch_cuda

pytestmark = pytest.mark.gpu


def _ctx():
    from paper_1501_03830_gb300 import bse

    return bse, bse.Context(0)


def _wait(ctx, tickets, timeout=300.0):
    done = {}
    t0 = time.time()
    while len(done) < len(tickets) and time.time() - t0 < timeout:
        for t in tickets:
            if t not in done:
                ok, res = ctx.poll(t)
                if ok:
                    done[t] = res
        time.sleep(0.002)
    assert len(done) == len(tickets), "requests did not finish"
    return done


def test_serving_results_same_alone_and_in_the_mix():
    torch_cuda()
    bse, ctx = _ctx()
    sizes = [300, 40, 129, 64, 257, 33, 180, 96, 50, 220]
    precs = ["mixed_refined", "fp64", "mixed_refined", "mixed", "mixed_refined", "fp64", "mixed_refined",
             "mixed_refined", "mixed", "fp64"]
    probs = [make_problem(n, 40 + i) for i, n in enumerate(sizes)]
    # alone: one solve at a time on a plain context
    alone = [ctx.solve(p.A, p.B, precision=pr)[:2] for p, pr in zip(probs, precs)]
    # in the mix: all submitted at once to a loop with 4 slots
    ctx.serve_start(4)
    reqs, outs, tickets = [], [], []
    for p, pr in zip(probs, precs):
        lam = np.empty(p.n)
        X = np.empty((2 * p.n, p.n), dtype=np.complex128, order="F")
        w = np.empty(p.n, dtype=np.complex128)
        r = bse.make_request(p.n, p.A, p.B, lam, X, p.d_r, p.d_l, w, precision=pr)
        reqs.append(r)
        outs.append((lam, X, w))
        tickets.append(ctx.submit(r))
    done = _wait(ctx, tickets)
    assert ctx.serve_stop(60.0) == 0
    for i, (p, pr) in enumerate(zip(probs, precs)):
        res = done[tickets[i]]
        assert res.status == 0 and res.n == p.n
        assert res.t_submit <= res.t_start <= res.t_done
        lam, X, w = outs[i]
        assert np.array_equal(lam, alone[i][0]) and np.array_equal(X, alone[i][1]), (p.n, pr)
        ref = D.solve(p.A, p.B)
        tol = 1e-4 if pr == "mixed" else 1e-10
        assert rel_err(lam, ref.lam) <= tol
        if pr != "mixed":
            wref = D.weights(ref.X, ref.Y, p.d_r, p.d_l)
            assert np.max(np.abs(w - wref)) <= 1e-8 * np.max(np.abs(wref))
    ctx.close()


def test_serving_overlaps_requests_on_the_device():
    """With 4 slots the mix finishes faster than the same requests one at a time."""
    torch_cuda()
    bse, ctx = _ctx()
    probs = [make_problem(n, 900 + n) for n in (160, 170, 180, 190, 200, 210, 220, 230)]

    def run(slots):
        ctx.serve_start(slots)
        reqs, tickets = [], []
        t0 = time.perf_counter()
        for p in probs:
            r = bse.make_request(p.n, p.A, p.B, np.empty(p.n), precision="mixed_refined")
            reqs.append(r)
            tickets.append(ctx.submit(r))
        done = _wait(ctx, tickets)
        dt = time.perf_counter() - t0
        assert ctx.serve_stop(60.0) == 0
        assert all(r.status == 0 for r in done.values())
        return dt

    run(1)  # warm the slot contexts' kernels
    t1 = min(run(1) for _ in range(2))
    t4 = min(run(4) for _ in range(2))
    assert t4 < 0.9 * t1, (t1, t4)
    ctx.close()


def test_serving_errors_and_stop():
    """A bad request fails alone (Eq. cond), unknown tickets are reported, and a
    stop that times out returns BSE_ERR_TIMEOUT after the running requests end."""
    torch_cuda()
    bse, ctx = _ctx()
    ctx.serve_start(2)
    bad = make_problem(64, 5)
    Abad = bad.A.copy()
    Abad[3, 3] = -40.0
    r_bad = bse.make_request(64, Abad, bad.B, np.empty(64))
    good = make_problem(72, 6)
    r_good = bse.make_request(72, good.A, good.B, np.empty(72))
    tb, tg = ctx.submit(r_bad), ctx.submit(r_good)
    done = _wait(ctx, [tb, tg])
    assert done[tb].status == -2 and done[tg].status == 0
    with pytest.raises(bse.BSEError) as ei:
        ctx.poll(tb)  # already collected: forgotten
    assert ei.value.code == -8
    # a stop with a tiny timeout while a large request runs
    big = make_problem(1024, 7)
    r_big = bse.make_request(1024, big.A, big.B, np.empty(1024))
    ctx.submit(r_big)
    time.sleep(0.05)
    assert ctx.serve_stop(0.001) == -6
    ctx.close()
