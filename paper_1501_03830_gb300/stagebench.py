"""Time one kernel family of the solver in isolation, on synthetic device data.

    python -m paper_1501_03830_gb300.stagebench tc32 --M 4096 --N 4096 --K 4096
    python -m paper_1501_03830_gb300.stagebench ozaki --M 4096 --N 4096 --K 16384 --s 8
    python -m paper_1501_03830_gb300.stagebench tridiag --m 8192 [--fp64]
    python -m paper_1501_03830_gb300.stagebench tdeig --m 16384 [--mrrr]
    python -m paper_1501_03830_gb300.stagebench sbr --m 16384
    python -m paper_1501_03830_gb300.stagebench solve --n 8192 [--precision mixed_refined]

Each run does --reps launches (CUDA events on the launch stream, after one
warm-up launch) and prints one line with the mean time and the achieved rate
charged with the algorithmic flops or bytes of the stage. It is the command the
kernel profiles are taken with (ncu -k <kernel> on the same command line).
"""
from __future__ import annotations

import argparse
import json

from . import bse


def _timed(torch, fn, reps):
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def run(argv=None) -> dict:
    import torch

    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("stage", choices=["tc32", "ozaki", "tridiag", "tdeig", "sbr", "solve"])
    ap.add_argument("--n", type=int, default=8192, help="solve: problem size (seeded synthetic problem)")
    ap.add_argument("--precision", default="mixed_refined", choices=["fp64", "mixed", "mixed_refined"])
    ap.add_argument("--M", type=int, default=4096)
    ap.add_argument("--N", type=int, default=4096)
    ap.add_argument("--K", type=int, default=4096)
    ap.add_argument("--s", type=int, default=8, help="digits per operand (ozaki)")
    ap.add_argument("--split", type=int, default=1, help="tc32: 1 = 3xTF32, 0 = one TF32 pass")
    ap.add_argument("--ta", type=int, default=0, help="tc32: op(A) = A^T")
    ap.add_argument("--tb", type=int, default=0, help="tc32: op(B) = B^T")
    ap.add_argument("--fp32-gemm", type=int, default=None,
                    help="engine of the FP32 products (bse_set_fp32_gemm: 0 SIMT, 1 in-kernel split, 2 pre-split)")
    ap.add_argument("--m", type=int, default=8192, help="matrix order (tridiag, tdeig)")
    ap.add_argument("--fp64", action="store_true", help="tridiag in FP64 instead of FP32")
    ap.add_argument("--mrrr", action="store_true", help="tdeig by the representation tree (bse_stage_tdeig_mrrr)")
    ap.add_argument("--gaptol", type=float, default=1e-3, help="tdeig --mrrr: relative gap of a singleton")
    ap.add_argument("--reps", type=int, default=3)
    a = ap.parse_args(argv)
    L = bse.lib()
    if a.fp32_gemm is not None:
        bse.check(L.bse_set_fp32_gemm(a.fp32_gemm), "bse_set_fp32_gemm")
    g = torch.Generator(device="cuda")
    g.manual_seed(1)
    st = torch.zeros(4, dtype=torch.int32, device="cuda")
    out = {"stage": a.stage}
    if a.stage == "tc32":
        # column-major operands: op(A) = A (M x K, ld M) or A^T (A: K x M, ld K); likewise B
        ar, ac = (a.K, a.M) if a.ta else (a.M, a.K)
        br, bc = (a.N, a.K) if a.tb else (a.K, a.N)
        A = torch.randn(ac, ar, generator=g, device="cuda")
        B = torch.randn(bc, br, generator=g, device="cuda")
        C = torch.zeros(a.N, a.M, device="cuda")
        fn = lambda: bse.check(L.bse_tc32_gemm(a.M, a.N, a.K, 1.0, A.data_ptr(), ar, a.ta, B.data_ptr(), br, a.tb,
                                                 0.0, C.data_ptr(), a.M, 0, a.split, st.data_ptr(), None), "tc32")
        ms = _timed(torch, fn, a.reps)
        out.update(M=a.M, N=a.N, K=a.K, ta=a.ta, tb=a.tb, split=a.split, ms=ms,
                   tflops=2.0 * a.M * a.N * a.K / ms / 1e9)
    elif a.stage == "ozaki":
        A = torch.randn(a.M, a.K, dtype=torch.float64, device="cuda", generator=g)
        B = torch.randn(a.N, a.K, dtype=torch.float64, device="cuda", generator=g)
        C = torch.zeros(a.N, a.M, dtype=torch.float64, device="cuda")
        work = torch.empty(L.bse_ozaki_worksize(a.M, a.N, a.K, a.s), dtype=torch.uint8, device="cuda")
        fn = lambda: bse.check(L.bse_ozaki_gemm(a.M, a.N, a.K, A.data_ptr(), a.K, B.data_ptr(), a.K, C.data_ptr(), a.M,
                                                a.s, work.data_ptr(), st.data_ptr(), None), "ozaki")
        ms = _timed(torch, fn, a.reps)
        units = a.s * (a.s + 1) // 2
        out.update(M=a.M, N=a.N, K=a.K, s=a.s, units=units, ms=ms,
                   fp64_tflops=2.0 * a.M * a.N * a.K / ms / 1e9,
                   bf16_tflops=2.0 * a.M * a.N * a.K * units / ms / 1e9)
    elif a.stage == "tridiag":
        fp32 = 0 if a.fp64 else 1
        dt = torch.float32 if fp32 else torch.float64
        m = a.m
        W0 = torch.tril(torch.randn(m, m, dtype=dt, device="cuda", generator=g), -1)
        Wm = torch.empty_like(W0)
        e = torch.empty(m, dtype=torch.float64, device="cuda")
        tau = torch.empty(m, dtype=dt, device="cuda")
        work = torch.empty(L.bse_stage_tridiag_worksize(m, fp32), dtype=torch.uint8, device="cuda")

        def fn():
            Wm.copy_(W0)
            bse.check(L.bse_stage_tridiag(m, Wm.data_ptr(), m, e.data_ptr(), tau.data_ptr(), fp32, work.data_ptr(),
                                          st.data_ptr(), None), "tridiag")

        ms = _timed(torch, fn, a.reps)
        esz = 4 if fp32 else 8
        out.update(m=m, fp32=fp32, ms=ms, symv_bytes=esz * m ** 3 / 6.0)
    elif a.stage == "solve":
        # one whole solve (device-resident inputs and outputs), the bench's workload
        import numpy as np

        from .synth import make_problem

        p = make_problem(a.n, a.n)
        m = 2 * a.n
        A = torch.from_numpy(np.ascontiguousarray(np.asfortranarray(p.A).T)).cuda()
        B = torch.from_numpy(np.ascontiguousarray(np.asfortranarray(p.B).T)).cuda()
        lam = torch.empty(a.n, dtype=torch.float64, device="cuda")
        X = torch.empty(m * a.n, dtype=torch.complex128, device="cuda")
        ctx = bse.Context(0)
        fn = lambda: ctx.solve(A, B, precision=a.precision, out={"lambda": lam, "X": X})
        ms = _timed(torch, fn, a.reps)
        out.update(n=a.n, precision=a.precision, ms=ms)
        ctx.close()
    elif a.stage == "sbr":
        # two-stage reduction of a random skew FP32 W (both stages), then Phi <- Phi Q2
        m = a.m
        ld = (m + 31) // 32 * 32
        # column j of W is row j of the (m, ld) tensor: its entries below the diagonal are i > j
        W0 = torch.triu(torch.randn(m, ld, device="cuda", generator=g), 1)
        Wm = torch.empty_like(W0)
        e = torch.empty(m, dtype=torch.float64, device="cuda")
        tau = torch.empty(m, device="cuda")
        work = torch.empty(L.bse_stage_sbr_worksize(m), dtype=torch.uint8, device="cuda")
        Phi = torch.randn(m, ld, device="cuda", generator=g)

        def fn():
            Wm.copy_(W0)
            bse.check(L.bse_stage_sbr(m, Wm.data_ptr(), ld, e.data_ptr(), tau.data_ptr(), work.data_ptr(),
                                      st.data_ptr(), None), "sbr")

        ms = _timed(torch, fn, a.reps)
        fq = lambda: bse.check(L.bse_stage_sbr_apply_q2(m, Phi.data_ptr(), ld, work.data_ptr(), None), "q2")
        ms_q2 = _timed(torch, fq, a.reps)
        bse.kprof_enable(True)
        fn()
        fq()
        torch.cuda.synchronize()
        kp = bse.kprof_read()
        bse.kprof_enable(False)
        out.update(m=m, ms_reduce=ms, ms_q2=ms_q2,
                   kernels={k: (v["launches"], round(v["ms"], 2)) for k, v in kp.items() if v["launches"]})
    else:
        m = a.m
        e = torch.rand(m, dtype=torch.float64, device="cuda", generator=g) + 0.5
        lam = torch.empty(m // 2, dtype=torch.float64, device="cuda")
        Vs = torch.empty(m * (m // 2), dtype=torch.float64, device="cuda")
        if a.mrrr:
            n = m // 2
            work = torch.empty(L.bse_stage_tdeig_mrrr_worksize(m, n, m), dtype=torch.uint8, device="cuda")
            fn = lambda: bse.check(L.bse_stage_tdeig_mrrr(m, None, e.data_ptr(), 1, n, m, a.gaptol, lam.data_ptr(),
                                                          Vs.data_ptr(), n, 1, work.data_ptr(), st.data_ptr(), None),
                                   "tdeig_mrrr")
        else:
            work = torch.empty(L.bse_stage_tdeig_worksize(m), dtype=torch.uint8, device="cuda")
            fn = lambda: bse.check(L.bse_stage_tdeig(m, e.data_ptr(), lam.data_ptr(), Vs.data_ptr(), work.data_ptr(),
                                                     st.data_ptr(), None), "tdeig")
        ms = _timed(torch, fn, a.reps)
        out.update(m=m, ms=ms, method="mrrr" if a.mrrr else "twisted")
    torch.cuda.synchronize()
    out["status"] = int(st[0].item())
    if out["status"] != 0:
        raise bse.BSEError(out["status"], a.stage, "device status")
    return out


def main(argv=None) -> None:
    print(json.dumps(run(argv)))


if __name__ == "__main__":
    main()
