#!/usr/bin/env python
"""Benchmark of the GB300 BSE solver: solves/s at n = 8192 (M is 16384 x 16384).

One step = one whole pass of the hot path on one problem resident in HBM:
form M, Cholesky, W, skew tridiagonal reduction, tridiagonal eigensolve,
back-transform, FP64 refinement (mixed path) and the absorption weights.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun: every rank solves its own independent problem
(replicas only: one solve does not shard), value = all ranks' solves / max time.
Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "BSE solves/s (FP64 vs mixed+refined, 1e-10 rel) at n=8192; serving p50/p99"
UNIT = "solves/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=8192)
    ap.add_argument("--precision", default="mixed_refined", choices=["fp64", "mixed", "mixed_refined"])
    ap.add_argument("--fp64-steps", type=int, default=1, help="timed solves of the plain FP64 path (0: skip)")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--cpu-n", type=int, default=1280, help="oracle sample size for cpu_baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--seed", type=int, default=8192)
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# --- clocks sampled during the timed region ----------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
                power.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        out_dir = os.path.join(ROOT, "gpurun_out")
        if os.path.isdir(out_dir):
            with open(os.path.join(out_dir, "bench_clocks.csv"), "w") as f:
                f.write(self.FIELDS + "\n" + "\n".join(self.lines) + "\n")
        return {
            "sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(smax) if smax else None,
            "power_w_max": max(power) if power else None,
            "samples": len(sm),
            "reasons": sorted(reasons),
        }


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        d["_source"] = "measured"
        return d
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "_source": "fallback"}


# --- CPU oracle baseline ------------------------------------------------------------

def cpu_baseline(n_target: int, n_sample: int, seed: int) -> dict:
    from oracle import definition as D
    from paper_1501_03830_gb300.synth import make_problem

    p = make_problem(n_sample, seed)
    t = time.perf_counter()
    D.solve(p.A, p.B)
    dt = time.perf_counter() - t
    scale = (n_target / n_sample) ** 3
    return {
        "value": 1.0 / (dt * scale),
        "unit": UNIT,
        "cores": os.cpu_count(),
        "kind": "oracle",
        "sample": f"one oracle solve (Cholesky of Omega + dense Hermitian eig, numpy FP64) at n={n_sample} "
                  f"took {dt:.2f} s; scaled by (n/{n_sample})^3 = {scale:.1f} to n={n_target}",
    }


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    steps = []
    for _ in range(args.warmup):
        cpu_baseline(args.n, args.cpu_n, args.seed)
    for _ in range(args.steps):
        steps.append(cpu_baseline(args.n, args.cpu_n, args.seed))
    value = statistics.median(s["value"] for s in steps)
    out = {
        "impl": "reference",
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": args.gpus,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1000.0 / value,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": workload_config(args),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                         "sample": steps[-1]["sample"]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))
    return 0


def workload_config(args) -> dict:
    n = args.n
    return {
        "workload": f"structure-preserving BSE solve + absorption weights, n={n} (H {2*n}x{2*n} complex, "
                    f"M {2*n}x{2*n} real), {args.precision}",
        "n": n,
        "precision": args.precision,
        "generator": "A = diag(U[1,10]) + 0.02/sqrt(n) Hermitian Gaussian, B = 0.02/sqrt(n) complex symmetric "
                     "Gaussian, seeded",
        "l2": f"inputs larger than L2 (A, B {16*n*n/1e9:.2f} GB each; M {8*4*n*n/1e9:.1f} GB)",
    }


# --- our GPU path -----------------------------------------------------------------

def to_dev_colmajor(torch, a, device):
    import numpy as np

    a = np.asfortranarray(a, dtype=np.complex128)
    return torch.from_numpy(np.ascontiguousarray(a.T)).to(device)


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1501_03830_gb300 import bse
    from paper_1501_03830_gb300.synth import make_problem

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl", init_method="env://")
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    n = args.n
    m = 2 * n

    # CPU baseline first (rank 0, N=1 only), before any heavy GPU work
    cpu = None
    if not args.no_cpu_baseline and ws == 1 and rank == 0:
        cpu = cpu_baseline(n, args.cpu_n, args.seed)

    p = make_problem(n, args.seed + rank)
    A = to_dev_colmajor(torch, p.A, device)
    B = to_dev_colmajor(torch, p.B, device)
    dr = torch.from_numpy(p.d_r).to(device)
    dl = torch.from_numpy(p.d_l).to(device)
    lam = torch.empty(n, dtype=torch.float64, device=device)
    X = torch.empty(m * n, dtype=torch.complex128, device=device)
    w = torch.empty(n, dtype=torch.complex128, device=device)

    ctx = bse.Context(local)
    stream = torch.cuda.Stream(device)
    ctx.set_stream(stream.cuda_stream)
    L = bse.lib()

    def step(prec):
        _, _, _, info, _ = ctx.solve(A, B, precision=prec, out={"lambda": lam, "X": X})
        bse.check(L.bse_stage_weights(n, X.data_ptr(), m, dr.data_ptr(), dl.data_ptr(), w.data_ptr(),
                                      stream.cuda_stream), "weights")
        return info

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize(device)

    for _ in range(args.warmup):
        step(args.precision)
    barrier()
    sampler = ClockSampler(local)
    sampler.start()
    launches0 = bse.launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    infos = [step(args.precision) for _ in range(args.steps)]
    ev1.record(stream)
    barrier()
    launches = bse.launch_count() - launches0
    clocks = sampler.stop()
    t_ms = ev0.elapsed_time(ev1)
    t_max = torch.tensor([t_ms], dtype=torch.float64, device=device)
    if ws > 1:
        dist.all_reduce(t_max, op=dist.ReduceOp.MAX)
    t_ms = float(t_max.item())
    value = ws * args.steps / (t_ms * 1e-3)
    last = infos[-1]

    # instrumented run: per-kernel-class device time (CUDA events on the launch stream)
    bse.kprof_enable(True)
    step(args.precision)
    torch.cuda.synchronize(device)
    kp = bse.kprof_read()
    bse.kprof_enable(False)
    peaks = measured_peaks()
    roof = roofline(kp, peaks, torch, device)

    # plain FP64 path on the same problem
    fp64 = None
    if args.fp64_steps > 0 and args.precision != "fp64":
        q = make_problem(256, 1)
        ctx.solve(q.A, q.B, precision="fp64")  # loads the FP64 kernels
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.fp64_steps):
            step("fp64")
        e1.record(stream)
        barrier()
        ms64 = e0.elapsed_time(e1) / args.fp64_steps
        fp64 = {"solves_per_s": 1000.0 / ms64, "ms_per_solve": ms64, "steps": args.fp64_steps,
                "mixed_refined_speedup": (1000.0 / ms64 and value / ws / (1000.0 / ms64))}

    # end to end through the public API with host buffers (pinned), copies inside the timed region
    e2e = None
    if args.e2e_steps > 0:
        Ah = torch.from_numpy(np.ascontiguousarray(np.asfortranarray(p.A).T)).pin_memory()
        Bh = torch.from_numpy(np.ascontiguousarray(np.asfortranarray(p.B).T)).pin_memory()
        drh = torch.from_numpy(p.d_r).pin_memory()
        dlh = torch.from_numpy(p.d_l).pin_memory()
        lamh = torch.empty(n, dtype=torch.float64).pin_memory()
        Xh = torch.empty(m * n, dtype=torch.complex128).pin_memory()
        wh = torch.empty(n, dtype=torch.complex128).pin_memory()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            _, _, _, _, sol = ctx.solve(Ah, Bh, precision=args.precision, out={"lambda": lamh, "X": Xh}, keep=True)
            ctx.spectrum(sol, drh, dlh, out=wh)
            sol.free()
        barrier()
        te = (time.perf_counter() - t0) / args.e2e_steps
        e2e = {"value": ws / te, "unit": UNIT, "h2d_bytes_per_step": 2 * 16 * n * n + 2 * 16 * m,
               "d2h_bytes_per_step": 8 * n + 16 * m * n + 16 * n,
               "how": "bse_solve with pinned host A, B -> host lambda, X; bse_spectrum with host dipoles -> host w"}

    if rank == 0:
        out = {
            "metric": METRIC,
            "value": value,
            "unit": UNIT,
            "n_gpus": ws,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": t_ms / args.steps,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f32+f64",
            "data": "synthetic",
            "config": workload_config(args),
            "accuracy": {
                "refined_scaled_residual_max": last.refine_resid,
                "refined_last_sweep_dlam": last.refine_dlam,
                "unrefined_fp32_rel_eig_err_est": last.unrefined_dlam,
                "sweeps": last.sweeps,
            },
            "fp64_path": fp64,
            "roofline": roof,
            "kernels": {k: v for k, v in kp.items() if v["launches"]},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": clocks,
        }
        print(json.dumps(out))
    ctx.close()
    if ws > 1:
        dist.destroy_process_group()
    return 0


def roofline(kp: dict, peaks: dict, torch, device) -> dict:
    """Roofline entry for the kernel class with the most device time."""
    top = max(kp.items(), key=lambda kv: kv[1]["ms"])
    name, st = top
    if st["ms"] <= 0:
        return None
    sec = st["ms"] * 1e-3
    if name in ("trd_symv", "weights", "form_M", "elementwise", "tdeig_vec"):
        achieved = st["bytes"] / sec / 1e9
        peak = float(peaks.get("hbm_gbs"))
        return {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": None, "launches": st["launches"],
                "avg_launch_ms": st["ms"] / max(1, st["launches"]),
                "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peaks['_source']})"}
    if name == "gemm_tc":
        achieved = st["flops"] / sec / 1e12
        peak = float(peaks.get("bf16_tflops"))
        return {"kernel": name, "bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None, "launches": st["launches"],
                "avg_launch_ms": st["ms"] / max(1, st["launches"]),
                "peak_source": f"MEASURED_PEAKS.json bf16_tflops ({peaks['_source']})"}
    if name == "gemm_tf32":
        # 3xTF32: three TF32 tensor passes per FP32 product; TF32 peak = measured bf16 x 1.1/2.25 (nominal ratio)
        achieved = st["flops"] / sec / 1e12
        peak = float(peaks.get("bf16_tflops")) * (1.1 / 2.25) / 3.0
        return {"kernel": name, "bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None, "launches": st["launches"],
                "avg_launch_ms": st["ms"] / max(1, st["launches"]),
                "peak_source": f"MEASURED_PEAKS.json bf16_tflops ({peaks['_source']}) x 1.1/2.25 (TF32) / 3 "
                               "(3xTF32 passes per FP32 flop)"}
    # SIMT GEMMs: bound by the FP64 or FP32 ALUs; the peak is cuBLAS of the same dtype measured here
    dt = torch.float64 if name == "gemm_f64" else torch.float32
    achieved = st["flops"] / sec / 1e12
    peak = cublas_peak(torch, dt, device)
    return {"kernel": name, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": None, "launches": st["launches"],
            "avg_launch_ms": st["ms"] / max(1, st["launches"]),
            "peak_source": f"cuBLAS {'DGEMM' if dt == torch.float64 else 'SGEMM (no TF32)'} 8192^3 measured in "
                           "this run"}


def cublas_peak(torch, dtype, device, N=8192, it=3) -> float:
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    a = torch.randn(N, N, dtype=dtype, device=device)
    b = torch.randn(N, N, dtype=dtype, device=device)
    a @ b
    torch.cuda.synchronize(device)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(it):
        a @ b
    e1.record()
    torch.cuda.synchronize(device)
    torch.backends.cuda.matmul.allow_tf32 = prev
    return 2.0 * N ** 3 * it / (e0.elapsed_time(e1) * 1e-3) / 1e12


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
