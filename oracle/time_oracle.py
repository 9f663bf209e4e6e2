"""Times the oracle's full solve once on this machine's host cores and caches it.

Test and benchmark infrastructure only. A full oracle solve at the benchmark size
(n = 8192: a Cholesky of the 16384 x 16384 complex Omega and a dense Hermitian
eigendecomposition) takes about a quarter of an hour on 16 cores, too long for
every benchmark run. This script measures it once per (n, seed), together with
a small-size solve timed in the same run, and records both in cpu_timings.json
beside this file (with the date, the core count and the CPU). The benchmark
reports the cached full-size time as measured, and times the small solve live.

    python -m oracle.time_oracle --n 8192 --seed 8192 --sample-n 1280
"""
from __future__ import annotations

import argparse
import datetime
import json
import os
import platform
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CACHE = os.path.join(HERE, "cpu_timings.json")


def cpu_model() -> str:
    try:
        import subprocess

        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                low = line.lower()
                if low.startswith("model name") or low.startswith("cpu part"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or "unknown"


def load(path: str = CACHE) -> list[dict]:
    if not os.path.exists(path):
        return []
    with open(path) as f:
        return json.load(f).get("entries", [])


def lookup(n: int, seed: int, cores: int, machine: str):
    """The cached entry for this problem measured on a host like this one, or None."""
    for e in load():
        if e["n"] == n and e["seed"] == seed and e["cores"] == cores and e["machine"] == machine:
            return e
    return None


def time_solve(n: int, seed: int) -> float:
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    from oracle import definition as D
    from paper_1501_03830_gb300.synth import make_problem

    p = make_problem(n, seed)
    t = time.perf_counter()
    D.solve(p.A, p.B)
    return time.perf_counter() - t


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--n", type=int, default=8192)
    ap.add_argument("--seed", type=int, default=8192)
    ap.add_argument("--sample-n", type=int, default=1280)
    ap.add_argument("--out", default=CACHE, help="cache file to update (default: cpu_timings.json here)")
    a = ap.parse_args(argv)
    t_small = time_solve(a.sample_n, a.seed)
    t_full = time_solve(a.n, a.seed)
    entry = {
        "n": a.n, "seed": a.seed, "seconds": t_full,
        "sample_n": a.sample_n, "sample_seconds": t_small,
        "cores": os.cpu_count(), "machine": platform.machine(), "cpu": cpu_model(),
        "date": datetime.datetime.now(datetime.timezone.utc).strftime("%Y-%m-%dT%H:%M:%SZ"),
        "what": "oracle.definition.solve (Cholesky of Omega, C = L^-1 S L^-H, numpy eigh), FP64, "
                "all host cores through the BLAS",
    }
    entries = [e for e in load(a.out) if not (e["n"] == a.n and e["seed"] == a.seed and e["cores"] == entry["cores"]
                                         and e["machine"] == entry["machine"])]
    entries.append(entry)
    with open(a.out, "w") as f:
        json.dump({"entries": entries}, f, indent=1)
        f.write("\n")
    print(json.dumps(entry))
    return 0


if __name__ == "__main__":
    sys.exit(main())
