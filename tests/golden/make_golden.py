"""Writes brute_force_eigs.json: 50-digit eigenvalues of H for tiny seeded problems.

Calls only the oracle (oracle.brute, mpmath) on inputs from the seeded generator.
Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import mpmath as mp  # noqa: E402

from oracle import brute  # noqa: E402
from paper_1501_03830_gb300.synth import make_problem  # noqa: E402

CASES = [(2, 11, False), (3, 12, False), (4, 13, False), (3, 14, True)]


def main():
    out = {
        "source": "oracle.brute.eig_H at 50 digits (mpmath general eigensolver on H of Eq. 1)",
        "cases": [],
    }
    for n, seed, real in CASES:
        p = make_problem(n, seed, real=real)
        Es, _ = brute.eig_H(p.A, p.B, dps=50)
        with mp.workdps(50):
            out["cases"].append(
                {
                    "n": n,
                    "seed": seed,
                    "real": real,
                    "eig_re": [mp.nstr(mp.re(e), 30) for e in Es],
                    "eig_im_absmax": mp.nstr(max(abs(mp.im(e)) for e in Es), 5),
                }
            )
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "brute_force_eigs.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
