"""Seeded synthetic Bethe--Salpeter inputs ("exciton-shaped" matrices).

This module only draws random numbers; it contains none of the solver's
arithmetic, so both the CUDA path and the CPU oracle can be fed from it.

Shape of the inputs (Section 1, Eq. 1-2 and the definiteness condition Eq. cond):

* A = diag(e) + c * (G + G^H) / 2     Hermitian, diagonally heavy
* B = s * (F + F^T) / 2               complex symmetric, weak
* d_r = d_l = complex Gaussian vector of length 2n (dipole vectors of Eq. absp)

with G, F complex Gaussian (unit variance, (N(0,1) + i N(0,1)) / sqrt 2).

Two size regimes:

* n <= 64  ("small"): e ~ U[1, 3],  c = 0.05,           s = 0.02
* n >  64  ("large"): e ~ U[1, 10], c = s = 0.02/sqrt(n)

The large regime keeps the spectral norm of both couplings near 0.03 at any n,
so [A B; conj(B) conj(A)] stays positive definite with eigenvalues in about
[0.94, 10.06]. The real variant takes the real parts of G, F and the dipoles.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

SMALL_N_MAX = 64


@dataclass
class BSEProblem:
    n: int
    seed: int
    A: np.ndarray  # (n, n) complex128 (or float64 for the real variant)
    B: np.ndarray  # (n, n)
    d_r: np.ndarray  # (2n,)
    d_l: np.ndarray  # (2n,)
    real: bool


def _cgauss(rng: np.random.Generator, shape) -> np.ndarray:
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2.0)


def recipe(n: int) -> tuple[float, float, float, float]:
    """(e_lo, e_hi, c, s) for problem size n."""
    if n <= SMALL_N_MAX:
        return 1.0, 3.0, 0.05, 0.02
    return 1.0, 10.0, 0.02 / np.sqrt(n), 0.02 / np.sqrt(n)


def make_problem(n: int, seed: int, real: bool = False) -> BSEProblem:
    """Draw one seeded problem of size n (H is 2n x 2n)."""
    if n < 1:
        raise ValueError("n must be >= 1")
    rng = np.random.default_rng(seed)
    e_lo, e_hi, c, s = recipe(n)
    e = rng.uniform(e_lo, e_hi, size=n)
    G = _cgauss(rng, (n, n))
    F = _cgauss(rng, (n, n))
    d = _cgauss(rng, 2 * n)
    if real:
        G, F, d = G.real.copy(), F.real.copy(), d.real.copy()
    A = np.diag(e).astype(G.dtype) + c * (G + G.conj().T) / 2
    B = s * (F + F.T) / 2
    if not real:
        A = A.astype(np.complex128)
        B = B.astype(np.complex128)
        d = d.astype(np.complex128)
    return BSEProblem(n=n, seed=seed, A=A, B=B, d_r=d.copy(), d_l=d.copy(), real=real)


def batch_sizes(count: int, n_lo: int, n_hi: int, seed: int) -> np.ndarray:
    """Sizes drawn log-uniform in [n_lo, n_hi] (integers)."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(np.log(n_lo), np.log(n_hi), size=count)
    return np.clip(np.rint(np.exp(u)).astype(np.int64), n_lo, n_hi)


def poisson_arrivals(count: int, rate_per_s: float, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson stream with the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=count))
