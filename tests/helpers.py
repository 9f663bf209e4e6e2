"""Shared helpers for the GPU tests (device buffers through torch, comparisons)."""
from __future__ import annotations

import numpy as np


def torch_cuda():
    import pytest

    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def dev_c128(torch, a: np.ndarray):
    """Column-major complex128 matrix -> CUDA tensor with the same memory layout
    (the tensor is the transpose view, so data_ptr() is column-major data)."""
    a = np.asfortranarray(a, dtype=np.complex128)
    t = torch.from_numpy(np.ascontiguousarray(a.T)).cuda()
    return t


def dev_f(torch, a: np.ndarray, dtype="float64"):
    """Column-major real matrix -> CUDA tensor holding the column-major data."""
    a = np.asfortranarray(a, dtype=dtype)
    return torch.from_numpy(np.ascontiguousarray(a.T)).cuda()


def host_colmajor(t, shape) -> np.ndarray:
    """CUDA tensor holding column-major data -> numpy array of the given shape."""
    a = t.detach().cpu().numpy()
    return np.asfortranarray(a.reshape(shape[::-1]).T)


def projector_gap(X1, X2, n):
    """Max over columns of || x1 y1^H - x2 y2^H || (phase-free, y = diag(I,-I) x)."""
    s = np.concatenate([np.ones(n), -np.ones(n)])[:, None]
    worst = 0.0
    for j in range(X1.shape[1]):
        P1 = np.outer(X1[:, j], (s * X1)[:, j].conj())
        P2 = np.outer(X2[:, j], (s * X2)[:, j].conj())
        worst = max(worst, float(np.max(np.abs(P1 - P2))))
    return worst


def rel_err(a, b) -> float:
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b)) / np.abs(np.asarray(b))))
