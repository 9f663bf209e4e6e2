"""The tcgen05 tensor-core GEMM and the FP64-accurate digit-split product built on it.

The digit product relies on the tensor cores accumulating integer-valued bf16
products exactly in FP32 (every partial sum is an integer below 2^24); the first
test checks exactly that against an FP64 product of the same integers.
"""
import numpy as np
import pytest

from tests.helpers import torch_cuda

pytestmark = pytest.mark.gpu


def _lib():
    from paper_1501_03830_gb300 import bse

    return bse.lib(), bse


def _tc(torch, L, bse, A, B, ldk):
    M, K = A.shape
    N = B.shape[0]
    Ap = torch.zeros(M, ldk, dtype=torch.bfloat16, device="cuda")
    Bp = torch.zeros(N, ldk, dtype=torch.bfloat16, device="cuda")
    Ap[:, :K] = A
    Bp[:, :K] = B
    C = torch.empty(N, M, dtype=torch.float32, device="cuda")  # column-major M x N
    st = torch.zeros(4, dtype=torch.int32, device="cuda")
    bse.check(L.bse_tc_gemm_bf16(M, N, K, Ap.data_ptr(), Bp.data_ptr(), ldk, C.data_ptr(), M, st.data_ptr(), None),
              "tc_gemm")
    torch.cuda.synchronize()
    assert int(st[0].item()) == 0
    return C.t()


@pytest.mark.parametrize("M,N,K,ldk", [(128, 256, 16384, 16384), (200, 300, 1000, 1024), (384, 512, 4096, 4096)])
def test_tc_gemm_exact_integer_digits(M, N, K, ldk):
    torch = torch_cuda()
    L, bse = _lib()
    g = torch.Generator(device="cuda")
    g.manual_seed(M + N + K)
    lim = 32 if K <= 16384 else 16
    A = torch.randint(-lim, lim + 1, (M, K), generator=g, device="cuda").to(torch.bfloat16)
    B = torch.randint(-lim, lim + 1, (N, K), generator=g, device="cuda").to(torch.bfloat16)
    C = _tc(torch, L, bse, A, B, ldk)
    ref = A.double() @ B.double().t()
    assert torch.equal(C.double(), ref)


def test_tc_gemm_random_values():
    torch = torch_cuda()
    L, bse = _lib()
    g = torch.Generator(device="cuda")
    g.manual_seed(7)
    M, N, K = 256, 512, 2048
    A = torch.randn(M, K, generator=g, device="cuda").to(torch.bfloat16)
    B = torch.randn(N, K, generator=g, device="cuda").to(torch.bfloat16)
    C = _tc(torch, L, bse, A, B, K)
    ref = A.double() @ B.double().t()
    assert torch.max(torch.abs(C.double() - ref)).item() <= 1e-4 * torch.max(torch.abs(ref)).item()


@pytest.mark.parametrize("M,N,K,s", [(256, 256, 2048, 8), (300, 200, 1500, 8), (512, 512, 16384, 10)])
def test_ozaki_fp64_accuracy(M, N, K, s):
    torch = torch_cuda()
    L, bse = _lib()
    rng = np.random.default_rng(M * N + K)
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((K, N))
    Ad = torch.from_numpy(np.ascontiguousarray(A)).cuda()  # row i contiguous: K-major
    Bd = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()  # column j contiguous
    C = torch.zeros(N, M, dtype=torch.float64, device="cuda")
    work = torch.empty(L.bse_ozaki_worksize(M, N, K, s), dtype=torch.uint8, device="cuda")
    st = torch.zeros(4, dtype=torch.int32, device="cuda")
    bse.check(L.bse_ozaki_gemm(M, N, K, Ad.data_ptr(), K, Bd.data_ptr(), K, C.data_ptr(), M, s, work.data_ptr(),
                               st.data_ptr(), None), "ozaki")
    torch.cuda.synchronize()
    assert int(st[0].item()) == 0
    got = C.cpu().numpy().T
    ref = A @ B
    scale = np.abs(A) @ np.abs(B)
    beta = (24 - int(np.ceil(np.log2((K + 63) // 64 * 64)))) // 2
    bound = 8.0 * 2.0 ** (-beta * s) * np.max(np.abs(A)) * np.max(np.abs(B)) * K
    assert np.max(np.abs(got - ref)) <= max(bound, 4e-16 * np.max(scale))
    # FP64-level: far below what FP32 accumulation gives
    assert np.max(np.abs(got - ref) / scale) <= 1e-12
