"""The tcgen05 tensor-core GEMM and the FP64-accurate digit-split product built on it.

The digit product relies on the tensor cores accumulating integer-valued bf16
products exactly in FP32 (every partial sum of a 256-deep chunk is an integer
below 2^22); the first test checks exactness against an FP64 product of the same
integers, and the integer-input digit-product test checks the whole chain
(digits, chunk sums, int32 anti-diagonal planes, FP64 combination) exactly.
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
    beta = L.bse_ozaki_digit_bits(K)
    assert beta == 8
    # the anti-diagonal bound K 2^(2 beta - 2) s < 2^31 lowers beta for many digits
    while K * 2.0 ** (2 * beta - 2) * s >= 2.0 ** 31:
        beta -= 1
    # s digits carry beta s - 1 bits relative to the row / column magnitudes
    bound = 16.0 * 2.0 ** (-beta * s) * np.max(np.abs(A)) * np.max(np.abs(B)) * K
    assert np.max(np.abs(got - ref)) <= max(bound, 4e-16 * np.max(scale))
    # FP64-level: far below what FP32 accumulation gives
    assert np.max(np.abs(got - ref) / scale) <= 1e-12


@pytest.mark.parametrize("M,N,K", [(384, 512, 4096), (512, 512, 1000), (256, 768, 16384)])
def test_ozaki_exact_on_integer_inputs(M, N, K):
    """Integer entries below 2^13 need two 8-bit digits (the leading one held to
    2^7), so s = 3 digit pairs (p + q < 3) cover every nonzero digit product; all
    sums are integers
    below 2^53, so the result must equal the integer product exactly. Row
    magnitudes vary (rows scaled down by powers of two) so the per-row digit
    scales differ."""
    torch = torch_cuda()
    L, bse = _lib()
    rng = np.random.default_rng(M + N + K)
    A = rng.integers(-(2 ** 13) + 1, 2 ** 13, size=(M, K)).astype(np.float64)
    A = np.trunc(A / (2.0 ** (np.arange(M) % 9))[:, None])
    B = rng.integers(-(2 ** 13) + 1, 2 ** 13, size=(K, N)).astype(np.float64)
    Ad = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    Bd = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()
    s = 3
    C = torch.full((N, M), np.nan, dtype=torch.float64, device="cuda")
    work = torch.empty(L.bse_ozaki_worksize(M, N, K, s), dtype=torch.uint8, device="cuda")
    st = torch.zeros(4, dtype=torch.int32, device="cuda")
    bse.check(L.bse_ozaki_gemm(M, N, K, Ad.data_ptr(), K, Bd.data_ptr(), K, C.data_ptr(), M, s, work.data_ptr(),
                               st.data_ptr(), None), "ozaki")
    torch.cuda.synchronize()
    assert int(st[0].item()) == 0
    ref = A @ B  # exact: |entries| < 2^13 * 2^13 * K < 2^53
    assert np.array_equal(C.cpu().numpy().T, ref)


# ---- FP32 GEMM on the tensor cores (3xTF32) ---------------------------------


def _colmajor(torch, rows, cols, ld, g):
    """A rows x cols FP32 matrix stored column-major with leading dimension ld,
    as (storage tensor, the matrix view)."""
    buf = torch.randn(cols, ld, generator=g, device="cuda", dtype=torch.float32)
    return buf, buf[:, :rows].t()


def _tc32(torch, L, bse, M, N, K, ta, tb, alpha, beta, uplo, split, seed):
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    pad = lambda x: (x + 3) // 4 * 4 + 4
    ar, ac = (K, M) if ta else (M, K)
    br, bc = (N, K) if tb else (K, N)
    Abuf, A = _colmajor(torch, ar, ac, pad(ar), g)
    Bbuf, B = _colmajor(torch, br, bc, pad(br), g)
    Cbuf, Cm = _colmajor(torch, M, N, M + 1, g)
    C0 = Cm.double().clone()
    st = torch.zeros(4, dtype=torch.int32, device="cuda")
    bse.check(L.bse_tc32_gemm(M, N, K, alpha, Abuf.data_ptr(), Abuf.shape[1], int(ta), Bbuf.data_ptr(),
                              Bbuf.shape[1], int(tb), beta, Cbuf.data_ptr(), M + 1, uplo, split, st.data_ptr(), None),
              "tc32")
    torch.cuda.synchronize()
    assert int(st[0].item()) == 0
    opA = A.double().t() if ta else A.double()
    opB = B.double().t() if tb else B.double()
    ref = alpha * (opA @ opB) + beta * C0
    scale = abs(alpha) * (opA.abs() @ opB.abs())
    return Cm.double(), ref, scale, C0


@pytest.mark.parametrize("ta,tb", [(0, 0), (0, 1), (1, 0), (1, 1)])
@pytest.mark.parametrize("M,N,K", [(128, 128, 32), (300, 200, 150), (257, 131, 77), (1000, 700, 600)])
def test_tc32_gemm_3xtf32(ta, tb, M, N, K):
    """3xTF32 reaches FP32-level accuracy for every transpose combination, with
    ragged tiles in M, N and K (bound: a few units of 2^-21 times |A||B|)."""
    torch = torch_cuda()
    L, bse = _lib()
    C, ref, scale, _ = _tc32(torch, L, bse, M, N, K, ta, tb, -1.5, 0.5, 0, 1, 11 + M + 2 * ta + tb)
    err = ((C - ref).abs() / (scale + 1e-30)).max().item()
    assert err < 4e-6, err


@pytest.mark.parametrize("ta,tb", [(0, 0), (1, 0)])
def test_tc32_gemm_single_pass(ta, tb):
    """One TF32 pass: 10-bit operands, so errors of order 2^-11 |A||B| and clearly
    above those of the 3xTF32 path on the same inputs."""
    torch = torch_cuda()
    L, bse = _lib()
    C1, ref, scale, _ = _tc32(torch, L, bse, 384, 256, 512, ta, tb, 1.0, 0.0, 0, 0, 5)
    C3, _, _, _ = _tc32(torch, L, bse, 384, 256, 512, ta, tb, 1.0, 0.0, 0, 1, 5)
    e1 = ((C1 - ref).abs() / scale).max().item()
    e3 = ((C3 - ref).abs() / scale).max().item()
    assert e1 < 2e-3 and e3 < 4e-6 and e1 > 20 * e3, (e1, e3)


@pytest.mark.parametrize("uplo", [1, 2])
def test_tc32_gemm_lower_triangle(uplo):
    """uplo = 1 / 2: the lower (strict lower) triangle is the product, the rest of C is untouched."""
    torch = torch_cuda()
    L, bse = _lib()
    n = 600
    C, ref, scale, C0 = _tc32(torch, L, bse, n, n, 128, 0, 1, 1.0, 1.0, uplo, 1, 21 + uplo)
    i = torch.arange(n, device="cuda")
    low = (i[:, None] >= i[None, :]) if uplo == 1 else (i[:, None] > i[None, :])
    assert torch.equal(C[~low], C0[~low])
    err = ((C - ref).abs() / scale)[low].max().item()
    assert err < 4e-6, err


@pytest.mark.parametrize("ta,tb", [(0, 0), (0, 1), (1, 0), (1, 1)])
@pytest.mark.parametrize("M,N,K,uplo", [(257, 131, 77, 0), (1000, 700, 600, 0), (600, 600, 200, 1), (300, 300, 33, 2)])
def test_tc32_presplit_matches_in_kernel_split(ta, tb, M, N, K, uplo):
    """Operands split once into TF32 hi / lo planes in global memory (mode 3: for
    every product) and split tile by tile in shared memory (mode 1) feed the
    tensor cores the same values in the same order: the products agree bit for
    bit, ragged tails and triangular C included."""
    torch = torch_cuda()
    L, bse = _lib()
    if uplo:
        N = M
    out = {}
    try:
        for mode in (1, 3):
            assert L.bse_set_fp32_gemm(mode) == 0
            out[mode] = _tc32(torch, L, bse, M, N, K, ta, tb, 0.75, -0.5, uplo, 1, 31 + M + K + 2 * ta + tb)
    finally:
        L.bse_set_fp32_gemm(2)
    assert torch.equal(out[1][0], out[3][0])
    C, ref, scale, C0 = out[3]
    rel = (C - ref).abs() / (scale + 1e-30)
    if uplo:
        i = torch.arange(M, device="cuda")
        low = (i[:, None] >= i[None, :]) if uplo == 1 else (i[:, None] > i[None, :])
        assert torch.equal(C[~low], C0[~low])
        rel = rel[low]
    assert rel.max().item() < 4e-6, rel.max().item()


def test_tc32_gemm_rejects_unaligned_pitch():
    torch = torch_cuda()
    L, bse = _lib()
    A = torch.zeros(64 * 65, device="cuda")
    C = torch.zeros(64 * 64, device="cuda")
    st = torch.zeros(4, dtype=torch.int32, device="cuda")
    rc = L.bse_tc32_gemm(64, 64, 64, 1.0, A.data_ptr(), 65, 0, A.data_ptr(), 65, 0, 0.0, C.data_ptr(), 64, 0, 1,
                         st.data_ptr(), None)
    assert rc == -1


@pytest.mark.parametrize("M,N,K,s", [(512, 512, 4096, 8), (1024, 768, 16384, 10), (1024, 1024, 8192, 10)])
def test_ozaki_fp64_accurate_and_repeatable(M, N, K, s):
    """The digit-split product over several 128 x 256 tiles and long K is
    FP64-accurate and gives bit-for-bit the same result when repeated (integer
    chunk sums, fixed combination order)."""
    torch = torch_cuda()
    L, bse = _lib()
    g = torch.Generator(device="cuda")
    g.manual_seed(M + K)
    A = torch.randn(M, K, dtype=torch.float64, device="cuda", generator=g)
    B = torch.randn(N, K, dtype=torch.float64, device="cuda", generator=g)
    work = torch.empty(L.bse_ozaki_worksize(M, N, K, s), dtype=torch.uint8, device="cuda")
    st = torch.zeros(4, dtype=torch.int32, device="cuda")
    out = []
    for _ in range(2):
        C = torch.zeros(N, M, dtype=torch.float64, device="cuda")
        bse.check(L.bse_ozaki_gemm(M, N, K, A.data_ptr(), K, B.data_ptr(), K, C.data_ptr(), M, s, work.data_ptr(),
                                   st.data_ptr(), None), "ozaki")
        torch.cuda.synchronize()
        assert int(st[0].item()) == 0
        out.append(C.t().clone())
    assert torch.equal(out[0], out[1])
    ref = A @ B.t()
    scale = A.abs().max(dim=1).values[:, None] * B.abs().max(dim=1).values[None, :] * K ** 0.5
    assert ((out[0] - ref).abs() / scale).max().item() < 1e-13
