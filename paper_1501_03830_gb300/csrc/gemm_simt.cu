// Host launchers for the SIMT GEMM (FP64: 64x64x16 tiles, 4x4 per thread;
// FP32: 128x128x16 tiles, 8x8 per thread; 256 threads per CTA).
#include "gemm_simt.cuh"
#include "tc32.cuh"

namespace bse {

template <typename T, int BM, int BN, int BK, int TM, int TN>
static int launch_gemm(const GemmArgs& g, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0) return BSE_OK;
  if (g.K <= 0 && g.beta == 1.0) return BSE_OK;
  constexpr int NT = (BM / TM) * (BN / TN);
  long tiles = (long)ceil_div(g.M, BM) * ceil_div(g.N, BN);
  dim3 grid((unsigned)tiles, 1, (unsigned)(g.batch > 0 ? g.batch : 1));
  // charged flops: 2MNK, halved for a triangular output and for each triangular operand
  double fl = 2.0 * g.M * g.N * (double)g.K * (g.batch > 0 ? g.batch : 1);
  if (g.c_uplo) fl *= 0.5;
  if (g.a_tri) fl *= 0.5;
  if (g.b_tri) fl *= 0.5;
  KprofScope ks(sizeof(T) == 8 ? K_GEMM_F64 : K_GEMM_F32, s, 0.0, fl);
  if (!g.transA && !g.transB)
    gemm_simt_kernel<T, BM, BN, BK, TM, TN, false, false><<<grid, NT, 0, s>>>(g);
  else if (!g.transA && g.transB)
    gemm_simt_kernel<T, BM, BN, BK, TM, TN, false, true><<<grid, NT, 0, s>>>(g);
  else if (g.transA && !g.transB)
    gemm_simt_kernel<T, BM, BN, BK, TM, TN, true, false><<<grid, NT, 0, s>>>(g);
  else
    gemm_simt_kernel<T, BM, BN, BK, TM, TN, true, true><<<grid, NT, 0, s>>>(g);
  BSE_LAUNCH_CHECK();
  return BSE_OK;
}

template <>
int gemm<double>(const GemmArgs& g, cudaStream_t s) {
  return launch_gemm<double, 64, 64, 16, 4, 4>(g, s);
}

// FP32: the 3xTF32 tensor-core kernel takes every product it can lay out
// (aligned operands, no triangular masks) that is large enough to fill the GPU;
// the rest runs on the SIMT kernel.
template <>
int gemm<float>(const GemmArgs& g, cudaStream_t s) {
  if (tc32::mode() >= 1 && (double)g.M * g.N * (double)g.K >= (double)(1 << 21) && tc32::eligible(g))
    return tc32::gemm(g, 1, nullptr, s);
  return launch_gemm<float, 128, 128, 16, 8, 8>(g, s);
}

}  // namespace bse
