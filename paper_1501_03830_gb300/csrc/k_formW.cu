// Algorithm 1 step 3: W = L^T J L (real skew-symmetric), using the block
// structure of L = [L11 0; L21 L22] and J = [0 I; -I 0]:
//
//   W = [ C - C^T      L11^T L22 ]      C = L11^T L21
//       [ -L22^T L11   0         ]
//
// Only the strict lower triangle of W is produced (that is all the skew
// tridiagonal reduction reads): W11 = C - C^T (strict lower), W21 = -L22^T L11,
// W22 = 0. C is formed in W's own (unused) upper-right block as scratch.
// Flops: n^3 (C, triangular x full) + 2n^3/3 (W21, triangular x triangular).
#include "common.cuh"
#include "gemm_simt.cuh"
#include "../../include/bse_stages.h"

namespace bse {

template <typename T>
__global__ void __launch_bounds__(256) skew_from_C_kernel(int n, T* __restrict__ W, long ldw) {
  // W[i, j] = C[i, j] - C[j, i] for i > j (C at W[0:n, n:2n]); W[i, i] = 0.
  __shared__ T Ct[32][33];
  const int I = blockIdx.x, J = blockIdx.y;
  if (I < J) return;
  const T* C = W + (long)n * ldw;
  const int tx = threadIdx.x, ty = threadIdx.y;
  // load the mirrored tile C[J*32 + a, I*32 + b] as Ct[a][b]
  for (int c = ty; c < 32; c += 8) {
    int gi = J * 32 + tx, gj = I * 32 + c;
    Ct[tx][c] = (gi < n && gj < n) ? C[gi + (long)gj * ldw] : T(0);
  }
  __syncthreads();
  for (int c = ty; c < 32; c += 8) {
    int gi = I * 32 + tx, gj = J * 32 + c;
    if (gi >= n || gj >= n || gi < gj) continue;
    T v = T(0);
    if (gi > gj) v = C[gi + (long)gj * ldw] - Ct[c][tx];
    W[gi + (long)gj * ldw] = v;
  }
}

template <typename T>
int form_W(int n, const T* L, long ldl, T* W, long ldw, cudaStream_t s) {
  const T* L11 = L;
  const T* L21 = L + n;
  const T* L22 = L + n + (long)n * ldl;
  T* Cs = W + (long)n * ldw;  // scratch: W[0:n, n:2n]
  // C = L11^T L21   (op(A)(i,k) = L11(k,i): zero for k < i)
  BSE_TRY(gemm<T>(n, n, n, 1.0, L11, ldl, true, L21, ldl, false, 0.0, Cs, ldw, s, TRI_UPPER, TRI_NONE, 0));
  dim3 grid(ceil_div(n, 32), ceil_div(n, 32));
  {
    KprofScope ks(K_ELEMENTWISE, s, 2.0 * sizeof(T) * n * n, 0.0);
    skew_from_C_kernel<T><<<grid, dim3(32, 8), 0, s>>>(n, W, ldw);
  }
  BSE_LAUNCH_CHECK();
  // W21 = -L22^T L11  (op(A) upper: zero for k < i; op(B) = L11 lower: zero for k < j)
  BSE_TRY(gemm<T>(n, n, n, -1.0, L22, ldl, true, L11, ldl, false, 0.0, W + n, ldw, s, TRI_UPPER, TRI_LOWER, 0));
  // W22 = 0
  BSE_CUDA(cudaMemset2DAsync(W + n + (long)n * ldw, ldw * sizeof(T), 0, n * sizeof(T), n, s));
  return BSE_OK;
}

template int form_W<double>(int, const double*, long, double*, long, cudaStream_t);
template int form_W<float>(int, const float*, long, float*, long, cudaStream_t);

}  // namespace bse

extern "C" int bse_stage_form_W(int n, const void* L, int ldl, void* W, int ldw, int fp32, void* stream) {
  if (n < 1 || !L || !W || ldl < 2 * n || ldw < 2 * n) return BSE_ERR_ARG;
  if (fp32) return bse::form_W<float>(n, (const float*)L, ldl, (float*)W, ldw, (cudaStream_t)stream);
  return bse::form_W<double>(n, (const double*)L, ldl, (double*)W, ldw, (cudaStream_t)stream);
}
