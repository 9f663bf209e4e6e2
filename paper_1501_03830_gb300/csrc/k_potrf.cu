// Algorithm 1 step 2: M = L L^T (Cholesky), blocked right-looking, in place.
//
// Per 64-column block k0:
//   1. potf2 + trtri of the diagonal block in one CTA, in FP64 arithmetic in
//      shared memory whatever the storage type (a pivot <= 0 or NaN records
//      BSE_ERR_NOT_DEFINITE with its 1-based column in the status word: Eq. cond
//      fails; later blocks are skipped);
//   2. panel solve P <- P L_kk^{-T} as a GEMM with the inverted diagonal block;
//   3. trailing update  A22 <- A22 - P P^T  on the lower triangle (GEMM).
// The strict upper triangle of the factored matrix is left untouched.
#include "common.cuh"
#include "gemm_simt.cuh"
#include "../../include/bse_stages.h"

namespace bse {

constexpr int POTRF_NB = 64;

template <typename T>
__global__ void __launch_bounds__(256) potf2_trtri_kernel(int kb, T* __restrict__ Akk, long lda,
                                                          T* __restrict__ Linv, int col0,
                                                          DevStatus* st) {
  __shared__ double L[POTRF_NB][POTRF_NB + 1];
  __shared__ double Li[POTRF_NB][POTRF_NB + 1];
  __shared__ int bad;
  if (st->code != 0) return;  // an earlier block already failed
  const int tid = threadIdx.x;
  for (int e = tid; e < kb * kb; e += blockDim.x) {
    int i = e % kb, j = e / kb;
    L[i][j] = (i >= j) ? (double)Akk[i + (long)j * lda] : 0.0;
    Li[i][j] = 0.0;
  }
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int j = 0; j < kb; ++j) {
    if (tid == 0) {
      double d = L[j][j];
      if (!(d > 0.0)) {
        bad = j + 1;
      } else {
        L[j][j] = sqrt(d);
      }
    }
    __syncthreads();
    if (bad) break;
    const double ljj = L[j][j];
    for (int i = j + 1 + tid; i < kb; i += blockDim.x) L[i][j] /= ljj;
    __syncthreads();
    // rank-1 update of the trailing lower triangle
    const int r = kb - j - 1;
    for (int e = tid; e < r * r; e += blockDim.x) {
      int i = j + 1 + e % r, k = j + 1 + e / r;
      if (i >= k) L[i][k] -= L[i][j] * L[k][j];
    }
    __syncthreads();
  }
  if (bad) {
    if (tid == 0) set_status(st, BSE_ERR_NOT_DEFINITE, col0 + bad);
    return;
  }
  // inverse of the lower-triangular factor, one column per thread
  if (tid < kb) {
    const int j = tid;
    Li[j][j] = 1.0 / L[j][j];
    for (int i = j + 1; i < kb; ++i) {
      double s = 0.0;
      for (int k = j; k < i; ++k) s += L[i][k] * Li[k][j];
      Li[i][j] = -s / L[i][i];
    }
  }
  __syncthreads();
  for (int e = tid; e < kb * kb; e += blockDim.x) {
    int i = e % kb, j = e / kb;
    if (i >= j) Akk[i + (long)j * lda] = (T)L[i][j];
    Linv[i + (long)j * POTRF_NB] = (T)Li[i][j];
  }
}

template <typename T>
size_t potrf_worksize(int m) {
  return sizeof(T) * ((size_t)POTRF_NB * POTRF_NB + (size_t)m * POTRF_NB);
}

template <typename T>
int potrf(int m, T* A, long lda, void* work, DevStatus* st, cudaStream_t s, int col_offset) {
  StatusScope ss(st);
  T* Linv = reinterpret_cast<T*>(work);
  T* Ptmp = Linv + POTRF_NB * POTRF_NB;
  for (int k0 = 0; k0 < m; k0 += POTRF_NB) {
    const int kb = min(POTRF_NB, m - k0);
    T* Akk = A + k0 + (long)k0 * lda;
    {
      KprofScope ks(K_POTRF_DIAG, s, 0.0, kb * (double)kb * kb / 3.0 + kb * (double)kb * kb / 3.0);
      potf2_trtri_kernel<T><<<1, 256, 0, s>>>(kb, Akk, lda, Linv, k0 + col_offset, st);
    }
    BSE_LAUNCH_CHECK();
    const int r = m - k0 - kb;
    if (r <= 0) break;
    T* P = A + (k0 + kb) + (long)k0 * lda;
    // Ptmp = P * Linv^T   (op(B)(k,j) = Linv(j,k): upper triangular)
    BSE_TRY(gemm<T>(r, kb, kb, 1.0, P, lda, false, Linv, POTRF_NB, true, 0.0, Ptmp, m, s, TRI_NONE,
                    TRI_UPPER, 0));
    BSE_CUDA(cudaMemcpy2DAsync(P, lda * sizeof(T), Ptmp, (size_t)m * sizeof(T), (size_t)r * sizeof(T), kb,
                               cudaMemcpyDeviceToDevice, s));
    // A22 -= P P^T, lower triangle
    T* A22 = A + (k0 + kb) + (long)(k0 + kb) * lda;
    BSE_TRY(gemm<T>(r, r, kb, -1.0, P, lda, false, P, lda, true, 1.0, A22, lda, s, TRI_NONE, TRI_NONE, 1));
  }
  return BSE_OK;
}

template size_t potrf_worksize<double>(int);
template size_t potrf_worksize<float>(int);
template int potrf<double>(int, double*, long, void*, DevStatus*, cudaStream_t, int);
template int potrf<float>(int, float*, long, void*, DevStatus*, cudaStream_t, int);

}  // namespace bse

extern "C" size_t bse_stage_potrf_worksize(int m, int fp32) {
  return fp32 ? bse::potrf_worksize<float>(m) : bse::potrf_worksize<double>(m);
}

extern "C" int bse_stage_potrf(int m, void* A, int lda, int fp32, void* work, int* dev_status, void* stream) {
  if (m < 1 || !A || lda < m || !work || !dev_status) return BSE_ERR_ARG;
  auto* st = reinterpret_cast<bse::DevStatus*>(dev_status);
  if (fp32) return bse::potrf<float>(m, (float*)A, lda, work, st, (cudaStream_t)stream, 0);
  return bse::potrf<double>(m, (double*)A, lda, work, st, (cudaStream_t)stream, 0);
}
