// Algorithm 1 step 1: M = [Re(A+B) Im(A-B); -Im(A+B) Re(A-B)]  (Theorem 2, Eq. embedding).
//
// A, B: n x n complex128, column-major, lower triangles read (A = A^H, B = B^T
// rebuild the upper ones). One CTA per 32x32 tile of (i, j); tiles above the
// diagonal read the mirrored lower tile and transpose it through shared memory,
// so every global read and write is coalesced along the column.
// Traffic per element pair (i, j): 32 B read (A, B) + 4 x 8 B written (M)
// (+ 4 x 4 B for the optional FP32 copy).
#include "common.cuh"
#include "../../include/bse_stages.h"

namespace bse {

__global__ void __launch_bounds__(256) form_M_kernel(int n, const double2* __restrict__ A, long lda,
                                                     const double2* __restrict__ B, long ldb,
                                                     double* __restrict__ M, long ldm,
                                                     float* __restrict__ Mf, long ldmf) {
  __shared__ double2 Sa[32][33];
  __shared__ double2 Sb[32][33];
  const int I = blockIdx.x, J = blockIdx.y;
  const bool upper = I < J;
  // source tile: (I, J) for lower/diagonal tiles, (J, I) for upper ones
  const int si = (upper ? J : I) * 32, sj = (upper ? I : J) * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int c = ty; c < 32; c += 8) {
    int gi = si + tx, gj = sj + c;
    double2 a = make_double2(0, 0), b = make_double2(0, 0);
    if (gi < n && gj < n) {
      a = A[gi + (long)gj * lda];
      b = B[gi + (long)gj * ldb];
    }
    Sa[tx][c] = a;  // Sa[row-in-source-tile][col-in-source-tile]
    Sb[tx][c] = b;
  }
  __syncthreads();
  for (int c = ty; c < 32; c += 8) {
    const int gi = I * 32 + tx, gj = J * 32 + c;
    if (gi >= n || gj >= n) continue;
    double2 a, b;
    if (upper) {
      // element (gi, gj) with gi < gj: A(gi,gj) = conj(A(gj,gi)), B(gi,gj) = B(gj,gi)
      a = Sa[c][tx];
      a.y = -a.y;
      b = Sb[c][tx];
    } else if (gi >= gj) {
      a = Sa[tx][c];
      b = Sb[tx][c];
      if (gi == gj) a.y = 0.0;  // Hermitian diagonal is real
    } else {
      // diagonal tile, strictly upper element: mirror inside the tile
      a = Sa[c][tx];
      a.y = -a.y;
      b = Sb[c][tx];
    }
    const double m11 = a.x + b.x;    // Re(A+B)
    const double m12 = a.y - b.y;    // Im(A-B)
    const double m21 = -(a.y + b.y); // -Im(A+B)
    const double m22 = a.x - b.x;    // Re(A-B)
    M[gi + (long)gj * ldm] = m11;
    M[gi + (long)(n + gj) * ldm] = m12;
    M[(n + gi) + (long)gj * ldm] = m21;
    M[(n + gi) + (long)(n + gj) * ldm] = m22;
    if (Mf) {
      Mf[gi + (long)gj * ldmf] = (float)m11;
      Mf[gi + (long)(n + gj) * ldmf] = (float)m12;
      Mf[(n + gi) + (long)gj * ldmf] = (float)m21;
      Mf[(n + gi) + (long)(n + gj) * ldmf] = (float)m22;
    }
  }
}

int form_M(int n, const double* A, int lda, const double* B, int ldb, double* M, int ldm, float* Mf,
           int ldmf, cudaStream_t s) {
  if (n <= 0) return BSE_OK;
  dim3 grid(ceil_div(n, 32), ceil_div(n, 32));
  KprofScope ks(K_FORM_M, s, 32.0 * n * n + 32.0 * n * n + (Mf ? 16.0 * n * n : 0.0), 0.0);
  form_M_kernel<<<grid, dim3(32, 8), 0, s>>>(n, reinterpret_cast<const double2*>(A), lda,
                                             reinterpret_cast<const double2*>(B), ldb, M, ldm, Mf, ldmf);
  BSE_LAUNCH_CHECK();
  return BSE_OK;
}

}  // namespace bse

extern "C" int bse_stage_form_M(int n, const double* A, int lda, const double* B, int ldb, double* M,
                                int ldm, float* Mf, int ldmf, void* stream) {
  if (n < 1 || !A || !B || !M || lda < n || ldb < n || ldm < 2 * n || (Mf && ldmf < 2 * n))
    return BSE_ERR_ARG;
  return bse::form_M(n, A, lda, B, ldb, M, ldm, Mf, ldmf, (cudaStream_t)stream);
}
