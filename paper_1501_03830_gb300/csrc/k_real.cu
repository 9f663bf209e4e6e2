// Real Bethe-Salpeter problems (Section 3.2, Theorem 5, Algorithm 2).
//
// For real symmetric A, B the matrix M of Theorem 2 is diag(A + B, A - B), so
// its Cholesky factor is diag(L1, L2) with A + B = L1 L1^T, A - B = L2 L2^T
// (Algorithm 2 step 1: two n x n factorizations), and W = L^T J L has the
// off-diagonal blocks L1^T L2 and -L2^T L1: the skew embedding of K = L2^T L1,
// whose eigenvalues +-i sigma_j carry the singular values of K and whose
// eigenvectors [v; i u] carry its singular vectors. The tridiagonal machinery of
// the complex path therefore computes the SVD of Algorithm 2 step 2, and its
// back-transform returns the eigenvectors x_j of H (Theorem 5's X up to a phase
// per column). Two kernels adapt the data at the ends:
//   real_to_complex   real n x n input -> complex128 with zero imaginary part
//   real_vectors      x_j -> the real X1, X2 of Algorithm 2: the phase that makes
//                     the largest-modulus entry real positive is removed, the
//                     real part kept and renormalized so x^T diag(I,-I) x = 1
//                     (X1^T X1 - X2^T X2 = I).
#include "common.cuh"
#include "internal.cuh"

namespace bse {

__global__ void __launch_bounds__(256) real_to_complex_kernel(int n, const double* __restrict__ R, long ldr,
                                                              double2* __restrict__ Z) {
  const int i = blockIdx.x * 256 + threadIdx.x;
  const int j = blockIdx.y;
  if (i < n) Z[i + (long)j * n] = make_double2(R[i + (long)j * ldr], 0.0);
}

int real_to_complex(int n, const double* R, long ldr, double* Z, cudaStream_t s) {
  kcount(1);
  real_to_complex_kernel<<<dim3(ceil_div(n, 256), n), 256, 0, s>>>(n, R, ldr, reinterpret_cast<double2*>(Z));
  BSE_LAUNCH_CHECK();
  return BSE_OK;
}

// One block per column j of X (2n complex entries, contiguous).
__global__ void __launch_bounds__(256) real_vectors_kernel(int n, const double2* __restrict__ X, long ldx,
                                                           double* __restrict__ X1, double* __restrict__ X2,
                                                           long ldo) {
  __shared__ double sv[8];
  __shared__ int si[8];
  __shared__ double snorm[8];
  __shared__ double2 sph;
  const int j = blockIdx.x, m = 2 * n;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const double2* x = X + (long)j * ldx;
  // largest modulus, smallest index among ties
  double best = -1.0;
  int bi = 0;
  for (int i = tid; i < m; i += 256) {
    const double2 v = x[i];
    const double a = v.x * v.x + v.y * v.y;
    if (a > best) {
      best = a;
      bi = i;
    }
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    const double ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ob > best || (ob == best && oi < bi)) {
      best = ob;
      bi = oi;
    }
  }
  if (lane == 0) {
    sv[wid] = best;
    si[wid] = bi;
  }
  __syncthreads();
  if (tid == 0) {
    double b = sv[0];
    int k = si[0];
    for (int w = 1; w < 8; ++w)
      if (sv[w] > b || (sv[w] == b && si[w] < k)) {
        b = sv[w];
        k = si[w];
      }
    const double2 v = x[k];
    const double r = sqrt(v.x * v.x + v.y * v.y);
    sph = r > 0.0 ? make_double2(v.x / r, -v.y / r) : make_double2(1.0, 0.0);  // conj(v) / |v|
  }
  __syncthreads();
  const double2 ph = sph;
  // real part after the phase, and its diag(I, -I) norm
  double s = 0.0;
  for (int i = tid; i < m; i += 256) {
    const double2 v = x[i];
    const double re = v.x * ph.x - v.y * ph.y;
    s += (i < n) ? re * re : -re * re;
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) snorm[wid] = s;
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int w = 0; w < 8; ++w) t += snorm[w];
  const double scale = t > 0.0 ? 1.0 / sqrt(t) : 1.0;
  for (int i = tid; i < m; i += 256) {
    const double2 v = x[i];
    const double re = (v.x * ph.x - v.y * ph.y) * scale;
    if (i < n) {
      if (X1) X1[i + (long)j * ldo] = re;
    } else if (X2) {
      X2[(i - n) + (long)j * ldo] = re;
    }
  }
}

int real_vectors(int n, const double* X, long ldx, double* X1, double* X2, long ldo, cudaStream_t s) {
  kcount(1);
  real_vectors_kernel<<<n, 256, 0, s>>>(n, reinterpret_cast<const double2*>(X), ldx, X1, X2, ldo);
  BSE_LAUNCH_CHECK();
  return BSE_OK;
}

}  // namespace bse
