// Absorption-spectrum weights (Section 1, Eq. absp):
//
//   w_j = (d_r^H x_j) (y_j^H d_l) / (y_j^H x_j),   y_j = diag(I,-I) x_j (Theorem 3)
//
// One CTA per eigenvector column; the column (2n complex128, contiguous) is
// streamed once and the three complex dot products are reduced together.
// HBM-bound: 32n bytes per column (the left eigenvector is derived on the fly).
#include "common.cuh"
#include "../../include/bse_stages.h"

namespace bse {

__device__ __forceinline__ double2 cmul_conj(double2 a, double2 b) {  // conj(a) * b
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

__global__ void __launch_bounds__(256) weights_kernel(int n, const double2* __restrict__ X, long ldx,
                                                      const double2* __restrict__ dr,
                                                      const double2* __restrict__ dl, double2* __restrict__ w) {
  __shared__ double red[8][5];
  const int j = blockIdx.x;
  const int m = 2 * n;
  const double2* x = X + (long)j * ldx;
  double ar = 0, ai = 0, br = 0, bi = 0, c = 0;
  for (int i = threadIdx.x; i < m; i += 256) {
    const double2 xi = x[i];
    const double s = (i < n) ? 1.0 : -1.0;
    const double2 a = cmul_conj(dr[i], xi);  // conj(d_r) x
    const double2 y = make_double2(s * xi.x, s * xi.y);
    const double2 b = cmul_conj(y, dl[i]);   // conj(y) d_l
    ar += a.x; ai += a.y; br += b.x; bi += b.y;
    c += s * (xi.x * xi.x + xi.y * xi.y);     // conj(y) x is real
  }
  for (int o = 16; o >= 1; o >>= 1) {
    ar += __shfl_xor_sync(0xffffffffu, ar, o);
    ai += __shfl_xor_sync(0xffffffffu, ai, o);
    br += __shfl_xor_sync(0xffffffffu, br, o);
    bi += __shfl_xor_sync(0xffffffffu, bi, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
  }
  const int wid = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    red[wid][0] = ar; red[wid][1] = ai; red[wid][2] = br; red[wid][3] = bi; red[wid][4] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s[5] = {0, 0, 0, 0, 0};
    for (int k = 0; k < 8; ++k)
      for (int q = 0; q < 5; ++q) s[q] += red[k][q];
    const double pr = s[0] * s[2] - s[1] * s[3];
    const double pi = s[0] * s[3] + s[1] * s[2];
    w[j] = make_double2(pr / s[4], pi / s[4]);
  }
}

int weights(int n, const double* X, long ldx, const double* dr, const double* dl, double* w, cudaStream_t s) {
  if (n <= 0) return BSE_OK;
  KprofScope ks(K_WEIGHTS, s, 32.0 * n * (double)n + 64.0 * n, 0.0);
  weights_kernel<<<n, 256, 0, s>>>(n, reinterpret_cast<const double2*>(X), ldx,
                                   reinterpret_cast<const double2*>(dr), reinterpret_cast<const double2*>(dl),
                                   reinterpret_cast<double2*>(w));
  BSE_LAUNCH_CHECK();
  return BSE_OK;
}

}  // namespace bse

extern "C" int bse_stage_weights(int n, const double* X, int ldx, const double* d_r, const double* d_l, double* w,
                                 void* stream) {
  if (n < 1 || !X || ldx < 2 * n || !d_r || !d_l || !w) return BSE_ERR_ARG;
  return bse::weights(n, X, ldx, d_r, d_l, w, (cudaStream_t)stream);
}
