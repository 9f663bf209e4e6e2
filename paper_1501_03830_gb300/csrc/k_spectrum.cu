// Spectral density and broadened optical absorption spectrum (Section 1,
// Eq. DOS and Eq. absp; Section 5 replaces the delta function by a Gaussian of
// standard deviation sigma):
//
//   g(t)      = exp(-t^2 / (2 sigma^2)) / (sqrt(2 pi) sigma)
//   phi(w)    = 1/(2n) sum_{j=1..n} [ g(w - lambda_j) + g(w + lambda_j) ]
//   eps+(w)   = sum_{j=1..n} w_j g(w - lambda_j)
//
// phi sums over all 2n eigenvalues of H, which are +-lambda_j (Theorem 1);
// eps+ over the positive half with the complex weights w_j of Eq. absp.
//
// One thread per grid point; the eigenvalues and weights are staged through
// shared memory 256 at a time. A term whose exponent is above 750 is skipped:
// exp(-750) is below the smallest FP64 subnormal, so the skipped term is an
// exact zero and the sum equals the full sum over j. Work n x n_omega (FP64
// exponentials, FP64-ALU bound); no HBM traffic to speak of.
#include <math.h>

#include "common.cuh"
#include "internal.cuh"
#include "solver.h"

namespace bse {

constexpr int SPEC_THREADS = 256;

__global__ void __launch_bounds__(SPEC_THREADS) broaden_kernel(int n, const double* __restrict__ lam,
                                                               const double2* __restrict__ w, int n_omega,
                                                               const double* __restrict__ omega, double sigma,
                                                               double* __restrict__ dos, double2* __restrict__ eps) {
  __shared__ double sl[SPEC_THREADS];
  __shared__ double2 sw[SPEC_THREADS];
  const int k = blockIdx.x * SPEC_THREADS + threadIdx.x;
  const double om = k < n_omega ? omega[k] : 0.0;
  const double h = 0.5 / (sigma * sigma);
  double d = 0.0, er = 0.0, ei = 0.0;
  for (int j0 = 0; j0 < n; j0 += SPEC_THREADS) {
    const int cnt = min(SPEC_THREADS, n - j0);
    if (threadIdx.x < cnt) {
      sl[threadIdx.x] = lam[j0 + threadIdx.x];
      if (w) sw[threadIdx.x] = w[j0 + threadIdx.x];
    }
    __syncthreads();
    for (int jj = 0; jj < cnt; ++jj) {
      const double l = sl[jj];
      const double tm = om - l, tp = om + l;
      const double am = tm * tm * h, ap = tp * tp * h;
      const double gm = am < 750.0 ? exp(-am) : 0.0;
      const double gp = ap < 750.0 ? exp(-ap) : 0.0;
      d += gm + gp;
      if (w) {
        er = fma(sw[jj].x, gm, er);
        ei = fma(sw[jj].y, gm, ei);
      }
    }
    __syncthreads();
  }
  if (k < n_omega) {
    const double g0 = 1.0 / (sqrt(2.0 * M_PI) * sigma);
    dos[k] = d * g0 / (2.0 * n);
    if (eps) eps[k] = make_double2(er * g0, ei * g0);
  }
}

int broaden(int n, const double* lam, const double* w, int n_omega, const double* omega, double sigma, double* dos,
            double* eps, cudaStream_t s) {
  if (n_omega <= 0) return BSE_OK;
  KprofScope ks(K_WEIGHTS, s, 8.0 * n_omega * 3.0, 0.0);
  broaden_kernel<<<ceil_div(n_omega, SPEC_THREADS), SPEC_THREADS, 0, s>>>(
      n, lam, reinterpret_cast<const double2*>(w), n_omega, omega, sigma, dos, reinterpret_cast<double2*>(eps));
  BSE_LAUNCH_CHECK();
  return BSE_OK;
}

}  // namespace bse

extern "C" int bse_stage_broaden(int n, const double* lambda, const double* w, int n_omega, const double* omega,
                                 double sigma, double* dos, double* eps, void* stream) {
  if (n < 1 || n_omega < 0 || !lambda || !(sigma > 0.0) || (n_omega > 0 && (!omega || !dos)) || (eps && !w))
    return BSE_ERR_ARG;
  return bse::broaden(n, lambda, w, n_omega, omega, sigma, dos, eps, (cudaStream_t)stream);
}

// Spectral density (and, with dipoles, the absorption spectrum) of a kept
// solution on a grid; every pointer may be host or device memory.
extern "C" int bse_absorption(bse_ctx* c, const bse_sol* sol, const double* d_r, const double* d_l, int n_omega,
                              const double* omega, double sigma, double* dos, double* eps) {
  if (!c || !sol || n_omega < 1 || !omega || !dos || !(sigma > 0.0) || (eps && (!d_r || !d_l)) ||
      (!d_r) != (!d_l))
    return BSE_ERR_ARG;
  BSE_CUDA(cudaSetDevice(c->device));
  cudaStream_t s = c->stream;
  const int n = sol->n, m = 2 * n;
  const bool want_eps = eps != nullptr;
  // staging: dipoles (2 x m complex), weights (n complex), grid, dos, eps
  const size_t nb = 16 * (size_t)(2 * m + n) + 8 * (size_t)n_omega * 4;
  char* buf = nullptr;
  BSE_CUDA(cudaMallocAsync((void**)&buf, nb, s));
  double* dr = reinterpret_cast<double*>(buf);
  double* dl = dr + 2 * m;
  double* dw = dl + 2 * m;
  double* dom = dw + 2 * n;
  double* ddos = dom + n_omega;
  double* deps = ddos + n_omega;
  int rc = BSE_OK;
  auto in = [&](double* dst, const double* src, size_t bytes) {
    const cudaMemcpyKind k = bse::is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    return cudaMemcpyAsync(dst, src, bytes, k, s);
  };
  auto out = [&](double* dst, const double* src, size_t bytes) {
    const cudaMemcpyKind k = bse::is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    return cudaMemcpyAsync(dst, src, bytes, k, s);
  };
  cudaError_t e = in(dom, omega, 8 * (size_t)n_omega);
  if (e == cudaSuccess && want_eps) {
    e = in(dr, d_r, 16 * (size_t)m);
    if (e == cudaSuccess) e = in(dl, d_l, 16 * (size_t)m);
  }
  if (e != cudaSuccess) {
    bse::record_error("cudaMemcpyAsync", e, __FILE__, __LINE__);
    rc = BSE_ERR_CUDA;
  }
  if (rc == BSE_OK && want_eps) rc = bse::weights(n, sol->X, m, dr, dl, dw, s);
  if (rc == BSE_OK)
    rc = bse::broaden(n, sol->lam, want_eps ? dw : nullptr, n_omega, dom, sigma, ddos, want_eps ? deps : nullptr, s);
  if (rc == BSE_OK) {
    e = out(dos, ddos, 8 * (size_t)n_omega);
    if (e == cudaSuccess && want_eps) e = out(eps, deps, 16 * (size_t)n_omega);
    if (e != cudaSuccess) {
      bse::record_error("cudaMemcpyAsync", e, __FILE__, __LINE__);
      rc = BSE_ERR_CUDA;
    }
  }
  cudaFreeAsync(buf, s);
  const cudaError_t se = cudaStreamSynchronize(s);
  if (rc == BSE_OK && se != cudaSuccess) {
    bse::record_error("cudaStreamSynchronize", se, __FILE__, __LINE__);
    rc = BSE_ERR_CUDA;
  }
  return rc;
}
