// Algorithm 3 step 2: positive spectral decomposition of Tsym = -i D^H T D.
//
// T is the skew tridiagonal from the reduction (sub-diagonal beta_k, super-
// diagonal -beta_k); with D = diag(i^k) (k = 0..m-1) Tsym is real symmetric
// tridiagonal with zero diagonal and off-diagonal alpha_k = -beta_k (remark 2).
// Its eigenvalues come in +/- pairs; the positive ones are lambda_1..lambda_n.
//
// Eigenvalues: bisection on the Sturm count of Tsym - sigma I (LDL^T pivots
// d_0 = -sigma, d_k = -sigma - alpha_{k-1}^2 / d_{k-1}), one thread per
// eigenvalue (the bisection of PDSTEBZ in the paper's implementation). For a
// zero-diagonal tridiagonal this determines every eigenvalue to high relative
// accuracy; iteration stops at a relative interval width of 2 eps.
//
// Eigenvectors: a twisted factorization per eigenvalue (forward and backward
// stationary LDL^T sweeps, twist index r = argmin |gamma_r|, then the two
// recurrences outward from z_r = 1), normalised. The D phase is folded in on
// output: the returned matrix is Vs[k][j] = s_k * v_k(lambda_j) with
// s_k = +1, +1, -1, -1 for k mod 4 = 0, 1, 2, 3, so that D V+ = Re + i Im with
// Re = the even rows of Vs and Im = the odd rows (used by the back-transform).
// Vs is ROW-major m x n (element (k, j) at k*n + j): thread j walks its own
// column and a warp touches 32 consecutive doubles per step.
#include <float.h>

#include <mutex>

#include "common.cuh"
#include "../../include/bse_stages.h"

namespace bse {

// e2[k] = beta_k^2; scal[0] = Gershgorin bound of Tsym, scal[1] = pivmin.
__global__ void __launch_bounds__(1024) tdeig_prep(int m, const double* __restrict__ e, double* __restrict__ e2,
                                                   double* __restrict__ scal) {
  __shared__ double smax[32], gmax[32];
  double mx = 0.0, gb = 0.0;
  for (int k = threadIdx.x; k < m - 1; k += blockDim.x) {
    const double b = e[k];
    e2[k] = b * b;
    mx = fmax(mx, b * b);
    const double left = (k > 0) ? fabs(e[k - 1]) : 0.0;
    gb = fmax(gb, fabs(b) + left);
    if (k == m - 2) gb = fmax(gb, fabs(b));
  }
  for (int o = 16; o >= 1; o >>= 1) {
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    gb = fmax(gb, __shfl_xor_sync(0xffffffffu, gb, o));
  }
  if ((threadIdx.x & 31) == 0) {
    smax[threadIdx.x >> 5] = mx;
    gmax[threadIdx.x >> 5] = gb;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, g = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a = fmax(a, smax[w]);
      g = fmax(g, gmax[w]);
    }
    scal[0] = g * (1.0 + 4.0 * DBL_EPSILON) + 4.0 * DBL_MIN;
    scal[1] = DBL_MIN * fmax(1.0, a);
  }
}

__device__ __forceinline__ int sturm_count(int m, const double* __restrict__ e2, double sigma, double pivmin) {
  double q = -sigma;
  if (fabs(q) < pivmin) q = -pivmin;
  int c = q < 0.0;
  for (int k = 1; k < m; ++k) {
    q = -sigma - e2[k - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    c += q < 0.0;
  }
  return c;
}

__global__ void __launch_bounds__(32) tdeig_bisect(int m, int n, const double* __restrict__ e2,
                                                   const double* __restrict__ scal, double* __restrict__ lam,
                                                   DevStatus* st) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int g = n + j;  // ascending index among all m eigenvalues
  const double pivmin = scal[1];
  double lo = 0.0, hi = scal[0];
  int it = 0;
  for (; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (hi - lo <= 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)) || mid <= lo || mid >= hi) break;
    if (sturm_count(m, e2, mid, pivmin) > g) hi = mid;
    else lo = mid;
  }
  if (it >= 200) set_status(st, BSE_ERR_NOT_CONVERGED, j + 1);
  lam[j] = 0.5 * (lo + hi);
}

__global__ void __launch_bounds__(32) tdeig_vectors(int m, int n, const double* __restrict__ e,
                                                    const double* __restrict__ scal,
                                                    const double* __restrict__ lam, double* __restrict__ Vs) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double pivmin = scal[1];
  const double l = lam[j];
  double* z = Vs + j;  // z[k * n]
  const long ld = n;
  // alpha_k = -e[k]; the recurrences below use alpha_k^2 and alpha_k / d.
  // forward: T - l I = L D L^T, store D
  double d = -l;
  if (fabs(d) < pivmin) d = -pivmin;
  z[0] = d;
  for (int k = 0; k < m - 1; ++k) {
    const double a = -e[k];
    double dn = -l - a * a / d;
    if (fabs(dn) < pivmin) dn = -pivmin;
    z[(long)(k + 1) * ld] = dn;
    d = dn;
  }
  // backward: T - l I = U R U^T; gamma_k = D_k + R_k + l (diagonal of T is 0)
  double rr = -l;
  if (fabs(rr) < pivmin) rr = -pivmin;
  int tw = m - 1;
  double gmin = fabs(z[(long)(m - 1) * ld] + rr + l);
  for (int k = m - 2; k >= 0; --k) {
    const double a = -e[k];
    double rn = -l - a * a / rr;
    if (fabs(rn) < pivmin) rn = -pivmin;
    rr = rn;
    const double gk = fabs(z[(long)k * ld] + rr + l);
    if (gk < gmin) {
      gmin = gk;
      tw = k;
    }
  }
  // recompute R_k for k > tw into z[k]
  rr = -l;
  if (fabs(rr) < pivmin) rr = -pivmin;
  for (int k = m - 1; k > tw; --k) {
    z[(long)k * ld] = rr;
    const double a = -e[k - 1];
    double rn = -l - a * a / rr;
    if (fabs(rn) < pivmin) rn = -pivmin;
    rr = rn;
  }
  // upward from the twist: z_{k+1} = -(alpha_k / R_{k+1}) z_k
  double zk = 1.0;
  double nrm = 1.0;
  for (int k = tw; k < m - 1; ++k) {
    const double a = -e[k];
    const double rk1 = z[(long)(k + 1) * ld];
    const double zn = -(a / rk1) * zk;
    z[(long)(k + 1) * ld] = zn;
    nrm += zn * zn;
    zk = zn;
  }
  // downward: z_k = -(alpha_k / D_k) z_{k+1}
  zk = 1.0;
  for (int k = tw - 1; k >= 0; --k) {
    const double a = -e[k];
    const double dk = z[(long)k * ld];
    const double zn = -(a / dk) * zk;
    z[(long)k * ld] = zn;
    nrm += zn * zn;
    zk = zn;
  }
  z[(long)tw * ld] = 1.0;
  const double inv = 1.0 / sqrt(nrm);
  for (int k = 0; k < m; ++k) {
    const double sgn = (k & 2) ? -inv : inv;
    z[(long)k * ld] *= sgn;
  }
}

int tdeig(int m, const double* e, double* lam, double* Vs, double* work, DevStatus* st, cudaStream_t s) {
  const int n = m / 2;
  double* e2 = work;
  double* scal = work + m;
  {
    KprofScope ks(K_ELEMENTWISE, s, 16.0 * m, 0.0);
    tdeig_prep<<<1, 1024, 0, s>>>(m, e, e2, scal);
  }
  BSE_LAUNCH_CHECK();
  {
    KprofScope ks(K_TDEIG_BISECT, s, 0.0, 0.0);
    tdeig_bisect<<<ceil_div(n, 32), 32, 0, s>>>(m, n, e2, scal, lam, st);
  }
  BSE_LAUNCH_CHECK();
  if (Vs) {
    KprofScope ks(K_TDEIG_VEC, s, 7.0 * 8.0 * m * n, 0.0);
    tdeig_vectors<<<ceil_div(n, 32), 32, 0, s>>>(m, n, e, scal, lam, Vs);
  }
  BSE_LAUNCH_CHECK();
  return BSE_OK;
}

}  // namespace bse

extern "C" size_t bse_stage_tdeig_worksize(int m) { return sizeof(double) * ((size_t)m + 8); }

// ---- allocation-free variant -------------------------------------------------
// The eigensolver's scratch (alpha^2 for every off-diagonal entry plus a few
// scalars) lives in a fixed array in the library's device image, so callers that
// must not allocate device memory can still run this stage. The array exists on
// every GPU that loads the library, until the process exits.
constexpr int kTdeigNoAllocMaxM = 65536;  // m <= 65536 (n <= 32768): 512 KiB of doubles
static __device__ __align__(256) double g_tdeig_scratch[kTdeigNoAllocMaxM + 8];

static std::mutex g_tdeig_scratch_mu;
static double* g_tdeig_scratch_dev[256];  // device address of the array, per device ordinal

// Device address of the static scratch on the current device. The host-side
// symbol is only a stand-in, so the address is looked up with
// cudaGetSymbolAddress once per device (with that device current) and cached.
static int tdeig_static_scratch(double** out) {
  int dev = -1;
  BSE_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) {
    bse::record_message("bse_stage_tdeig_noalloc: device ordinal out of range");
    return BSE_ERR_ARG;
  }
  std::lock_guard<std::mutex> lk(g_tdeig_scratch_mu);
  if (!g_tdeig_scratch_dev[dev]) {
    void* p = nullptr;
    cudaError_t err = cudaGetSymbolAddress(&p, g_tdeig_scratch);
    if (err != cudaSuccess || !p) {
      bse::record_error("cudaGetSymbolAddress(g_tdeig_scratch)", err, __FILE__, __LINE__);
      return BSE_ERR_CUDA;
    }
    g_tdeig_scratch_dev[dev] = static_cast<double*>(p);
  }
  *out = g_tdeig_scratch_dev[dev];
  return BSE_OK;
}

extern "C" int bse_stage_tdeig_noalloc(int m, const double* e, double* lam, double* Vs, int* dev_status,
                                       void* stream) {
  if (m < 2 || (m & 1) || !e || !lam || !dev_status) return BSE_ERR_ARG;
  if (m > kTdeigNoAllocMaxM) {
    bse::record_message("bse_stage_tdeig_noalloc: m exceeds 65536, the size of its static scratch");
    return BSE_ERR_ARG;
  }
  double* work = nullptr;
  BSE_TRY(tdeig_static_scratch(&work));
  // Every scratch value the kernels read is written earlier in the same call
  // (tdeig_prep fills alpha^2 and the scalars), so stale contents from a
  // previous call need no clearing.
  return bse::tdeig(m, e, lam, Vs, work, reinterpret_cast<bse::DevStatus*>(dev_status), (cudaStream_t)stream);
}

extern "C" int bse_stage_tdeig(int m, const double* e, double* lam, double* Vs, void* work, int* dev_status,
                               void* stream) {
  if (m < 2 || (m & 1) || !e || !lam || !work || !dev_status) return BSE_ERR_ARG;
  return bse::tdeig(m, e, lam, Vs, (double*)work, reinterpret_cast<bse::DevStatus*>(dev_status),
                    (cudaStream_t)stream);
}
