// FP64 structure-preserving refinement of the positive eigenpairs (mixed path).
//
// Pencil form (Theorem 2 and Eq. GMG): with u = Q^H x, H x = lambda x is
//   M u = lambda K u,   K = Q^H S Q = -i J  (Hermitian, involutory),
// and the Theorem 3 normalisation y^H x = 1 is u^H K u = 1. The eigenvectors
// of -lambda are conj(u) (M is real), so the full basis is V = [U, conj(U)]
// with V^H K V = diag(I, -I) and V^H M V = diag(Lambda, Lambda).
//
// One sweep is a first-order (Newton / Ogita-Aishima type) correction of the
// whole basis, written so that only the residual needs FP64 accuracy:
//   P  = M U                                  (FP64)
//   lambda_j = Re(u_j^H P_j) / Re(u_j^H K u_j)  (two-sided Rayleigh quotient)
//   R  = P - K U diag(lambda)                 (FP64; ||R_j|| / (||M||_F ||u_j||)
//                                              equals the scaled residual of H)
//   C1 = U^H R,  C2 = U^T R
//   E11_ij = C1_ij / (lambda_j - lambda_i)  (i != j),  E11_jj = (1 - u_j^H K u_j)/2
//   E21_ij = -C2_ij / (lambda_i + lambda_j)
//   U <- U + U E11 + conj(U) E21
// Only U is stored: the update of conj(U) is the conjugate of this one, so the
// +/- pairing and the left/right structure y = diag(I,-I) x stay exact.
// Pairs closer than the current error level are not divided by their gap
// (E11_ij = 0); the next sweep sees them again.
#include <float.h>
#include <string.h>

#include <utility>

#include "common.cuh"
#include "gemm_simt.cuh"
#include "internal.cuh"
#include "../../include/bse_stages.h"

namespace bse {

static inline size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

struct RefWork {
  double *Ur, *Ui, *Pr, *Pi, *Vr, *Vi;
  double *G1, *G2, *G3, *G4, *Fa, *Fb, *Fc, *Fd;
  double *lam_new, *bnorm, *scal;
  unsigned long long* maxes;  // [0] max resid, [1] max dlam (as ordered bit patterns)
};

size_t refine_worksize(int n) {
  const size_t m = 2 * (size_t)n;
  return 6 * al256(8 * m * n) + 8 * al256(8 * (size_t)n * n) + 2 * al256(8 * (size_t)n) + al256(64) + al256(64);
}

static RefWork carve_ref(void* work, int n) {
  const size_t m = 2 * (size_t)n;
  char* p = (char*)work;
  RefWork w;
  auto take = [&](size_t sz) {
    void* r = p;
    p += al256(sz);
    return r;
  };
  w.Ur = (double*)take(8 * m * n); w.Ui = (double*)take(8 * m * n);
  w.Pr = (double*)take(8 * m * n); w.Pi = (double*)take(8 * m * n);
  w.Vr = (double*)take(8 * m * n); w.Vi = (double*)take(8 * m * n);
  w.G1 = (double*)take(8 * (size_t)n * n); w.G2 = (double*)take(8 * (size_t)n * n);
  w.G3 = (double*)take(8 * (size_t)n * n); w.G4 = (double*)take(8 * (size_t)n * n);
  w.Fa = (double*)take(8 * (size_t)n * n); w.Fb = (double*)take(8 * (size_t)n * n);
  w.Fc = (double*)take(8 * (size_t)n * n); w.Fd = (double*)take(8 * (size_t)n * n);
  w.lam_new = (double*)take(8 * (size_t)n);
  w.bnorm = (double*)take(8 * (size_t)n);
  w.scal = (double*)take(64);
  w.maxes = (unsigned long long*)take(64);
  return w;
}

// u = Q^H x:  u_top = (x1 + x2)/sqrt2,  u_bot = i (x1 - x2)/sqrt2
__global__ void ref_x_to_u(int n, const double2* __restrict__ X, double* __restrict__ Ur, double* __restrict__ Ui) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= n) return;
  const long m = 2L * n, c = (long)j * m;
  const double2 x1 = X[i + c], x2 = X[n + i + c];
  const double h = 0.70710678118654752440;
  Ur[i + c] = (x1.x + x2.x) * h;
  Ui[i + c] = (x1.y + x2.y) * h;
  // i (a + ib) = -b + ia with a + ib = x1 - x2
  Ur[n + i + c] = -(x1.y - x2.y) * h;
  Ui[n + i + c] = (x1.x - x2.x) * h;
}

// x = Q u:  x1 = (u_top - i u_bot)/sqrt2,  x2 = (u_top + i u_bot)/sqrt2
__global__ void ref_u_to_x(int n, const double* __restrict__ Ur, const double* __restrict__ Ui, double2* __restrict__ X) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= n) return;
  const long m = 2L * n, c = (long)j * m;
  const double tr = Ur[i + c], ti = Ui[i + c], br = Ur[n + i + c], bi = Ui[n + i + c];
  const double h = 0.70710678118654752440;
  // -i (br + i bi) = bi - i br ;  i (br + i bi) = -bi + i br
  X[i + c] = make_double2((tr + bi) * h, (ti - br) * h);
  X[n + i + c] = make_double2((tr - bi) * h, (ti + br) * h);
}

__global__ void ref_frob(long count, const double* __restrict__ M, double* __restrict__ out) {
  __shared__ double red[8];
  double s = 0.0;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (long)gridDim.x * blockDim.x)
    s += M[i] * M[i];
  for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < 8; ++k) t += red[k];
    atomicAdd(out, t);
  }
}

__device__ __forceinline__ void atomic_max_pos(unsigned long long* p, double v) {
  atomicMax(p, (unsigned long long)__double_as_longlong(v));
}

__device__ __forceinline__ double block_sum256(double v, double* red) {
  for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  for (int k = 0; k < 8; ++k) t += red[k];
  return t;
}

// Per column: Rayleigh quotient, normalisation, residual R = P - K U lambda (in place in P).
__global__ void __launch_bounds__(256) ref_colstats(int n, const double* __restrict__ Ur, const double* __restrict__ Ui,
                                                    double* __restrict__ Pr, double* __restrict__ Pi,
                                                    const double* __restrict__ lam_old, double* __restrict__ lam_new,
                                                    double* __restrict__ bnorm, const double* __restrict__ scal,
                                                    unsigned long long* __restrict__ maxes) {
  __shared__ double red[8];
  const int j = blockIdx.x;
  const long m = 2L * n, c = (long)j * m;
  double a = 0.0, b = 0.0, nu = 0.0;
  for (int i = threadIdx.x; i < m; i += 256) {
    const double ur = Ur[i + c], ui = Ui[i + c];
    a += ur * Pr[i + c] + ui * Pi[i + c];
    nu += ur * ur + ui * ui;
    if (i < n) b += 2.0 * (ur * Ui[n + i + c] - ui * Ur[n + i + c]);
  }
  a = block_sum256(a, red);
  b = block_sum256(b, red);
  nu = block_sum256(nu, red);
  const double lam = a / b;
  double rr = 0.0;
  for (int i = threadIdx.x; i < m; i += 256) {
    double kr, ki;  // (K u)_i
    if (i < n) { kr = Ui[n + i + c]; ki = -Ur[n + i + c]; }
    else { kr = -Ui[i - n + c]; ki = Ur[i - n + c]; }
    const double r1 = Pr[i + c] - lam * kr, r2 = Pi[i + c] - lam * ki;
    Pr[i + c] = r1;
    Pi[i + c] = r2;
    rr += r1 * r1 + r2 * r2;
  }
  rr = block_sum256(rr, red);
  if (threadIdx.x == 0) {
    lam_new[j] = lam;
    bnorm[j] = b;
    const double res = sqrt(rr) / (scal[0] * sqrt(nu));
    const double dl = fabs(lam - lam_old[j]) / fabs(lam);
    atomic_max_pos(&maxes[0], res);
    atomic_max_pos(&maxes[1], dl);
  }
}

// E from C1 = U^H R, C2 = U^T R (given as G1 = Ur^T Rr, G2 = Ui^T Ri, G3 = Ur^T Ri, G4 = Ui^T Rr).
__global__ void ref_buildE(int n, const double* __restrict__ G1, const double* __restrict__ G2,
                           const double* __restrict__ G3, const double* __restrict__ G4,
                           const double* __restrict__ lam, const double* __restrict__ bnorm, double gap_tol,
                           double* __restrict__ Fa, double* __restrict__ Fb, double* __restrict__ Fc,
                           double* __restrict__ Fd) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= n) return;
  const long k = i + (long)j * n;
  const double g1 = G1[k], g2 = G2[k], g3 = G3[k], g4 = G4[k];
  const double c1r = g1 + g2, c1i = g3 - g4;
  const double c2r = g1 - g2, c2i = g3 + g4;
  const double li = lam[i], lj = lam[j];
  double e1r = 0.0, e1i = 0.0;
  if (i == j) {
    e1r = 0.5 * (1.0 - bnorm[j]);
  } else {
    const double d = lj - li;
    if (fabs(d) > gap_tol * fmax(fabs(li), fabs(lj))) {
      e1r = c1r / d;
      e1i = c1i / d;
    }
  }
  const double s = -1.0 / (li + lj);
  const double e2r = c2r * s, e2i = c2i * s;
  Fa[k] = e1r + e2r;
  Fb[k] = e2i - e1i;
  Fc[k] = e1i + e2i;
  Fd[k] = e1r - e2r;
}

int refine(int n, const double* M, double* lam, double* X, int max_sweeps, double tol, void* work, DevStatus* st,
           cudaStream_t s, int* sweeps_done, double* resid, double* dlam_last, double* dlam_first) {
  (void)st;
  const int m = 2 * n;
  RefWork w = carve_ref(work, n);
  const dim3 eg(ceil_div(n, 128), n);
  kcount(2);
  ref_x_to_u<<<eg, 128, 0, s>>>(n, reinterpret_cast<const double2*>(X), w.Ur, w.Ui);
  BSE_LAUNCH_CHECK();
  BSE_CUDA(cudaMemsetAsync(w.scal, 0, 64, s));
  ref_frob<<<1024, 256, 0, s>>>((long)m * m, M, w.scal);
  BSE_LAUNCH_CHECK();
  // scal[0] = ||M||_F
  double fro2 = 0.0;
  BSE_CUDA(cudaMemcpyAsync(&fro2, w.scal, 8, cudaMemcpyDeviceToHost, s));
  BSE_CUDA(cudaStreamSynchronize(s));
  const double fro = sqrt(fro2);
  BSE_CUDA(cudaMemcpyAsync(w.scal, &fro, 8, cudaMemcpyHostToDevice, s));
  const double res_target = tol > 0 ? tol : 4.0 * (double)n * DBL_EPSILON;
  int sweeps = 0;
  double res = 0, dl = 0;
  *dlam_first = 0;
  for (int it = 0;; ++it) {
    // P = M U
    BSE_TRY(gemm<double>(m, n, m, 1.0, M, m, false, w.Ur, m, false, 0.0, w.Pr, m, s));
    BSE_TRY(gemm<double>(m, n, m, 1.0, M, m, false, w.Ui, m, false, 0.0, w.Pi, m, s));
    BSE_CUDA(cudaMemsetAsync(w.maxes, 0, 16, s));
    kcount(1);
    ref_colstats<<<n, 256, 0, s>>>(n, w.Ur, w.Ui, w.Pr, w.Pi, lam, w.lam_new, w.bnorm, w.scal, w.maxes);
    BSE_LAUNCH_CHECK();
    unsigned long long hm[2];
    BSE_CUDA(cudaMemcpyAsync(hm, w.maxes, 16, cudaMemcpyDeviceToHost, s));
    BSE_CUDA(cudaMemcpyAsync(lam, w.lam_new, 8 * (size_t)n, cudaMemcpyDeviceToDevice, s));
    BSE_CUDA(cudaStreamSynchronize(s));
    memcpy(&res, &hm[0], 8);
    memcpy(&dl, &hm[1], 8);
    if (it == 0) *dlam_first = dl;
    const bool converged = (res <= res_target && (it > 0 && dl <= 1e-13));
    if (converged || it >= max_sweeps) break;
    // C1, C2 from four real products
    BSE_TRY(gemm<double>(n, n, m, 1.0, w.Ur, m, true, w.Pr, m, false, 0.0, w.G1, n, s));
    BSE_TRY(gemm<double>(n, n, m, 1.0, w.Ui, m, true, w.Pi, m, false, 0.0, w.G2, n, s));
    BSE_TRY(gemm<double>(n, n, m, 1.0, w.Ur, m, true, w.Pi, m, false, 0.0, w.G3, n, s));
    BSE_TRY(gemm<double>(n, n, m, 1.0, w.Ui, m, true, w.Pr, m, false, 0.0, w.G4, n, s));
    const double gap_tol = fmax(1e-14, 4.0 * dl);
    kcount(1);
    ref_buildE<<<eg, 128, 0, s>>>(n, w.G1, w.G2, w.G3, w.G4, lam, w.bnorm, gap_tol, w.Fa, w.Fb, w.Fc, w.Fd);
    BSE_LAUNCH_CHECK();
    // V = U + Ur [Fa Fc] + Ui [Fb Fd]
    BSE_CUDA(cudaMemcpyAsync(w.Vr, w.Ur, 8 * (size_t)m * n, cudaMemcpyDeviceToDevice, s));
    BSE_CUDA(cudaMemcpyAsync(w.Vi, w.Ui, 8 * (size_t)m * n, cudaMemcpyDeviceToDevice, s));
    BSE_TRY(gemm<double>(m, n, n, 1.0, w.Ur, m, false, w.Fa, n, false, 1.0, w.Vr, m, s));
    BSE_TRY(gemm<double>(m, n, n, 1.0, w.Ui, m, false, w.Fb, n, false, 1.0, w.Vr, m, s));
    BSE_TRY(gemm<double>(m, n, n, 1.0, w.Ur, m, false, w.Fc, n, false, 1.0, w.Vi, m, s));
    BSE_TRY(gemm<double>(m, n, n, 1.0, w.Ui, m, false, w.Fd, n, false, 1.0, w.Vi, m, s));
    std::swap(w.Ur, w.Vr);
    std::swap(w.Ui, w.Vi);
    ++sweeps;
  }
  kcount(1);
  ref_u_to_x<<<eg, 128, 0, s>>>(n, w.Ur, w.Ui, reinterpret_cast<double2*>(X));
  BSE_LAUNCH_CHECK();
  *sweeps_done = sweeps;
  *resid = res;
  *dlam_last = dl;
  return BSE_OK;
}

}  // namespace bse

extern "C" size_t bse_stage_refine_worksize(int n) { return bse::refine_worksize(n); }

extern "C" int bse_stage_refine(int n, const double* M, double* lam, double* X, int max_sweeps, void* work,
                                int* dev_status, void* stream, int* sweeps, double* diag3) {
  if (n < 1 || !M || !lam || !X || !work || !dev_status) return BSE_ERR_ARG;
  int sw = 0;
  double r = 0, d = 0, d0 = 0;
  int rc = bse::refine(n, M, lam, X, max_sweeps, 0.0, work, reinterpret_cast<bse::DevStatus*>(dev_status),
                       (cudaStream_t)stream, &sw, &r, &d, &d0);
  if (sweeps) *sweeps = sw;
  if (diag3) {
    diag3[0] = r;
    diag3[1] = d;
    diag3[2] = d0;
  }
  return rc;
}
