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
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <utility>
#include <vector>

#include "common.cuh"
#include "gemm_simt.cuh"
#include "tc32.cuh"
#include "internal.cuh"
#include "../../include/bse_stages.h"

namespace bse {

static inline size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

constexpr int kRRMax = 32;      // largest cluster re-solved by Rayleigh-Ritz
constexpr int kRRChunks = 8;    // row chunks of a cluster's Gram matrices and rotation (blocks per cluster)
constexpr int kBandW = 48;      // band biorthogonalization: index distance 1..kBandW
constexpr int kBandChunk = 16;  // couplings per thread block pass

struct RefWork {
  double *Ur, *Ui, *Pr, *Pi;          // FP64 U = Q^H X and P = M U (then R)
  float *Urf, *Uif, *Rrf, *Rif;       // FP32 copies for the projections
  float *dUr, *dUi;                   // FP32 correction U E11 + conj(U) E21
  float *G1, *G2, *G3, *G4, *Fa, *Fb, *Fc, *Fd;
  double *lam_new, *bnorm, *scal;
  unsigned long long* maxes;  // [0] max resid, [1] max dlam (as ordered bit patterns)
  int* cid;                   // cluster id per column
  int2* clus;                 // (first column, size) per cluster
  int* coff;                  // per cluster: first of its k^2 (a, b) pairs in rrpart / rrcoef
  double2* rrpart;            // [pair][kRRChunks][2]: partial U^H P and U^H K U over row chunks
  double2* rrcoef;            // [pair]: the cluster's rotation Cc (row-major k x k)
  void* oz;                   // digit-split tensor-core product workspace (M U)
  void* oz2;                  // same for the projections and the update
  double* Gbig;               // 2n x 2n: [Ur Ui]^T [Rr Ri]
  double2* Bband;             // n x kBandW couplings of the band biorthogonalization
};

// Bits carried by the FP64-accurate product M U (8-bit digits at m <= 16384, s
// digits carrying 8 s - 1 bits; M keeps 7 digits, so at most 55 bits). The first
// sweep starts from an FP32-level solution (scaled residual ~1e-8): 39 bits
// (5 digits) put the product's error four orders below what that sweep corrects.
// The second sweep's residual sets the couplings y_i^H x_j of the final basis,
// which come out as (product error) / gap: 50 bits (7 digits, 55 bits) --
// measured at n = 8192, 46 bits there raise the couplings of far pairs 50-100x
// (Table 1's biorthogonality 1e-12 -> 1e-10). The product of a third pass is
// normally the final check, which feeds the reported residual, the Rayleigh
// quotients and the rotations inside clusters; those rotations set the couplings
// of the closest pairs (relative gap 1.9e-6 at n = 8192), which 47 bits left at
// 2e-10 against 1e-12 at 49: 48 bits (7 digits, 55 bits) when that product is
// formed in full. It is normally formed as P + M dU instead (incremental_digits),
// which carries at least kSecondSweepBits of U with far fewer digit pairs.
#ifndef BSE_FIRST_SWEEP_BITS
#define BSE_FIRST_SWEEP_BITS 39
#endif
#ifndef BSE_SECOND_SWEEP_BITS
#define BSE_SECOND_SWEEP_BITS 50
#endif
#ifndef BSE_LATER_BITS
#define BSE_LATER_BITS 48
#endif
constexpr int kFirstSweepBits = BSE_FIRST_SWEEP_BITS;
constexpr int kSecondSweepBits = BSE_SECOND_SWEEP_BITS;
constexpr int kLaterBits = BSE_LATER_BITS;

// digits of the correction-sized products: ~25 bits
static int corr_digits(long m) { return ozaki_digits((int)m, 25); }

// The FP64-accurate M U runs on the tensor cores (digit splitting) from this order
// m = 2n on; below it the FP64 GEMM (measured on the 512-problem batch: with the
// tensor cores from m = 256 instead of 1024, 392 instead of 333 solves/s).
#ifndef BSE_REFINE_TC_MIN_M
#define BSE_REFINE_TC_MIN_M 256
#endif
static bool refine_uses_tc(int n) { return 2 * n >= BSE_REFINE_TC_MIN_M; }

// Digits of dU for the incremental product P + M dU (third and later passes):
// with r = max_j max_i |dU_ij| / max_i |U_ij|, s digits of dU (8 s - 1 bits of
// dU's column scale) carry 8 s - 1 + log2(1/r) bits of U's, so
// kSecondSweepBits relative to U (the accuracy asked of the second sweep's full
// product) need s = digits(kSecondSweepBits - floor(log2(1/r))). Returns 0 for a
// zero update and -1 (the full product) when dU is not small enough to save digits.
static int incremental_digits(long m, double r) {
  if (!(r >= 0.0)) return -1;
  if (r == 0.0) return 0;
  const int sd = ozaki_digits((int)m);
  const int lg = (int)floor(-log2(r));
  if (lg < 8) return -1;
  const int s = ozaki_digits((int)m, std::max(1, kSecondSweepBits - lg));
  return s < sd ? s : -1;
}

size_t refine_worksize(int n) {
  const size_t m = 2 * (size_t)n;
  size_t b = 2 * al256(16 * m * n) + 6 * al256(4 * m * n) + 8 * al256(4 * (size_t)n * n) + 2 * al256(8 * (size_t)n) +
             al256(64) + al256(64) + al256(4 * (size_t)n) + al256(8 * ((size_t)n / 2 + 2)) +
             al256(16 * (size_t)n * kBandW) + al256(4 * ((size_t)n / 2 + 2)) +
             al256(16 * 2 * kRRChunks * (size_t)kRRMax * n) + al256(16 * (size_t)kRRMax * n);
  if (refine_uses_tc(n)) {
    b += al256(ozaki_worksize((int)m, 2 * n, (int)m, ozaki_digits((int)m)));
    b += al256(ozaki_worksize(2 * n, 2 * n, (int)m, corr_digits(m)));
    b += al256(8 * (size_t)4 * n * n);
  }
  return b;
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
  // [Ur | Ui] and [Pr | Pi] are contiguous m x 2n blocks
  w.Ur = (double*)take(16 * m * n); w.Ui = w.Ur + m * n;
  w.Pr = (double*)take(16 * m * n); w.Pi = w.Pr + m * n;
  w.Urf = (float*)take(4 * m * n); w.Uif = (float*)take(4 * m * n);
  w.Rrf = (float*)take(8 * m * n); w.Rif = w.Rrf + m * n;  // [Rrf | Rif] contiguous
  w.dUr = (float*)take(8 * m * n); w.dUi = w.dUr + m * n;  // [dUr | dUi] contiguous
  w.G1 = (float*)take(4 * (size_t)n * n); w.G2 = (float*)take(4 * (size_t)n * n);
  w.G3 = (float*)take(4 * (size_t)n * n); w.G4 = (float*)take(4 * (size_t)n * n);
  w.Fa = (float*)take(4 * (size_t)n * n); w.Fb = (float*)take(4 * (size_t)n * n);
  w.Fc = (float*)take(4 * (size_t)n * n); w.Fd = (float*)take(4 * (size_t)n * n);
  w.lam_new = (double*)take(8 * (size_t)n);
  w.bnorm = (double*)take(8 * (size_t)n);
  w.scal = (double*)take(64);
  w.maxes = (unsigned long long*)take(64);
  w.cid = (int*)take(4 * (size_t)n);
  w.clus = (int2*)take(8 * ((size_t)n / 2 + 2));
  w.coff = (int*)take(4 * ((size_t)n / 2 + 2));
  // clusters hold <= kRRMax of the n columns each, so their k^2 pairs number <= kRRMax n
  w.rrpart = (double2*)take(16 * 2 * kRRChunks * (size_t)kRRMax * n);
  w.rrcoef = (double2*)take(16 * (size_t)kRRMax * n);
  w.Bband = (double2*)take(16 * (size_t)n * kBandW);
  w.oz = w.oz2 = nullptr;
  w.Gbig = nullptr;
  if (refine_uses_tc(n)) {
    w.oz = take(ozaki_worksize((int)m, 2 * n, (int)m, ozaki_digits((int)m)));
    w.oz2 = take(ozaki_worksize(2 * n, 2 * n, (int)m, corr_digits(m)));
    w.Gbig = (double*)take(8 * (size_t)4 * n * n);
  }
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

// Per column: Rayleigh quotient, normalisation, residual R = P - K U lambda (FP32 copy
// for the projections; its norm in FP64 for the convergence test).
__global__ void __launch_bounds__(256) ref_colstats(int n, const double* __restrict__ Ur, const double* __restrict__ Ui,
                                                    const double* __restrict__ Pr, const double* __restrict__ Pi,
                                                    float* __restrict__ Urf, float* __restrict__ Uif,
                                                    float* __restrict__ Rrf, float* __restrict__ Rif,
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
    const double r1 = Pr[i + c] - lam * kr, r2 = Pi[i + c] - lam * ki;  // P stays intact
    Rrf[i + c] = (float)r1;
    Rif[i + c] = (float)r2;
    Urf[i + c] = (float)Ur[i + c];
    Uif[i + c] = (float)Ui[i + c];
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

// u_j /= sqrt(b_j), b_j = u_j^H K u_j: exact Theorem 3 normalisation y_j^H x_j = 1.
__global__ void ref_normalize(int n, double* __restrict__ Ur, double* __restrict__ Ui,
                              const double* __restrict__ bnorm) {
  const int j = blockIdx.y;
  const long m = 2L * n, c = (long)j * m;
  const double s = rsqrt(bnorm[j]);
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (long)gridDim.x * blockDim.x) {
    Ur[i + c] *= s;
    Ui[i + c] *= s;
  }
}

// E from C1 = U^H R, C2 = U^T R (given as G1 = Ur^T Rr, G2 = Ui^T Ri, G3 = Ur^T Ri, G4 = Ui^T Rr).
__global__ void ref_buildE(int n, const float* __restrict__ G1, const float* __restrict__ G2,
                           const float* __restrict__ G3, const float* __restrict__ G4,
                           const double* __restrict__ lam, const double* __restrict__ bnorm,
                           const int* __restrict__ cluster_id,
                           float* __restrict__ Fa, float* __restrict__ Fb, float* __restrict__ Fc,
                           float* __restrict__ Fd) {
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
    // pairs inside one cluster were resolved exactly by its Rayleigh-Ritz step
    if (cluster_id[i] != cluster_id[j] && fabs(d) > 1e-14 * fmax(fabs(li), fabs(lj))) {
      e1r = c1r / d;
      e1i = c1i / d;
    }
  }
  const double s = -1.0 / (li + lj);
  const double e2r = c2r * s, e2i = c2i * s;
  Fa[k] = (float)(e1r + e2r);
  Fb[k] = (float)(e2i - e1i);
  Fc[k] = (float)(e1i + e2i);
  Fd[k] = (float)(e1r - e2r);
}

// E from G = [Ur Ui]^T [Rr Ri] (2n x 2n, FP64); writes the FP32 coefficient blocks
// Fa, Fb, Fc, Fd (n x n) of the update U <- U + U E11 + conj(U) E21.
__global__ void ref_buildE_big(int n, const double* __restrict__ G, const double* __restrict__ lam,
                               const double* __restrict__ bnorm, const int* __restrict__ cluster_id,
                               float* __restrict__ Fa, float* __restrict__ Fb, float* __restrict__ Fc,
                               float* __restrict__ Fd) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= n) return;
  const long ld = 2L * n;
  const double g1 = G[i + (long)j * ld], g3 = G[i + (long)(n + j) * ld];
  const double g4 = G[n + i + (long)j * ld], g2 = G[n + i + (long)(n + j) * ld];
  const double c1r = g1 + g2, c1i = g3 - g4;
  const double c2r = g1 - g2, c2i = g3 + g4;
  const double li = lam[i], lj = lam[j];
  double e1r = 0.0, e1i = 0.0;
  if (i == j) {
    e1r = 0.5 * (1.0 - bnorm[j]);
  } else {
    const double d = lj - li;
    if (cluster_id[i] != cluster_id[j] && fabs(d) > 1e-14 * fmax(fabs(li), fabs(lj))) {
      e1r = c1r / d;
      e1i = c1i / d;
    }
  }
  const double sc = -1.0 / (li + lj);
  const double e2r = c2r * sc, e2i = c2i * sc;
  const long k = i + (long)j * n;
  Fa[k] = (float)(e1r + e2r);
  Fb[k] = (float)(e2i - e1i);
  Fc[k] = (float)(e1i + e2i);
  Fd[k] = (float)(e1r - e2r);
}

// U += dU (FP64 += FP32 correction)
__global__ void ref_apply(long count, double* __restrict__ Ur, double* __restrict__ Ui, const float* __restrict__ dUr,
                          const float* __restrict__ dUi) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (long)gridDim.x * blockDim.x) {
    Ur[i] += (double)dUr[i];
    Ui[i] += (double)dUi[i];
  }
}

__device__ __forceinline__ double block_max256(double v, double* red) {
  for (int o = 16; o >= 1; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  for (int k = 0; k < 8; ++k) t = fmax(t, red[k]);
  return t;
}

// U += dU one column per block, and the update's size relative to the vector,
// max_i |dU_ij| / max_i |U_ij| (real and imaginary parts together), max over the
// columns into *ratio (ordered bit pattern): it sets how many digits of dU the next
// product M U = P + M dU needs (see incremental_digits).
__global__ void __launch_bounds__(256) ref_apply_cols(int n, double* __restrict__ Ur, double* __restrict__ Ui,
                                                      const float* __restrict__ dUr, const float* __restrict__ dUi,
                                                      unsigned long long* __restrict__ ratio) {
  __shared__ double red[8];
  const long m = 2L * n, c = (long)blockIdx.x * m;
  double du = 0.0, u = 0.0;
#pragma unroll 4
  for (long i = c + threadIdx.x; i < c + m; i += 256) {
    const double dr = (double)dUr[i], di = (double)dUi[i];
    const double ur = Ur[i] + dr, ui = Ui[i] + di;
    Ur[i] = ur;
    Ui[i] = ui;
    du = fmax(du, fmax(fabs(dr), fabs(di)));
    u = fmax(u, fmax(fabs(ur), fabs(ui)));
  }
  du = block_max256(du, red);
  u = block_max256(u, red);
  if (threadIdx.x == 0 && du > 0.0) atomic_max_pos(ratio, u > 0.0 ? du / u : 1.0);
}

// ---- cluster Rayleigh-Ritz ---------------------------------------------------
// For a run I of k <= kRRMax consecutive eigenvalues closer than the current
// error level, the first-order correction cannot separate the pair mixing, so
// the pencil is solved exactly on span(U_I) in FP64:
//   A_I = U_I^H M U_I = U_I^H P_I,  B_I = U_I^H K U_I,  A_I c = mu B_I c,
// with B_I = L L^H, C = L^{-1} A_I L^{-H} diagonalised by cyclic complex Jacobi,
// and U_I <- U_I Cc, P_I <- P_I Cc (P is linear in U), Cc = L^{-H} Z, so that
// Cc^H B_I Cc = I (the Theorem 3 normalisation) and the mu come out ascending.

struct cplx {
  double x, y;
};
__device__ __forceinline__ cplx cmk(double a, double b) { return {a, b}; }
__device__ __forceinline__ cplx cadd(cplx a, cplx b) { return {a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ cplx csub(cplx a, cplx b) { return {a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ cplx cmul(cplx a, cplx b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__device__ __forceinline__ cplx cconjmul(cplx a, cplx b) { return {a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x}; }
__device__ __forceinline__ cplx cconj(cplx a) { return {a.x, -a.y}; }
__device__ __forceinline__ cplx cscale(cplx a, double s) { return {a.x * s, a.y * s}; }

// The pencil's small matrices over the cluster's columns, in row chunks (one
// block per cluster and chunk, so a large cluster's FP64 work spreads over the
// GPU): partial A = U_I^H P_I and B = U_I^H K U_I over rows [i0, i1) of the top
// half and the matching rows of the bottom half. The chunk's k columns are staged
// in shared memory kRRRows rows at a time (coalesced loads); thread t sums pairs
// t, t + 256, ... (k^2 <= 1024).
constexpr int kRRRows = 16;

__global__ void __launch_bounds__(256) ref_rr_gram(int n, const int2* __restrict__ clusters,
                                                   const int* __restrict__ coff, const double* __restrict__ Ur,
                                                   const double* __restrict__ Ui, const double* __restrict__ Pr,
                                                   const double* __restrict__ Pi, double2* __restrict__ part) {
  __shared__ cplx ut_s[kRRMax][kRRRows], ub_s[kRRMax][kRRRows], pt_s[kRRMax][kRRRows], pb_s[kRRMax][kRRRows];
  const int2 cl = clusters[blockIdx.x];
  const int c0 = cl.x, k = cl.y;
  const int tid = threadIdx.x;
  const long m = 2L * n;
  const int R = (n + gridDim.y - 1) / gridDim.y;
  const int i0 = blockIdx.y * R, i1 = min(n, i0 + R);
  cplx sa[4], sb[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) sa[q] = sb[q] = cmk(0, 0);
  for (int ib = i0; ib < i1; ib += kRRRows) {
    for (int e = tid; e < k * kRRRows; e += blockDim.x) {
      const int a = e / kRRRows, r = e % kRRRows, i = ib + r;
      const long col = (long)(c0 + a) * m;
      const bool ok = i < i1;
      ut_s[a][r] = ok ? cmk(Ur[col + i], Ui[col + i]) : cmk(0, 0);
      ub_s[a][r] = ok ? cmk(Ur[col + n + i], Ui[col + n + i]) : cmk(0, 0);
      pt_s[a][r] = ok ? cmk(Pr[col + i], Pi[col + i]) : cmk(0, 0);
      pb_s[a][r] = ok ? cmk(Pr[col + n + i], Pi[col + n + i]) : cmk(0, 0);
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int pr = tid + 256 * q;
      if (pr < k * k) {
        const int a = pr % k, b = pr / k;
#pragma unroll 4
        for (int r = 0; r < kRRRows; ++r) {
          const cplx ut = ut_s[a][r], ub = ub_s[a][r], vt = ut_s[b][r], vb = ub_s[b][r];
          sa[q] = cadd(sa[q], cconjmul(ut, pt_s[b][r]));
          sa[q] = cadd(sa[q], cconjmul(ub, pb_s[b][r]));
          // (K u)_top = -i u_bot = (Ui_bot, -Ur_bot); (K u)_bot = i u_top = (-Ui_top, Ur_top)
          sb[q] = cadd(sb[q], cconjmul(ut, cmk(vb.y, -vb.x)));
          sb[q] = cadd(sb[q], cconjmul(ub, cmk(-vt.y, vt.x)));
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int pr = tid + 256 * q;
    if (pr < k * k) {
      double2* o = part + ((long)(coff[blockIdx.x] + pr) * gridDim.y + blockIdx.y) * 2;
      o[0] = make_double2(sa[q].x, sa[q].y);
      o[1] = make_double2(sb[q].x, sb[q].y);
    }
  }
}

// One block per cluster: the pencil A c = mu B c solved exactly (below), the
// eigenvalues written to lam_out and the rotation Cc to coef.
__global__ void __launch_bounds__(256) ref_rr_solve(int n, int nchunks, const int2* __restrict__ clusters,
                                                    const int* __restrict__ coff, const double2* __restrict__ part,
                                                    double2* __restrict__ coef, double* lam_out) {
  __shared__ cplx A[kRRMax][kRRMax + 1];
  __shared__ cplx Bm[kRRMax][kRRMax + 1];
  __shared__ cplx Z[kRRMax][kRRMax + 1];
  __shared__ double mu[kRRMax];
  __shared__ int order[kRRMax];
  __shared__ double rot[4];
  __shared__ double off;
  const int2 cl = clusters[blockIdx.x];
  const int c0 = cl.x, k = cl.y;
  const int tid = threadIdx.x;
  // 1. A = U^H P and B = U^H K U: the row chunks' partial sums, added in chunk order
  for (int pr = tid; pr < k * k; pr += blockDim.x) {
    const int a = pr % k, b = pr / k;
    const double2* p = part + (long)(coff[blockIdx.x] + pr) * nchunks * 2;
    cplx sa = cmk(0, 0), sb = cmk(0, 0);
    for (int ch = 0; ch < nchunks; ++ch) {
      sa = cadd(sa, cmk(p[2 * ch].x, p[2 * ch].y));
      sb = cadd(sb, cmk(p[2 * ch + 1].x, p[2 * ch + 1].y));
    }
    A[a][b] = sa;
    Bm[a][b] = sb;
  }
  __syncthreads();
  // exact Hermitian pencils from the lower halves
  for (int pr = tid; pr < k * k; pr += blockDim.x) {
    const int a = pr % k, b = pr / k;
    if (a > b) {
      const cplx x = cscale(cadd(A[a][b], cconj(A[b][a])), 0.5);
      const cplx y = cscale(cadd(Bm[a][b], cconj(Bm[b][a])), 0.5);
      A[a][b] = x;
      Bm[a][b] = y;
    }
  }
  __syncthreads();
  for (int pr = tid; pr < k * k; pr += blockDim.x) {
    const int a = pr % k, b = pr / k;
    if (a < b) {
      A[a][b] = cconj(A[b][a]);
      Bm[a][b] = cconj(Bm[b][a]);
    } else if (a == b) {
      A[a][a].y = 0.0;
      Bm[a][a].y = 0.0;
    }
  }
  __syncthreads();
  if (tid == 0) {
    // B = L L^H, L (lower) in Bm
    for (int j = 0; j < k; ++j) {
      double d = Bm[j][j].x;
      for (int t = 0; t < j; ++t) d -= Bm[j][t].x * Bm[j][t].x + Bm[j][t].y * Bm[j][t].y;
      d = sqrt(fmax(d, 1e-300));
      Bm[j][j] = cmk(d, 0.0);
      for (int i = j + 1; i < k; ++i) {
        cplx s2 = Bm[i][j];
        for (int t = 0; t < j; ++t) s2 = csub(s2, cmul(Bm[i][t], cconj(Bm[j][t])));
        Bm[i][j] = cscale(s2, 1.0 / d);
      }
    }
  }
  __syncthreads();
  // X = L^{-1} A, one column per thread, into Z
  if (tid < k) {
    const int col = tid;
    for (int i = 0; i < k; ++i) {
      cplx s2 = A[i][col];
      for (int t = 0; t < i; ++t) s2 = csub(s2, cmul(Bm[i][t], Z[t][col]));
      Z[i][col] = cscale(s2, 1.0 / Bm[i][i].x);
    }
  }
  __syncthreads();
  // C = X L^{-H}: row r of C solves L conj(C[r,:])^T = conj(X[r,:])^T; y = conj(C[r,:]) into A
  if (tid < k) {
    const int row = tid;
    for (int i = 0; i < k; ++i) {
      cplx s2 = cconj(Z[row][i]);
      for (int t = 0; t < i; ++t) s2 = csub(s2, cmul(Bm[i][t], A[row][t]));
      A[row][i] = cscale(s2, 1.0 / Bm[i][i].x);
    }
  }
  __syncthreads();
  for (int pr = tid; pr < k * k; pr += blockDim.x) {
    const int a = pr % k, b = pr / k;
    A[a][b] = cconj(A[a][b]);  // C[a][b]
  }
  __syncthreads();
  for (int pr = tid; pr < k * k; pr += blockDim.x) {
    const int a = pr % k, b = pr / k;
    if (a < b) A[a][b] = cconj(A[b][a]);
    if (a == b) A[a][a].y = 0.0;
    Z[a][b] = cmk(a == b ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  // cyclic Jacobi on the Hermitian C (in A), eigenvectors in Z
  for (int sweep = 0; sweep < 30; ++sweep) {
    if (tid == 0) {
      double o = 0.0, dg = 0.0;
      for (int a = 0; a < k; ++a)
        for (int b = 0; b < k; ++b) {
          const double v = A[a][b].x * A[a][b].x + A[a][b].y * A[a][b].y;
          if (a == b) dg += v;
          else o += v;
        }
      off = (o <= 1e-30 * dg) ? -1.0 : o;
    }
    __syncthreads();
    if (off < 0.0) break;
    for (int p = 0; p < k - 1; ++p)
      for (int q = p + 1; q < k; ++q) {
        if (tid == 0) {
          const cplx apq = A[p][q];
          const double r = sqrt(apq.x * apq.x + apq.y * apq.y);
          if (r < 1e-300) {
            rot[0] = 1.0; rot[1] = 0.0; rot[2] = 1.0; rot[3] = 0.0;
          } else {
            const double theta = (A[q][q].x - A[p][p].x) / (2.0 * r);
            const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
            const double c = 1.0 / sqrt(t * t + 1.0);
            rot[0] = c; rot[1] = t * c; rot[2] = apq.x / r; rot[3] = apq.y / r;  // e^{i phi}
          }
        }
        __syncthreads();
        const double c = rot[0], sn = rot[1];
        const cplx ph = cmk(rot[2], rot[3]);
        // similarity by G = diag(1, e^{-i phi}) * [[c, s], [-s, c]] on (p, q): columns ...
        if (tid < k) {
          const int r2 = tid;
          const cplx ap = A[r2][p], aq = cmul(A[r2][q], cconj(ph));
          A[r2][p] = csub(cscale(ap, c), cscale(aq, sn));
          A[r2][q] = cadd(cscale(ap, sn), cscale(aq, c));
          const cplx zp = Z[r2][p], zq = cmul(Z[r2][q], cconj(ph));
          Z[r2][p] = csub(cscale(zp, c), cscale(zq, sn));
          Z[r2][q] = cadd(cscale(zp, sn), cscale(zq, c));
        }
        __syncthreads();
        // ... and rows (G^H on the left)
        if (tid < k) {
          const int c2 = tid;
          const cplx ap = A[p][c2], aq = cmul(A[q][c2], ph);
          A[p][c2] = csub(cscale(ap, c), cscale(aq, sn));
          A[q][c2] = cadd(cscale(ap, sn), cscale(aq, c));
        }
        __syncthreads();
      }
  }
  if (tid == 0) {
    for (int a = 0; a < k; ++a) {
      mu[a] = A[a][a].x;
      order[a] = a;
    }
    for (int a = 0; a < k; ++a)
      for (int b = a + 1; b < k; ++b)
        if (mu[order[b]] < mu[order[a]]) {
          const int t = order[a]; order[a] = order[b]; order[b] = t;
        }
  }
  __syncthreads();
  // Cc = L^{-H} Z in ascending order, one column per thread, into Bm's upper part? -> into A
  if (tid < k) {
    const int col = order[tid];
    for (int i = k - 1; i >= 0; --i) {
      cplx s2 = Z[i][col];
      for (int t = i + 1; t < k; ++t) s2 = csub(s2, cmul(cconj(Bm[t][i]), A[t][tid]));
      A[i][tid] = cscale(s2, 1.0 / Bm[i][i].x);
    }
  }
  __syncthreads();
  if (tid < k) lam_out[c0 + tid] = mu[order[tid]];
  for (int pr = tid; pr < k * k; pr += blockDim.x) {
    const int a = pr / k, b = pr % k;  // Cc[a][b], row-major
    coef[coff[blockIdx.x] + pr] = make_double2(A[a][b].x, A[a][b].y);
  }
}

// U_I <- U_I Cc and P_I <- P_I Cc over rows of one chunk (one block per cluster
// and chunk): thread per row, the k new entries of the row summed in registers
// before any is stored (the update is in place).
__global__ void __launch_bounds__(256) ref_rr_apply(int n, const int2* __restrict__ clusters,
                                                    const int* __restrict__ coff, const double2* __restrict__ coef,
                                                    double* Ur, double* Ui, double* Pr, double* Pi) {
  __shared__ cplx C[kRRMax * kRRMax];
  const int2 cl = clusters[blockIdx.x];
  const int c0 = cl.x, k = cl.y;
  const long m = 2L * n;
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const double2 v = coef[coff[blockIdx.x] + e];
    C[e] = cmk(v.x, v.y);
  }
  __syncthreads();
  const long R = (m + gridDim.y - 1) / gridDim.y;
  const long i0 = blockIdx.y * R, i1 = min(m, i0 + R);
  for (long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
#pragma unroll 1
    for (int pass = 0; pass < 2; ++pass) {
      double* Xr = pass == 0 ? Ur : Pr;
      double* Xi = pass == 0 ? Ui : Pi;
      cplx acc[kRRMax];
#pragma unroll
      for (int b = 0; b < kRRMax; ++b) acc[b] = cmk(0, 0);
      for (int a = 0; a < k; ++a) {
        const cplx x = cmk(Xr[i + (long)(c0 + a) * m], Xi[i + (long)(c0 + a) * m]);
#pragma unroll
        for (int b = 0; b < kRRMax; ++b)
          if (b < k) acc[b] = cadd(acc[b], cmul(x, C[a * k + b]));
      }
#pragma unroll
      for (int b = 0; b < kRRMax; ++b)
        if (b < k) {
          Xr[i + (long)(c0 + b) * m] = acc[b].x;
          Xi[i + (long)(c0 + b) * m] = acc[b].y;
        }
    }
  }
}

// Cluster threshold of the final Rayleigh-Ritz polish (relative gap): 20x the
// first sweep's eigenvalue change, within [floor, cap].
#ifndef BSE_FINAL_TAU_FLOOR
#define BSE_FINAL_TAU_FLOOR 0.0
#endif
#ifndef BSE_FINAL_TAU_CAP
#define BSE_FINAL_TAU_CAP 1e-3
#endif
constexpr double kFinalTauFloor = BSE_FINAL_TAU_FLOOR;
constexpr double kFinalTauCap = BSE_FINAL_TAU_CAP;

// Runs of consecutive eigenvalues with relative gaps below tau, split to at most
// kRRMax at their widest internal gap; cluster_id[j] = first index of j's run.
// Rayleigh-Ritz on every cluster: partial Gram matrices over row chunks, the small
// pencils, the rotation of U and P (three launches). coff: host scratch for the
// clusters' pair offsets (kept by the caller until the stream has consumed it).
static int cluster_rr(int n, const std::vector<int2>& clusters, std::vector<int>& coff, RefWork& w, double* lam,
                      cudaStream_t s) {
  const int nc = (int)clusters.size();
  coff.resize(nc);
  int acc = 0;
  for (int c = 0; c < nc; ++c) {
    coff[c] = acc;
    acc += clusters[c].y * clusters[c].y;
  }
  BSE_CUDA(cudaMemcpyAsync(w.clus, clusters.data(), sizeof(int2) * nc, cudaMemcpyHostToDevice, s));
  BSE_CUDA(cudaMemcpyAsync(w.coff, coff.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, s));
  kcount(3);
  ref_rr_gram<<<dim3(nc, kRRChunks), 256, 0, s>>>(n, w.clus, w.coff, w.Ur, w.Ui, w.Pr, w.Pi, w.rrpart);
  BSE_LAUNCH_CHECK();
  ref_rr_solve<<<nc, 256, 0, s>>>(n, kRRChunks, w.clus, w.coff, w.rrpart, w.rrcoef, lam);
  BSE_LAUNCH_CHECK();
  ref_rr_apply<<<dim3(nc, kRRChunks), 256, 0, s>>>(n, w.clus, w.coff, w.rrcoef, w.Ur, w.Ui, w.Pr, w.Pi);
  BSE_LAUNCH_CHECK();
  return BSE_OK;
}

static void find_clusters(const std::vector<double>& lam, double tau, std::vector<int2>& out, std::vector<int>& id) {
  const int n = (int)lam.size();
  out.clear();
  id.resize(n);
  int a = 0;
  while (a < n) {
    int b = a + 1;
    while (b < n && (lam[b] - lam[b - 1]) <= tau * fabs(lam[b])) ++b;
    std::vector<std::pair<int, int>> stack{{a, b}};
    while (!stack.empty()) {
      const std::pair<int, int> xy = stack.back();
      stack.pop_back();
      const int x = xy.first, y = xy.second;
      if (y - x <= kRRMax) {
        for (int j = x; j < y; ++j) id[j] = x;
        if (y - x >= 2) out.push_back(make_int2(x, y - x));
        continue;
      }
      int cut = x + 1;
      double best = -1.0;
      for (int j = x + 1; j < y; ++j)
        if (lam[j] - lam[j - 1] > best) {
          best = lam[j] - lam[j - 1];
          cut = j;
        }
      stack.push_back({x, cut});
      stack.push_back({cut, y});
    }
    a = b;
  }
}

// ---- band biorthogonalization (end of the refinement) ------------------------
// After the sweeps the basis is biorthogonal to first order only: pairs of
// nearby eigenvalues keep a coupling b_ij = u_i^H K u_j (= y_i^H x_j, Theorem 3)
// of up to ~1e-9, which falls off with the index distance |i - j| (measured at
// n = 8192: ~1e-11 at distance 10, below 1e-12 beyond ~40). A symmetric
// (Loewdin) step U <- U (I - E/2), E = U^H K U - I restricted to the band
// 0 < |i - j| <= kBandW, removes it to second order without dividing by any gap;
// the diagonal of E is handled by the exact rescaling that follows. b_ij needs
// FP64 accumulation (it is a cancelling sum of O(1) terms); the update is as
// small as b_ij, so FP32 carries it.

// Bband[j * kBandW + q] = u_i^H K u_j for i = j - 1 - q (grid: n x kBandW / kBandChunk)
__global__ void __launch_bounds__(256) ref_band_gram(int n, const double* __restrict__ Ur,
                                                     const double* __restrict__ Ui, double2* __restrict__ Bband) {
  __shared__ double red[8][2 * kBandChunk];
  const int j = blockIdx.x, q0 = blockIdx.y * kBandChunk;
  const long m = 2L * n, cj = (long)j * m;
  const int nq = max(0, min(kBandChunk, j - q0));  // i = j-1-q >= 0
  double ar[kBandChunk], ai[kBandChunk];
#pragma unroll
  for (int q = 0; q < kBandChunk; ++q) ar[q] = ai[q] = 0.0;
  if (nq > 0) {
    for (int k = threadIdx.x; k < n; k += 256) {
      // K u_j: top = -i u_bot = (ub.y, -ub.x), bottom = i u_top = (-ut.y, ut.x)
      const double tr = Ur[k + cj], ti = Ui[k + cj], br = Ur[n + k + cj], bi = Ui[n + k + cj];
      const double ktr = bi, kti = -br, kbr = -ti, kbi = tr;
#pragma unroll
      for (int q = 0; q < kBandChunk; ++q) {
        if (q < nq) {
          const long ci = (long)(j - 1 - q0 - q) * m;
          const double xr = Ur[k + ci], xi = Ui[k + ci], yr = Ur[n + k + ci], yi = Ui[n + k + ci];
          // conj(x) * kt + conj(y) * kb
          ar[q] = fma(xr, ktr, fma(xi, kti, fma(yr, kbr, fma(yi, kbi, ar[q]))));
          ai[q] = fma(xr, kti, fma(-xi, ktr, fma(yr, kbi, fma(-yi, kbr, ai[q]))));
        }
      }
    }
  }
#pragma unroll
  for (int q = 0; q < kBandChunk; ++q) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
      ar[q] += __shfl_xor_sync(0xffffffffu, ar[q], o);
      ai[q] += __shfl_xor_sync(0xffffffffu, ai[q], o);
    }
  }
  const int wid = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int q = 0; q < kBandChunk; ++q) {
      red[wid][2 * q] = ar[q];
      red[wid][2 * q + 1] = ai[q];
    }
  }
  __syncthreads();
  if (threadIdx.x < kBandChunk) {
    const int q = threadIdx.x;
    double sr = 0.0, si = 0.0;
    for (int w = 0; w < 8; ++w) {
      sr += red[w][2 * q];
      si += red[w][2 * q + 1];
    }
    Bband[(long)j * kBandW + q0 + q] = (q < nq) ? make_double2(sr, si) : make_double2(0.0, 0.0);
  }
}

// dU_j = -1/2 sum_{0 < |i - j| <= kBandW} u_i b_ij (FP32), b_ij = conj(b_ji) for i > j.
__global__ void __launch_bounds__(256) ref_band_apply(int n, const float* __restrict__ Urf,
                                                      const float* __restrict__ Uif,
                                                      const double2* __restrict__ Bband, float* __restrict__ dUr,
                                                      float* __restrict__ dUi) {
  __shared__ float2 coef[2 * kBandW];
  __shared__ int col[2 * kBandW];
  const int j = blockIdx.y;
  const long m = 2L * n;
  if (threadIdx.x < 2 * kBandW) {
    const int t = threadIdx.x;
    int i;
    double2 b;
    if (t < kBandW) {  // i = j - 1 - t < j: stored as B[i, j]
      i = j - 1 - t;
      b = i >= 0 ? Bband[(long)j * kBandW + t] : make_double2(0.0, 0.0);
    } else {  // i = j + 1 + (t - kBandW) > j: b_ij = conj(B[j, i])
      const int q = t - kBandW;
      i = j + 1 + q;
      b = i < n ? Bband[(long)i * kBandW + q] : make_double2(0.0, 0.0);
      b.y = -b.y;
    }
    col[t] = (i >= 0 && i < n) ? i : j;
    coef[t] = (i >= 0 && i < n) ? make_float2((float)(-0.5 * b.x), (float)(-0.5 * b.y)) : make_float2(0.f, 0.f);
  }
  __syncthreads();
  for (long r = (long)blockIdx.x * blockDim.x + threadIdx.x; r < m; r += (long)gridDim.x * blockDim.x) {
    float sr = 0.f, si = 0.f;
#pragma unroll 8
    for (int t = 0; t < 2 * kBandW; ++t) {
      const long c = (long)col[t] * m + r;
      const float xr = Urf[c], xi = Uif[c];
      const float2 e = coef[t];
      sr = fmaf(xr, e.x, fmaf(-xi, e.y, sr));
      si = fmaf(xr, e.y, fmaf(xi, e.x, si));
    }
    dUr[r + (long)j * m] = sr;
    dUi[r + (long)j * m] = si;
  }
}

// Precision of the FP32 products of a sweep (projections U^H R, U^T R and the
// update U E): 3xTF32 on the tensor cores (FP32 level), or one TF32 pass where
// the sweep's own accuracy allows it.
#ifndef BSE_SWEEP0_ONEPASS
#define BSE_SWEEP0_ONEPASS 0
#endif
constexpr bool kSweep0OnePass = BSE_SWEEP0_ONEPASS != 0;

static int sweep_gemm(bool one_pass, int M, int N, int K, const float* A, long lda, bool ta, const float* B, long ldb,
                      bool tb, double beta, float* C, long ldc, cudaStream_t s) {
  if (one_pass && tc32::mode() >= 1) {
    GemmArgs g{};
    g.M = M; g.N = N; g.K = K;
    g.A = A; g.lda = lda; g.B = B; g.ldb = ldb; g.C = C; g.ldc = ldc;
    g.alpha = 1.0; g.beta = beta; g.transA = ta; g.transB = tb; g.batch = 1;
    if ((double)M * N * (double)K >= (double)(1 << 21) && tc32::eligible(g)) return tc32::gemm(g, 0, nullptr, s);
  }
  return gemm<float>(M, N, K, 1.0, A, lda, ta, B, ldb, tb, beta, C, ldc, s);
}

int refine(int n, const double* M, double* lam, double* X, int max_sweeps, double tol, void* work, DevStatus* st,
           cudaStream_t s, int* sweeps_done, double* resid, double* dlam_last, double* dlam_first) {
  StatusScope ss(st);
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
  static const bool verbose = getenv("BSE_REFINE_VERBOSE") != nullptr;
  int sweeps = 0;
  double res = 0, dl = 0, dl_level = 0;
  std::vector<double> hlam(n);
  std::vector<int2> clusters;
  std::vector<int> cid;
  std::vector<int> coff;  // pair offsets of the clusters (cluster_rr)
  double upd_ratio = 1.0;  // max over the columns of max |dU| / max |U| of the last update
  *dlam_first = 0;
  for (int it = 0;; ++it) {
    // P = M U, FP64-accurate: [Pr | Pi] = M [Ur | Ui]
    const int s_inc = it >= 2 ? incremental_digits(m, upd_ratio) : -1;
    if (s_inc == 0) {
      // the last update was zero: P = M U already
    } else if (refine_uses_tc(n) && s_inc > 0) {
      // P + M dU = M (U + dU) up to the FP64 rounding of U + dU (2^-53 of U): the
      // third and later products add the last update's product to the rotated P
      // of the sweep before (which kept P = M U), with dU's digits only as many as
      // its size below U leaves to carry
      OzOperand ma{M, m, false, false}, db{w.dUr, m, false, true};
      BSE_TRY(ozaki_gemm_ex(ma, db, m, 2 * n, m, w.Pr, m, ozaki_digits(m), true, w.oz, false,
                            reinterpret_cast<int*>(st), s, s_inc));
    } else if (refine_uses_tc(n)) {
      // M is symmetric, so its column-major storage is also its K-major row layout;
      // its digits are split once and reused by every sweep
      // bits of the product per sweep (see kFirstSweepBits): 39, then 50, then 48
      // (a later product is formed in full only when the update is too large for P + M dU)
      const int sd = ozaki_digits(m);
      const int bits = it == 0 ? kFirstSweepBits : (it == 1 ? kSecondSweepBits : kLaterBits);
      BSE_TRY(ozaki_gemm(m, 2 * n, m, M, m, w.Ur, m, w.Pr, m, sd, w.oz, it == 0, reinterpret_cast<int*>(st), s,
                         std::min(sd, ozaki_digits(m, bits))));
    } else {
      BSE_TRY(gemm<double>(m, n, m, 1.0, M, m, false, w.Ur, m, false, 0.0, w.Pr, m, s));
      BSE_TRY(gemm<double>(m, n, m, 1.0, M, m, false, w.Ui, m, false, 0.0, w.Pi, m, s));
    }
    BSE_CUDA(cudaMemsetAsync(w.maxes, 0, 16, s));
    kcount(1);
    ref_colstats<<<n, 256, 0, s>>>(n, w.Ur, w.Ui, w.Pr, w.Pi, w.Urf, w.Uif, w.Rrf, w.Rif, lam, w.lam_new, w.bnorm,
                                   w.scal, w.maxes);
    BSE_LAUNCH_CHECK();
    unsigned long long hm[2];
    BSE_CUDA(cudaMemcpyAsync(hm, w.maxes, 16, cudaMemcpyDeviceToHost, s));
    BSE_CUDA(cudaMemcpyAsync(lam, w.lam_new, 8 * (size_t)n, cudaMemcpyDeviceToDevice, s));
    BSE_CUDA(cudaStreamSynchronize(s));
    memcpy(&res, &hm[0], 8);
    memcpy(&dl, &hm[1], 8);
    if (it == 0) *dlam_first = dl;
    if (it == 0) dl_level = dl;
    if (verbose) fprintf(stderr, "[bse refine] n=%d sweep %d: max scaled residual %.3e, max rel dlambda %.3e\n", n, it, res, dl);
    // the Rayleigh quotient's error is second order in the vectors' error, so once
    // a sweep moves the eigenvalues by <= 1e-12 (relative) they are settled
    const bool converged = (res <= res_target && (it > 0 && dl <= 1e-12));
    if (converged || it >= max_sweeps) {
      // Final polish, no new M U. (1) Pairs closer than the first sweep's cluster
      // level are re-solved by Rayleigh-Ritz on the current (U, P). (2) The band
      // biorthogonalization removes the remaining couplings of nearby pairs
      // (invisible in the residual). (3) Every column is rescaled to y^H x = 1.
      BSE_CUDA(cudaMemcpyAsync(hlam.data(), lam, 8 * (size_t)n, cudaMemcpyDeviceToHost, s));
      BSE_CUDA(cudaStreamSynchronize(s));
      find_clusters(hlam, fmin(kFinalTauCap, fmax(kFinalTauFloor, fmax(1e-13, 20.0 * dl_level))), clusters, cid);
      BSE_CUDA(cudaMemcpyAsync(w.cid, cid.data(), 4 * (size_t)n, cudaMemcpyHostToDevice, s));
      if (!clusters.empty()) {
        BSE_TRY(cluster_rr(n, clusters, coff, w, lam, s));
      }
      BSE_CUDA(cudaMemsetAsync(w.maxes, 0, 16, s));
      kcount(1);
      ref_colstats<<<n, 256, 0, s>>>(n, w.Ur, w.Ui, w.Pr, w.Pi, w.Urf, w.Uif, w.Rrf, w.Rif, lam, w.lam_new, w.bnorm,
                                     w.scal, w.maxes);
      BSE_LAUNCH_CHECK();
      BSE_CUDA(cudaMemcpyAsync(lam, w.lam_new, 8 * (size_t)n, cudaMemcpyDeviceToDevice, s));
      BSE_CUDA(cudaMemcpyAsync(hm, w.maxes, 16, cudaMemcpyDeviceToHost, s));
      // band biorthogonalization from the U copies ref_colstats just wrote
      {
        double2* Bband = w.Bband;
        kcount(3);
        ref_band_gram<<<dim3(n, kBandW / kBandChunk), 256, 0, s>>>(n, w.Ur, w.Ui, Bband);
        BSE_LAUNCH_CHECK();
        ref_band_apply<<<dim3(ceil_div(m, 256 * 8), n), 256, 0, s>>>(n, w.Urf, w.Uif, Bband, w.dUr, w.dUi);
        BSE_LAUNCH_CHECK();
        ref_apply<<<1024, 256, 0, s>>>((long)m * n, w.Ur, w.Ui, w.dUr, w.dUi);
        BSE_LAUNCH_CHECK();
      }
      // bnorm of the corrected columns (the Rayleigh quotients it also writes are
      // not used: P is not updated by the correction)
      kcount(2);
      ref_colstats<<<n, 256, 0, s>>>(n, w.Ur, w.Ui, w.Pr, w.Pi, w.Urf, w.Uif, w.Rrf, w.Rif, lam, w.lam_new, w.bnorm,
                                     w.scal, w.maxes);
      BSE_LAUNCH_CHECK();
      ref_normalize<<<dim3(ceil_div(m, 256 * 4), n), 256, 0, s>>>(n, w.Ur, w.Ui, w.bnorm);
      BSE_LAUNCH_CHECK();
      // the host vectors must outlive the asynchronous uploads above
      BSE_CUDA(cudaStreamSynchronize(s));
      memcpy(&res, &hm[0], 8);
      if (verbose) fprintf(stderr, "[bse refine] n=%d final: %zu clusters, max scaled residual %.3e\n", n,
                           clusters.size(), res);
      break;
    }
    // clusters: runs closer than ~20x the current eigenvalue error level
    BSE_CUDA(cudaMemcpyAsync(hlam.data(), lam, 8 * (size_t)n, cudaMemcpyDeviceToHost, s));
    BSE_CUDA(cudaStreamSynchronize(s));
    const double tau = fmin(1e-3, fmax(1e-13, 20.0 * (it == 0 ? dl_level : dl)));
    find_clusters(hlam, tau, clusters, cid);
    BSE_CUDA(cudaMemcpyAsync(w.cid, cid.data(), 4 * (size_t)n, cudaMemcpyHostToDevice, s));
    if (!clusters.empty()) {
      BSE_TRY(cluster_rr(n, clusters, coff, w, lam, s));
      kcount(1);
      // statistics and FP32 copies again for the rotated columns
      BSE_CUDA(cudaMemsetAsync(w.maxes, 0, 16, s));
      ref_colstats<<<n, 256, 0, s>>>(n, w.Ur, w.Ui, w.Pr, w.Pi, w.Urf, w.Uif, w.Rrf, w.Rif, lam, w.lam_new, w.bnorm,
                                     w.scal, w.maxes);
      BSE_LAUNCH_CHECK();
      BSE_CUDA(cudaMemcpyAsync(lam, w.lam_new, 8 * (size_t)n, cudaMemcpyDeviceToDevice, s));
    }
    // the host vectors must outlive the asynchronous uploads above
    BSE_CUDA(cudaStreamSynchronize(s));
    if (verbose) {
      int kmax = 0, cols = 0, big = 0;
      for (const int2& c : clusters) {
        kmax = c.y > kmax ? c.y : kmax;
        cols += c.y;
        big += c.y >= 8;
      }
      fprintf(stderr, "[bse refine] n=%d sweep %d: %zu clusters (tau %.1e): %d columns, largest %d, %d of >= 8\n", n,
              it, clusters.size(), tau, cols, kmax, big);
    }
    if (refine_uses_tc(n) && !(tc32::mode() >= 1 && n % 2 == 0)) {
      // tensor cores: C1 = U^H R and C2 = U^T R from the one real 2n x 2n product
      // G = [Ur Ui]^T [Rr Ri]; each operand column (an eigenvector, a residual) has a
      // uniform scale, so ~25-bit digits carry these residual-sized products fully
      OzOperand ua{w.Ur, m, false, false}, rb{w.Rrf, m, false, true};
      BSE_TRY(ozaki_gemm_ex(ua, rb, 2 * n, 2 * n, m, w.Gbig, 2 * n, corr_digits(m), false, w.oz2, true,
                            reinterpret_cast<int*>(st), s));
      kcount(1);
      ref_buildE_big<<<eg, 128, 0, s>>>(n, w.Gbig, lam, w.bnorm, w.cid, w.Fa, w.Fb, w.Fc, w.Fd);
      BSE_LAUNCH_CHECK();
    } else {
      // C1 = U^H R, C2 = U^T R from four real FP32 products (R is residual-sized, so FP32
      // rounding of these products is eps32 relative to a quantity that is itself small);
      // with aligned operands they run on the 3xTF32 tensor-core kernel
      const bool op = kSweep0OnePass && it == 0;
      BSE_TRY(sweep_gemm(op, n, n, m, w.Urf, m, true, w.Rrf, m, false, 0.0, w.G1, n, s));
      BSE_TRY(sweep_gemm(op, n, n, m, w.Uif, m, true, w.Rif, m, false, 0.0, w.G2, n, s));
      BSE_TRY(sweep_gemm(op, n, n, m, w.Urf, m, true, w.Rif, m, false, 0.0, w.G3, n, s));
      BSE_TRY(sweep_gemm(op, n, n, m, w.Uif, m, true, w.Rrf, m, false, 0.0, w.G4, n, s));
      kcount(1);
      ref_buildE<<<eg, 128, 0, s>>>(n, w.G1, w.G2, w.G3, w.G4, lam, w.bnorm, w.cid, w.Fa, w.Fb, w.Fc, w.Fd);
      BSE_LAUNCH_CHECK();
    }
    // the update keeps FP32 entries (not column-scaled digits): a column of F mixes one
    // near-cluster coefficient with many tiny ones, and each of them needs its own bits
    // dU = Ur [Fa Fc] + Ui [Fb Fd] in FP32 (a correction of size |E|), then U += dU in FP64
    {
      const bool op = kSweep0OnePass && it == 0;
      BSE_TRY(sweep_gemm(op, m, n, n, w.Urf, m, false, w.Fa, n, false, 0.0, w.dUr, m, s));
      BSE_TRY(sweep_gemm(op, m, n, n, w.Uif, m, false, w.Fb, n, false, 1.0, w.dUr, m, s));
      BSE_TRY(sweep_gemm(op, m, n, n, w.Urf, m, false, w.Fc, n, false, 0.0, w.dUi, m, s));
      BSE_TRY(sweep_gemm(op, m, n, n, w.Uif, m, false, w.Fd, n, false, 1.0, w.dUi, m, s));
    }
    kcount(1);
    BSE_CUDA(cudaMemsetAsync(w.maxes + 2, 0, 8, s));
    ref_apply_cols<<<n, 256, 0, s>>>(n, w.Ur, w.Ui, w.dUr, w.dUi, w.maxes + 2);
    BSE_LAUNCH_CHECK();
    {
      unsigned long long rb = 0;
      BSE_CUDA(cudaMemcpyAsync(&rb, w.maxes + 2, 8, cudaMemcpyDeviceToHost, s));
      BSE_CUDA(cudaStreamSynchronize(s));
      memcpy(&upd_ratio, &rb, 8);
    }
    if (verbose)
      fprintf(stderr, "[bse refine] n=%d sweep %d: update max |dU|/|U| %.3e (next product: %d digits of dU)\n", n, it,
              upd_ratio, refine_uses_tc(n) && it + 1 >= 2 ? incremental_digits(m, upd_ratio) : -1);
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
