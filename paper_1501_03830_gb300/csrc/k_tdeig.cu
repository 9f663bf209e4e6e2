// Algorithm 3 step 2: positive spectral decomposition of Tsym = -i D^H T D.
//
// T is the skew tridiagonal from the reduction (sub-diagonal beta_k, super-
// diagonal -beta_k); with D = diag(i^k) (k = 0..m-1) Tsym is real symmetric
// tridiagonal with zero diagonal and off-diagonal alpha_k = -beta_k (remark 2).
// Its eigenvalues come in +/- pairs; the positive ones are lambda_1..lambda_n.
//
// Eigenvalues: bisection on the Sturm count of Tsym - sigma I (the number of
// sign changes among its leading principal minors), as PDSTEBZ does in the
// paper's implementation, here as multisection with a group of lanes per
// eigenvalue; iteration stops at a relative interval width of 2 eps.
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

// Number of eigenvalues of Tsym below sigma: sign changes of the leading
// principal minors p_k = det(T_k - sigma I), p_0 = 1, p_1 = -sigma,
// p_k = -sigma p_{k-1} - alpha_{k-2}^2 p_{k-2}. The product -alpha^2 p_{k-2} is
// ready one step early, so each step has a single FP64 FMA on its dependent
// path (FP64 latency is long on this GPU; an FP64 division, as in the ratio form
// p_k / p_{k-1}, is ~20x longer still); the sign tests run on the integer pipe
// from the bit patterns. A minor that vanishes exactly is replaced by 2^-900
// with the sign opposite to p_{k-1} (the ratio form's guard for a zero pivot:
// the ratio is taken as tiny and negative). Every 8 steps the pair
// (p_{k-1}, p_k) is rescaled by an exact power of two when it drifts out of
// [2^-480, 2^480], which changes no sign.
__device__ __forceinline__ void sturm_step(double ns, double e2k, double& p0, double& p1, int& c) {
  const double t = -e2k * p0;  // off the dependent path
  const double p2 = fma(ns, p1, t);
  long long b2 = __double_as_longlong(p2);
  const long long b1 = __double_as_longlong(p1);
  // an exactly zero minor becomes 2^-900 with the sign opposite to p_{k-1}
  // (integer select, no FP64 operation on the dependent path)
  b2 = ((b2 << 1) == 0) ? ((~b1 & (long long)0x8000000000000000ULL) | 0x07b0000000000000LL) : b2;
  c += (b2 ^ b1) < 0;
  p0 = p1;
  p1 = __longlong_as_double(b2);
}

__device__ __forceinline__ void sturm_rescale(double& p0, double& p1) {
  const int x0 = (int)((__double_as_longlong(p0) >> 52) & 0x7ff);
  const int x1 = (int)((__double_as_longlong(p1) >> 52) & 0x7ff);
  const int x = max(x0, x1);
  if (x > 1023 + 480) {
    p0 *= 0x1p-480;
    p1 *= 0x1p-480;
  } else if (x < 1023 - 480) {
    p0 *= 0x1p480;
    p1 *= 0x1p480;
  }
}

__device__ __forceinline__ int sturm_count(int m, const double* __restrict__ e2, double sigma, double pivmin) {
  const double ns = -sigma;
  double p0 = 1.0;  // p_{k-1}
  double p1 = ns;   // p_k
  if (fabs(p1) < pivmin) p1 = -pivmin;
  int c = p1 < 0.0;
  int k = 1;
  for (; k + 8 <= m; k += 8) {
    double ev[8];  // the block's couplings, loaded before the dependent chain starts
#pragma unroll
    for (int u = 0; u < 8; ++u) ev[u] = __ldg(e2 + k - 1 + u);
#pragma unroll
    for (int u = 0; u < 8; ++u) sturm_step(ns, ev[u], p0, p1, c);
    sturm_rescale(p0, p1);
  }
  for (; k < m; ++k) sturm_step(ns, e2[k - 1], p0, p1, c);
  return c;
}

// Multisection: a group of L lanes brackets one eigenvalue; each round the
// lanes count at L interior points splitting [lo, hi] into L+1 parts, and the
// part holding eigenvalue number g (the first point whose count exceeds g)
// becomes the new bracket: log2(L+1) bits per round instead of one, with L
// independent Sturm chains in flight to hide the FP64 latency. Every lane of
// a group takes the same decision from the group's ballot, so the bracket
// stays identical across the group without a broadcast. The loop ends at a
// relative width of 2 eps (or when the points can no longer split it).
template <int L>
__global__ void __launch_bounds__(256) tdeig_msect(int m, int n, const double* __restrict__ e2,
                                                   const double* __restrict__ scal, double* __restrict__ lam,
                                                   DevStatus* st) {
  static_assert(L == 4 || L == 8 || L == 16 || L == 32, "group size");
  const int lane = threadIdx.x & 31;
  const int gl = lane % L;       // lane within the group
  const int gshift = lane - gl;  // first lane of the group in the warp
  const int j = (int)(((long)blockIdx.x * blockDim.x + threadIdx.x) / L);
  const double pivmin = scal[1];
  const int g = n + j;  // ascending index among all m eigenvalues
  double lo = 0.0, hi = scal[0];
  bool done = j >= n;
  int rounds = 0;
  while (!__all_sync(0xffffffffu, done)) {
    const double h = (hi - lo) / (double)(L + 1);
    const double sigma = lo + (double)(gl + 1) * h;
    const int c = done ? 0 : sturm_count(m, e2, sigma, pivmin);
    const unsigned above = __ballot_sync(0xffffffffu, !done && c > g);
    const unsigned mask = (L == 32) ? above : ((above >> gshift) & ((1u << L) - 1u));
    if (!done) {
      // first point whose count exceeds g: the eigenvalue lies just below it
      const int first = mask ? __ffs(mask) - 1 : L;
      const double nlo = first == 0 ? lo : lo + (double)first * h;
      const double nhi = first == L ? hi : lo + (double)(first + 1) * h;
      lo = nlo;
      hi = fmax(nhi, nlo);
      if (hi - lo <= 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)) || h <= 0.0) done = true;
      if (++rounds >= 128 && !done) {
        set_status(st, BSE_ERR_NOT_CONVERGED, j + 1);
        done = true;
      }
    }
  }
  if (j < n && gl == 0) lam[j] = 0.5 * (lo + hi);
}

// Pivots of T - l I from minors: d_k = p_k / p_{k-1} with p the leading
// (forward) or trailing (backward) minors of the recurrence
// p_{k+1} = -l p_k - a_k^2 p_{k-1}. The minors carry the dependent chain (one
// FMA per step); the divisions that give the pivots depend on nothing later, so
// they overlap with the following steps instead of chaining (an FP64 division
// is ~0.5 us of latency here). The pair (p_{k-1}, p_k) is rescaled by exact
// powers of two every 8 steps, which leaves every ratio unchanged.
struct MinorPair {
  double p0, p1;  // p_{k-1}, p_k
};

__device__ __forceinline__ double guard_pivot(double d, double pivmin) { return fabs(d) < pivmin ? -pivmin : d; }

__device__ __forceinline__ void minor_rescale(MinorPair& q) {
  const int x0 = (int)((__double_as_longlong(q.p0) >> 52) & 0x7ff);
  const int x1 = (int)((__double_as_longlong(q.p1) >> 52) & 0x7ff);
  const int x = max(x0, x1);
  if (x > 1023 + 480) {
    q.p0 *= 0x1p-480;
    q.p1 *= 0x1p-480;
  } else if (x < 1023 - 480) {
    q.p0 *= 0x1p480;
    q.p1 *= 0x1p480;
  }
}

// p_next = -l p1 - a2 p0 with an exactly zero minor nudged off zero (sign
// opposite to p1), as in the Sturm count.
__device__ __forceinline__ double minor_next(double nl, double a2, const MinorPair& q) {
  const double p2 = fma(nl, q.p1, -a2 * q.p0);
  long long b2 = __double_as_longlong(p2);
  const long long b1 = __double_as_longlong(q.p1);
  b2 = ((b2 << 1) == 0) ? ((~b1 & (long long)0x8000000000000000ULL) | 0x07b0000000000000LL) : b2;
  return __longlong_as_double(b2);
}

__global__ void __launch_bounds__(32) tdeig_vectors(int m, int n, const double* __restrict__ e,
                                                    const double* __restrict__ scal,
                                                    const double* __restrict__ lam, double* __restrict__ Vs) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double pivmin = scal[1];
  const double l = lam[j];
  const double nl = -l;
  double* z = Vs + j;  // z[k * n]
  const long ld = n;
  // forward: D_k = p_k / p_{k-1} (leading minors, p_{-1} = 1, p_0 = -l), stored in z
  MinorPair f{1.0, nl};
  if ((__double_as_longlong(f.p1) << 1) == 0) f.p1 = -0x1p-900;
  z[0] = guard_pivot(f.p1 / f.p0, pivmin);
  for (int k = 0; k < m - 1; ++k) {
    const double a = e[k];
    const double p2 = minor_next(nl, a * a, f);
    f.p0 = f.p1;
    f.p1 = p2;
    z[(long)(k + 1) * ld] = guard_pivot(f.p1 / f.p0, pivmin);
    if ((k & 7) == 7) minor_rescale(f);
  }
  // backward: R_k = q_k / q_{k+1} (trailing minors); gamma_k = D_k + R_k + l
  MinorPair b{1.0, nl};
  if ((__double_as_longlong(b.p1) << 1) == 0) b.p1 = -0x1p-900;
  int tw = m - 1;
  double gmin = fabs(z[(long)(m - 1) * ld] + guard_pivot(b.p1 / b.p0, pivmin) + l);
  for (int k = m - 2; k >= 0; --k) {
    const double a = e[k];
    const double q2 = minor_next(nl, a * a, b);
    b.p0 = b.p1;
    b.p1 = q2;
    const double rk = guard_pivot(b.p1 / b.p0, pivmin);
    const double gk = fabs(z[(long)k * ld] + rk + l);
    if (gk < gmin) {
      gmin = gk;
      tw = k;
    }
    if (((m - 2 - k) & 7) == 7) minor_rescale(b);
  }
  // R_k for k > tw into z[k] (the same backward minors again)
  MinorPair r{1.0, nl};
  if ((__double_as_longlong(r.p1) << 1) == 0) r.p1 = -0x1p-900;
  for (int k = m - 1; k > tw; --k) {
    z[(long)k * ld] = guard_pivot(r.p1 / r.p0, pivmin);
    const double a = e[k - 1];
    const double q2 = minor_next(nl, a * a, r);
    r.p0 = r.p1;
    r.p1 = q2;
    if (((m - 1 - k) & 7) == 7) minor_rescale(r);
  }
  // upward from the twist: z_{k+1} = -(alpha_k / R_{k+1}) z_k (alpha_k = -e[k]);
  // the quotient is independent of z, only the product chains
  double zk = 1.0;
  double nrm = 1.0;
  for (int k = tw; k < m - 1; ++k) {
    const double c = e[k] / z[(long)(k + 1) * ld];
    const double zn = c * zk;
    z[(long)(k + 1) * ld] = zn;
    nrm = fma(zn, zn, nrm);
    zk = zn;
  }
  // downward: z_k = -(alpha_k / D_k) z_{k+1}
  zk = 1.0;
  for (int k = tw - 1; k >= 0; --k) {
    const double c = e[k] / z[(long)k * ld];
    const double zn = c * zk;
    z[(long)k * ld] = zn;
    nrm = fma(zn, zn, nrm);
    zk = zn;
  }
  z[(long)tw * ld] = 1.0;
  const double inv = 1.0 / sqrt(nrm);
  for (int k = 0; k < m; ++k) {
    const double sgn = (k & 2) ? -inv : inv;
    z[(long)k * ld] *= sgn;
  }
}

// The same vectors with two threads per eigenvalue (adjacent lanes): the forward
// pivots D_k (into Vs) and the backward pivots R_k (into Rb, an m x n scratch with
// Vs's layout) are independent chains, and so are the two recurrences outward
// from the twist, so each thread runs one of each; the twist index (argmin
// |gamma_k| over the two halves) and the norm are combined by a shuffle.
__global__ void __launch_bounds__(64) tdeig_vectors2(int m, int n, const double* __restrict__ e,
                                                     const double* __restrict__ scal, const double* __restrict__ lam,
                                                     double* __restrict__ Vs, double* __restrict__ Rb) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = t >> 1, role = t & 1;
  const bool live = j < n;
  const long ld = n;
  const double pivmin = scal[1];
  const double l = live ? lam[j] : 0.0;
  const double nl = -l;
  double* z = Vs + (live ? j : 0);
  double* r = Rb + (live ? j : 0);
  if (live) {
    if (role == 0) {
      // forward: D_k = p_k / p_{k-1} (leading minors, p_{-1} = 1, p_0 = -l)
      MinorPair f{1.0, nl};
      if ((__double_as_longlong(f.p1) << 1) == 0) f.p1 = -0x1p-900;
      z[0] = guard_pivot(f.p1 / f.p0, pivmin);
      for (int k = 0; k < m - 1; ++k) {
        const double a = e[k];
        const double p2 = minor_next(nl, a * a, f);
        f.p0 = f.p1;
        f.p1 = p2;
        z[(long)(k + 1) * ld] = guard_pivot(f.p1 / f.p0, pivmin);
        if ((k & 7) == 7) minor_rescale(f);
      }
    } else {
      // backward: R_k = q_k / q_{k+1} (trailing minors)
      MinorPair b{1.0, nl};
      if ((__double_as_longlong(b.p1) << 1) == 0) b.p1 = -0x1p-900;
      r[(long)(m - 1) * ld] = guard_pivot(b.p1 / b.p0, pivmin);
      for (int k = m - 2; k >= 0; --k) {
        const double a = e[k];
        const double q2 = minor_next(nl, a * a, b);
        b.p0 = b.p1;
        b.p1 = q2;
        r[(long)k * ld] = guard_pivot(b.p1 / b.p0, pivmin);
        if (((m - 2 - k) & 7) == 7) minor_rescale(b);
      }
    }
  }
  __syncwarp();
  // twist: gamma_k = D_k + R_k + l, smallest |gamma_k| (ties: the larger k)
  const int half = m / 2;
  double gmin = 1.7976931348623157e308;
  int tw = -1;
  if (live) {
    const int k0 = role == 0 ? 0 : half, k1 = role == 0 ? half : m;
    for (int k = k1 - 1; k >= k0; --k) {
      const double gk = fabs(z[(long)k * ld] + r[(long)k * ld] + l);
      if (gk < gmin) {
        gmin = gk;
        tw = k;
      }
    }
  }
  const double g_o = __shfl_xor_sync(0xffffffffu, gmin, 1);
  const int tw_o = __shfl_xor_sync(0xffffffffu, tw, 1);
  // the upper half (role 1) wins ties, as a scan from the bottom would
  if (role == 0 ? (g_o <= gmin) : (g_o < gmin)) tw = tw_o;
  __syncwarp();
  double nrm = 0.0;
  if (live) {
    if (role == 1) {
      // upward from the twist: z_{k+1} = -(alpha_k / R_{k+1}) z_k (alpha_k = -e[k])
      double zk = 1.0;
      for (int k = tw; k < m - 1; ++k) {
        const double c = e[k] / r[(long)(k + 1) * ld];
        const double zn = c * zk;
        z[(long)(k + 1) * ld] = zn;
        nrm = fma(zn, zn, nrm);
        zk = zn;
      }
    } else {
      // downward: z_k = -(alpha_k / D_k) z_{k+1}
      double zk = 1.0;
      nrm = 1.0;
      for (int k = tw - 1; k >= 0; --k) {
        const double c = e[k] / z[(long)k * ld];
        const double zn = c * zk;
        z[(long)k * ld] = zn;
        nrm = fma(zn, zn, nrm);
        zk = zn;
      }
    }
  }
  __syncwarp();
  nrm += __shfl_xor_sync(0xffffffffu, nrm, 1);
  if (!live) return;
  if (role == 0) z[(long)tw * ld] = 1.0;
  const double inv = 1.0 / sqrt(nrm);
  // each thread scales its part: role 0 rows <= tw, role 1 rows > tw
  const int k0 = role == 0 ? 0 : tw + 1, k1 = role == 0 ? tw + 1 : m;
  for (int k = k0; k < k1; ++k) {
    const double sgn = (k & 2) ? -inv : inv;
    z[(long)k * ld] *= sgn;
  }
}

// ---- reorthogonalization (remark 2) ----------------------------------------------
// Twisted-factorization vectors of close eigenvalues are orthogonal only to
// O(eps ||T|| / gap): at n = 8192 the closest pairs (relative gaps ~1e-6)
// keep |v_i^T v_j| ~ 1e-9. Remark 2 asks for reorthogonalization when high
// accuracy is wanted. Here a symmetric (Loewdin) step within a band of index
// distances does it without an order: G_ij = v_i^T v_j for 0 < |i - j| <= W,
// v_j <- v_j - 1/2 sum_i v_i G_ij, then unit norms; the eigenvalues sit in
// ascending order, so close eigenvalues are close in index. Twice, so that a
// larger defect is also taken to rounding level. Vs is row-major with the D
// signs folded into its rows, which leaves every inner product unchanged.
constexpr int kReorthW = 48;    // index distance covered
constexpr int kReorthCols = 32;  // columns per thread block

// Gband[j * W + q] = v_{j-1-q}^T v_j; column norms^2 in nrm2[j].
__global__ void __launch_bounds__(256) tdeig_reorth_gram(int m, int n, const double* __restrict__ Vs,
                                                         double* __restrict__ Gband, double* __restrict__ nrm2) {
  __shared__ double red[8][kReorthCols];
  const int j0 = blockIdx.x * kReorthCols;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  // lane = column j0 + lane; each warp takes rows wid, wid + 8, ...
  const int j = j0 + lane;
  double acc[kReorthW + 1];
#pragma unroll
  for (int q = 0; q <= kReorthW; ++q) acc[q] = 0.0;
  if (j < n) {
    for (int k = wid; k < m; k += 8) {
      const double* row = Vs + (long)k * n;
      const double vj = row[j];
#pragma unroll
      for (int q = 0; q <= kReorthW; ++q) {
        const int i = j - q;  // q = 0: the norm
        if (i >= 0) acc[q] = fma(row[i], vj, acc[q]);
      }
    }
  }
#pragma unroll
  for (int q = 0; q <= kReorthW; ++q) {
    red[wid][lane] = acc[q];
    __syncthreads();
    if (wid == 0 && j < n) {
      double t = 0.0;
      for (int w = 0; w < 8; ++w) t += red[w][lane];
      if (q == 0) nrm2[j] = t;
      else Gband[(long)j * kReorthW + (q - 1)] = (j - q >= 0) ? t : 0.0;
    }
    __syncthreads();
  }
}

// Vnew[k, j] = (v_j - 1/2 sum_{0 < |i-j| <= W} v_i G_ij)[k] / sqrt(G_jj) (first order)
__global__ void __launch_bounds__(256) tdeig_reorth_apply(int m, int n, const double* __restrict__ Vs,
                                                          const double* __restrict__ Gband,
                                                          const double* __restrict__ nrm2, double* __restrict__ Vo) {
  __shared__ double coef[kReorthCols][2 * kReorthW];
  const int j0 = blockIdx.x * kReorthCols;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int e = tid; e < kReorthCols * 2 * kReorthW; e += 256) {
    const int c = e / (2 * kReorthW), t = e % (2 * kReorthW);
    const int j = j0 + c;
    double g = 0.0;
    if (j < n) {
      if (t < kReorthW) {  // i = j - 1 - t
        if (j - 1 - t >= 0) g = Gband[(long)j * kReorthW + t];
      } else {  // i = j + 1 + (t - W): G_ij = Gband[i * W + (i - 1 - j)]
        const int q = t - kReorthW, i = j + 1 + q;
        if (i < n) g = Gband[(long)i * kReorthW + q];
      }
    }
    coef[c][t] = -0.5 * g;
  }
  __syncthreads();
  const int j = j0 + lane;
  if (j >= n) return;
  const double inv = rsqrt(nrm2[j]);
  for (int k = wid; k < m; k += 8) {
    const double* row = Vs + (long)k * n;
    double v = row[j];
#pragma unroll 8
    for (int t = 0; t < kReorthW; ++t) {
      const int i = j - 1 - t;
      if (i >= 0) v = fma(row[i], coef[lane][t], v);
      const int i2 = j + 1 + t;
      if (i2 < n) v = fma(row[i2], coef[lane][kReorthW + t], v);
    }
    Vo[(long)k * n + j] = v * inv;
  }
}

size_t tdeig_reorth_worksize(int m) {
  const size_t n = m / 2;
  return sizeof(double) * (n * kReorthW + n + (size_t)m * n) + 256;
}

// work: tdeig_reorth_worksize(m) bytes (band, norms and one m x n copy of Vs)
int tdeig_reorth(int m, double* Vs, void* work, cudaStream_t s) {
  const int n = m / 2;
  double* G = reinterpret_cast<double*>(work);
  double* nrm2 = G + (size_t)n * kReorthW;
  double* V2 = nrm2 + n;
  const int blocks = ceil_div(n, kReorthCols);
  for (int pass = 0; pass < 2; ++pass) {
    KprofScope ks(K_ELEMENTWISE, s, 16.0 * m * (double)n, 4.0 * kReorthW * (double)m * n);
    tdeig_reorth_gram<<<blocks, 256, 0, s>>>(m, n, Vs, G, nrm2);
    BSE_LAUNCH_CHECK();
    tdeig_reorth_apply<<<blocks, 256, 0, s>>>(m, n, Vs, G, nrm2, V2);
    BSE_LAUNCH_CHECK();
    BSE_CUDA(cudaMemcpyAsync(Vs, V2, sizeof(double) * (size_t)m * n, cudaMemcpyDeviceToDevice, s));
  }
  return BSE_OK;
}

int tdeig(int m, const double* e, double* lam, double* Vs, double* work, DevStatus* st, cudaStream_t s,
          double* vec_scratch) {
  const int n = m / 2;
  double* e2 = work;
  double* scal = work + m;
  {
    KprofScope ks(K_ELEMENTWISE, s, 16.0 * m, 0.0);
    tdeig_prep<<<1, 1024, 0, s>>>(m, e, e2, scal);
  }
  BSE_LAUNCH_CHECK();
  {
    // lanes per eigenvalue: enough independent Sturm chains to cover the GPU,
    // few enough not to waste FP64 throughput on large problems
    KprofScope ks(K_TDEIG_BISECT, s, 0.0, 0.0);
    // one warp per block (the kernel shares nothing across warps): the FP64 work
    // then spreads over every SM instead of n L / 256 blocks (128 of 152 SMs at
    // n = 8192)
    if (n >= 4096)
      tdeig_msect<4><<<ceil_div((long)n * 4, 32), 32, 0, s>>>(m, n, e2, scal, lam, st);
    else if (n >= 1024)
      tdeig_msect<16><<<ceil_div((long)n * 16, 32), 32, 0, s>>>(m, n, e2, scal, lam, st);
    else
      tdeig_msect<32><<<ceil_div((long)n * 32, 32), 32, 0, s>>>(m, n, e2, scal, lam, st);
  }
  BSE_LAUNCH_CHECK();
  if (Vs) {
    KprofScope ks(K_TDEIG_VEC, s, 7.0 * 8.0 * m * n, 0.0);
    if (vec_scratch)
      tdeig_vectors2<<<ceil_div(2L * n, 64), 64, 0, s>>>(m, n, e, scal, lam, Vs, vec_scratch);
    else
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
  return bse::tdeig(m, e, lam, Vs, work, reinterpret_cast<bse::DevStatus*>(dev_status), (cudaStream_t)stream,
                    nullptr);
}

extern "C" size_t bse_stage_tdeig_reorth_worksize(int m) { return m >= 2 ? bse::tdeig_reorth_worksize(m) : 0; }

extern "C" int bse_stage_tdeig_reorth(int m, double* Vs, void* work, void* stream) {
  if (m < 2 || (m & 1) || !Vs || !work) return BSE_ERR_ARG;
  return bse::tdeig_reorth(m, Vs, work, (cudaStream_t)stream);
}

extern "C" int bse_stage_tdeig(int m, const double* e, double* lam, double* Vs, void* work, int* dev_status,
                               void* stream) {
  if (m < 2 || (m & 1) || !e || !lam || !work || !dev_status) return BSE_ERR_ARG;
  return bse::tdeig(m, e, lam, Vs, (double*)work, reinterpret_cast<bse::DevStatus*>(dev_status),
                    (cudaStream_t)stream, nullptr);
}
