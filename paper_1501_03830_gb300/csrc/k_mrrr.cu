// Algorithm 3 step 2 with eigenvectors that are orthogonal without
// reorthogonalization: the representation tree of the MRRR method, which the
// paper's closing remarks of Section 3.3 name for the tridiagonal step (remark 2
// asks for reorthogonalization of the computed vectors when high accuracy is
// wanted; the tree makes that unnecessary). Dhillon and Parlett (Linear Algebra
// Appl. 387, 2004) give the method; the tree rules here are the oracle's.
//
//   root     T - sigma I = L D L^T, sigma below the Gershgorin interval (positive
//            definite, so a relatively robust representation)
//   values   multisection on the representation: the count of eigenvalues of
//            L D L^T below x is the number of negative pivots d+_i of the
//            stationary transform L D L^T - x I = L+ D+ L+^T. The transform is run
//            in a projective form without divisions: with s_i = p_i / q_i,
//              q_{i+1} = p_i + d_i q_i           (so d+_i = q_{i+1} / q_i)
//              p_{i+1} = d_i l_i^2 p_i - x q_{i+1}
//            which is s_{i+1} = d_i l_i^2 s_i / d+_i - x of the transform, one FMA
//            pair per step on the dependent chain (an FP64 division is a long
//            chain of its own on this GPU); (p, q) are rescaled by powers of two
//            every 8 steps, which changes no sign
//   tree     per level: runs of eigenvalues of one representation whose relative
//            gaps are below gaptol form clusters; a cluster gets a child
//            representation L D L^T - tau I by the stationary transform (with
//            divisions, as written) with tau just left of it; singletons (and
//            clusters at the depth limit) get their vectors at that level
//   vectors  twisted factorization of the representation shifted by the
//            eigenvalue (stationary transform from the top, progressive from the
//            bottom, twist r = argmin |gamma_r|, z_r = 1, the two recurrences
//            outward), three Rayleigh-quotient corrections gamma_r / |z|^2, then
//            the final vector, normalised
//
// One CUDA thread per eigenvalue for the sequential transforms, a group of
// kLanes lanes per eigenvalue for the counts; a host loop over the levels reads
// one counter per level (the number of new child representations).
#include <float.h>

#include "common.cuh"
#include "../../include/bse_stages.h"

namespace bse {
namespace mrrr {

constexpr double kEps = 2.220446049250313e-16;  // 2^-52
constexpr double kTiny = 0x1p-1000;             // an exactly zero pivot of the transforms becomes -kTiny
constexpr double kTinyQ = 0x1p-500;             // the same in the projective count (relative to q)
constexpr int kMaxDepth = 8;                    // levels for clusters of <= 1/gaptol members
constexpr int kMaxPeels = 64;                   // levels that peel a larger cluster
constexpr int kLanes = 8;                       // multisection lanes per eigenvalue

enum : int { S_DONE = 0, S_ACTIVE = 1, S_FINAL = 2 };

struct Node {
  double shift;  // the matrix's eigenvalues are this representation's plus shift
  double tau;    // shift of this representation from its parent's
  int parent, depth, peels, pad;
};

struct Work {
  double* rep[2];  // per level parity: [cap][2m] doubles, D (m) then l (m - 1)
  Node* meta[2];   // [cap]
  int* node[2];    // [nz] representation of each eigenvalue at the level
  int* state[2];   // [nz]
  double* lamloc;  // [nz] eigenvalue relative to its representation
  double* lo;      // [nz] bracket
  double* hi;      // [nz]
  int* nchild;     // [2] new child representations per level parity
  double* scal;    // [4] glo, ghi, sigma
};

static inline size_t al(size_t b) { return (b + 255) & ~(size_t)255; }
static inline int capacity(int nz) { return nz / 2 + 1; }  // clusters have >= 2 members

size_t worksize(int m, int nz) {
  const size_t cap = (size_t)capacity(nz);
  size_t b = 0;
  b += 2 * al(sizeof(double) * cap * 2 * (size_t)m);
  b += 2 * al(sizeof(Node) * cap);
  b += 4 * al(sizeof(int) * (size_t)nz);
  b += 3 * al(sizeof(double) * (size_t)nz);
  b += al(sizeof(int) * 2) + al(sizeof(double) * 4);
  return b;
}

static Work carve(void* w, int m, int nz) {
  const size_t cap = (size_t)capacity(nz);
  char* p = (char*)w;
  Work k;
  for (int i = 0; i < 2; ++i) {
    k.rep[i] = (double*)p;
    p += al(sizeof(double) * cap * 2 * (size_t)m);
  }
  for (int i = 0; i < 2; ++i) {
    k.meta[i] = (Node*)p;
    p += al(sizeof(Node) * cap);
  }
  for (int i = 0; i < 2; ++i) {
    k.node[i] = (int*)p;
    p += al(sizeof(int) * (size_t)nz);
  }
  for (int i = 0; i < 2; ++i) {
    k.state[i] = (int*)p;
    p += al(sizeof(int) * (size_t)nz);
  }
  k.lamloc = (double*)p; p += al(sizeof(double) * (size_t)nz);
  k.lo = (double*)p; p += al(sizeof(double) * (size_t)nz);
  k.hi = (double*)p; p += al(sizeof(double) * (size_t)nz);
  k.nchild = (int*)p; p += al(sizeof(int) * 2);
  k.scal = (double*)p;
  return k;
}

__device__ __forceinline__ double nz_pivot(double x) { return x != 0.0 ? x : -kTiny; }

// The tridiagonal's entries: diagonal a (zero when a is null) and off-diagonal b;
// in the BSE form the off-diagonal is -e (e: the sub-diagonal of the skew T, so
// that T_sym = -i D^H T D of remark 2 has off-diagonal alpha_k = -beta_k).
struct Tri {
  const double* a;
  const double* b;
  int bse;
  __device__ double diag(int i) const { return a ? a[i] : 0.0; }
  __device__ double off(int i) const { return bse ? -b[i] : b[i]; }
};

// Gershgorin interval (block reduction), then L D L^T = T - sigma I by one thread.
__global__ void __launch_bounds__(1024) mrrr_root(int m, Tri t, double* rep0, Node* meta0, double* scal) {
  __shared__ double slo[32], shi[32];
  double lo = DBL_MAX, hi = -DBL_MAX;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const double r = (i > 0 ? fabs(t.off(i - 1)) : 0.0) + (i < m - 1 ? fabs(t.off(i)) : 0.0);
    lo = fmin(lo, t.diag(i) - r);
    hi = fmax(hi, t.diag(i) + r);
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  if ((threadIdx.x & 31) == 0) {
    slo[threadIdx.x >> 5] = lo;
    shi[threadIdx.x >> 5] = hi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double glo = DBL_MAX, ghi = -DBL_MAX;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      glo = fmin(glo, slo[w]);
      ghi = fmax(ghi, shi[w]);
    }
    const double sigma = glo - 1e-3 * (ghi - glo) - 1e-300;
    double* D = rep0;
    double* l = rep0 + m;
    D[0] = t.diag(0) - sigma;
    for (int i = 0; i + 1 < m; ++i) {
      const double b = t.off(i);
      l[i] = b / D[i];
      D[i + 1] = t.diag(i + 1) - sigma - l[i] * b;
    }
    meta0[0] = Node{sigma, 0.0, -1, 0, 0, 0};
    scal[0] = glo;
    scal[1] = ghi;
    scal[2] = sigma;
  }
}

__global__ void mrrr_init(int nz, const double* scal, int* node, int* state, double* lo, double* hi) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nz) return;
  node[j] = 0;
  state[j] = S_ACTIVE;
  lo[j] = 0.0;
  hi[j] = (scal[1] - scal[2]) * (1.0 + 1e-12);
}

// Number of eigenvalues of L D L^T below x: the negative pivots of the
// stationary transform, in the projective form described at the top.
__device__ __forceinline__ int negcount(int m, const double* __restrict__ D, const double* __restrict__ l,
                                       double x) {
  double p = -x, q = 1.0;
  int c = 0;
  for (int i = 0; i + 1 < m; ++i) {
    const double di = __ldg(D + i), li = __ldg(l + i);
    const double cp = di * li * li * p;  // off the q chain
    double qn = fma(di, q, p);
    // d+_i = 0 exactly: -kTiny relative to q (negative pivot, as the transform does)
    if (qn == 0.0) qn = -kTinyQ * q;
    c += (__double_as_longlong(qn) ^ __double_as_longlong(q)) < 0;
    p = fma(-x, qn, cp);
    q = qn;
    if ((i & 7) == 7) {
      const int e = max((int)((__double_as_longlong(p) >> 52) & 0x7ff), (int)((__double_as_longlong(q) >> 52) & 0x7ff));
      if (e > 1023 + 400) {
        p *= 0x1p-400;
        q *= 0x1p-400;
      } else if (e < 1023 - 400) {
        p *= 0x1p400;
        q *= 0x1p400;
      }
    }
  }
  double qn = fma(__ldg(D + m - 1), q, p);
  if (qn == 0.0) qn = -kTinyQ * q;
  c += (__double_as_longlong(qn) ^ __double_as_longlong(q)) < 0;
  return c;
}

// Eigenvalue il + j of its representation, within [lo, hi], to a relative width of
// 4 eps (the oracle's bisection stopping rule): kLanes points per round split the
// bracket into kLanes + 1 parts and the part holding the eigenvalue is kept.
__global__ void __launch_bounds__(256) mrrr_bisect(int m, int nz, int il, const double* __restrict__ rep,
                                                   const int* __restrict__ node, const int* __restrict__ state,
                                                   const double* __restrict__ lo_in, const double* __restrict__ hi_in,
                                                   double* __restrict__ lamloc, DevStatus* st) {
  const int lane = threadIdx.x & 31;
  const int gl = lane % kLanes, gshift = lane - gl;
  const int j = (int)(((long)blockIdx.x * blockDim.x + threadIdx.x) / kLanes);
  bool done = j >= nz || state[j] != S_ACTIVE;
  const double* D = rep + (done ? 0 : (long)node[j] * 2 * m);
  const double* l = D + m;
  const int k = il + j;
  double lo = done ? 0.0 : lo_in[j], hi = done ? 0.0 : hi_in[j];
  if (!done && !(hi - lo > 4.0 * kEps * fmax(fabs(lo), fabs(hi)))) done = true;
  int rounds = 0;
  while (!__all_sync(0xffffffffu, done)) {
    const double h = (hi - lo) / (double)(kLanes + 1);
    const double x = lo + (double)(gl + 1) * h;
    const int c = done ? 0 : negcount(m, D, l, x);
    const unsigned above = __ballot_sync(0xffffffffu, !done && c > k);
    const unsigned mask = (above >> gshift) & ((1u << kLanes) - 1u);
    if (!done) {
      const int first = mask ? __ffs(mask) - 1 : kLanes;
      const double nlo = first == 0 ? lo : lo + (double)first * h;
      const double nhi = first == kLanes ? hi : lo + (double)(first + 1) * h;
      const bool stuck = (nlo == lo && nhi == hi);
      lo = nlo;
      hi = fmax(nhi, nlo);
      if (stuck || !(hi - lo > 4.0 * kEps * fmax(fabs(lo), fabs(hi)))) done = true;
      if (++rounds >= 160 && !done) {
        set_status(st, BSE_ERR_NOT_CONVERGED, j + 1);
        done = true;
      }
    }
  }
  if (j < nz && state[j] == S_ACTIVE && gl == 0) lamloc[j] = 0.5 * (lo + hi);
}

// One thread per eigenvalue: the first of each run of an active representation
// (a cluster head) decides the run's fate, as the oracle's tree does, and writes
// the next level's state of every member.
__global__ void mrrr_classify(int nz, double gaptol, const int* __restrict__ node, const int* __restrict__ state,
                              const double* __restrict__ lam, const Node* __restrict__ meta, int* node_next,
                              int* state_next, double* lo, double* hi, Node* meta_next, int* nchild_next) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nz) return;
  if (state[j] != S_ACTIVE) {
    state_next[j] = S_DONE;
    return;
  }
  const int nd = node[j];
  auto member = [&](int t) { return t >= 0 && t < nz && state[t] == S_ACTIVE && node[t] == nd; };
  auto joined = [&](int t) {  // t and t + 1 are in one cluster
    return member(t + 1) && (lam[t + 1] - lam[t]) < gaptol * fmax(fabs(lam[t]), fabs(lam[t + 1]));
  };
  const bool has_left = member(j - 1);
  if (has_left && joined(j - 1)) return;  // not the first of its run
  int e = j;
  while (joined(e)) ++e;
  const int size = e - j + 1;
  const bool large = (double)size * gaptol > 1.0;
  const Node pm = meta[nd];
  if (e == j || (pm.depth >= kMaxDepth && !large) || (large && pm.peels >= kMaxPeels)) {
    for (int t = j; t <= e; ++t) {
      state_next[t] = S_FINAL;
      node_next[t] = nd;
    }
    return;
  }
  // child representation just left of the cluster: a quarter of the gap to its
  // left neighbour or of its width away (for more than 1/gaptol members, at most a
  // quarter of mean gap / gaptol, so that the first ~1/gaptol of them separate)
  const double lj = lam[j], le = lam[e];
  const double left = has_left ? lam[j - 1] : lj - (le - lj) - fabs(lj) * 1e-3;
  const double width = le - lj;
  double off = fmin(lj - left, width + fabs(lj) * 1e-3);
  if (large) off = fmin(off, width / (double)(size - 1) / gaptol);
  const double tau = lj - fmax(0.25 * off, fabs(lj) * 8.0 * kEps);
  const int c = atomicAdd(nchild_next, 1);  // < nz / 2 + 1: clusters have >= 2 members
  meta_next[c] = Node{pm.shift + tau, tau, nd, large ? pm.depth : pm.depth + 1, large ? pm.peels + 1 : pm.peels, 0};
  const double lo_c = (lj - tau) * (1.0 - 1e-6);
  const double hi_c = (le - tau) * (1.0 + 1e-6) + fabs(le) * 4.0 * kEps;
  for (int t = j; t <= e; ++t) {
    state_next[t] = S_ACTIVE;
    node_next[t] = c;
    lo[t] = lo_c;
    hi[t] = hi_c;
  }
}

// Child representations by the stationary transform (as written, with divisions).
__global__ void mrrr_child(int m, const int* __restrict__ nchild, const Node* __restrict__ meta_next,
                           const double* __restrict__ rep_cur, double* __restrict__ rep_next) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= *nchild) return;
  const Node nd = meta_next[c];
  const double* D = rep_cur + (long)nd.parent * 2 * m;
  const double* l = D + m;
  double* Dc = rep_next + (long)c * 2 * m;
  double* lc = Dc + m;
  const double tau = nd.tau;
  double s = -tau;
  for (int i = 0; i + 1 < m; ++i) {
    const double dp = nz_pivot(s + D[i]);
    const double lp = D[i] * l[i] / dp;
    Dc[i] = dp;
    lc[i] = lp;
    s = lp * l[i] * s - tau;
  }
  Dc[m - 1] = nz_pivot(s + D[m - 1]);
}

// Twisted factorization of L D L^T - lam I into the column z (stride ld): z_r = 1,
// returns gamma_r and |z|^2.
__device__ void twisted(int m, const double* __restrict__ D, const double* __restrict__ l, double lam, double* z,
                        long ld, double* gamma_r, double* nrm2) {
  // stationary transform from the top: s_i into z[i]
  double s = -lam;
  for (int i = 0; i + 1 < m; ++i) {
    z[(long)i * ld] = s;
    const double dp = nz_pivot(s + D[i]);
    s = (D[i] * l[i] / dp) * l[i] * s - lam;
  }
  z[(long)(m - 1) * ld] = s;
  // progressive transform from the bottom; gamma_i = s_i + p_i + lam
  double p = D[m - 1] - lam;
  int r = m - 1;
  double g = z[(long)(m - 1) * ld] + p + lam;
  double best = fabs(g);
  for (int i = m - 2; i >= 0; --i) {
    const double dm = nz_pivot(D[i] * l[i] * l[i] + p);
    p = p * (D[i] / dm) - lam;
    const double gi = z[(long)i * ld] + p + lam;
    if (fabs(gi) <= best) {  // the first index of the smallest |gamma|, as argmin takes
      best = fabs(gi);
      g = gi;
      r = i;
    }
  }
  // u_i (i >= r) into z[i + 1], from the bottom again
  p = D[m - 1] - lam;
  for (int i = m - 2; i >= r; --i) {
    const double dm = nz_pivot(D[i] * l[i] * l[i] + p);
    const double t = D[i] / dm;
    z[(long)(i + 1) * ld] = l[i] * t;
    p = p * t - lam;
  }
  // l+_i (i < r) into z[i], from the top again
  s = -lam;
  for (int i = 0; i < r; ++i) {
    const double dp = nz_pivot(s + D[i]);
    const double lp = D[i] * l[i] / dp;
    z[(long)i * ld] = lp;
    s = lp * l[i] * s - lam;
  }
  // z_r = 1 and the two recurrences outward
  double nrm = 1.0, zk = 1.0;
  for (int i = r - 1; i >= 0; --i) {
    zk = -z[(long)i * ld] * zk;
    z[(long)i * ld] = zk;
    nrm = fma(zk, zk, nrm);
  }
  zk = 1.0;
  for (int i = r; i + 1 < m; ++i) {
    zk = -z[(long)(i + 1) * ld] * zk;
    z[(long)(i + 1) * ld] = zk;
    nrm = fma(zk, zk, nrm);
  }
  z[(long)r * ld] = 1.0;
  *gamma_r = g;
  *nrm2 = nrm;
}

__global__ void __launch_bounds__(32) mrrr_vectors(int m, int nz, const double* __restrict__ rep,
                                                   const int* __restrict__ node, const Node* __restrict__ meta,
                                                   int* state_next, const double* __restrict__ lamloc,
                                                   double* __restrict__ lam_out, double* __restrict__ Z, long ldz,
                                                   int bse_signs) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nz || state_next[j] != S_FINAL) return;
  const int nd = node[j];
  const double* D = rep + (long)nd * 2 * m;
  const double* l = D + m;
  double* z = Z + j;
  double lam = lamloc[j], g = 0.0, nrm2 = 1.0;
  for (int it = 0; it < 3; ++it) {
    twisted(m, D, l, lam, z, ldz, &g, &nrm2);
    lam += g / nrm2;
  }
  twisted(m, D, l, lam, z, ldz, &g, &nrm2);
  const double inv = 1.0 / sqrt(nrm2);
  for (int k = 0; k < m; ++k) {
    // BSE form: the D phase of remark 2 folded in (s_k = +1, +1, -1, -1 for k mod 4)
    const double sgn = (bse_signs && (k & 2)) ? -inv : inv;
    z[(long)k * ldz] *= sgn;
  }
  lam_out[j] = lam + meta[nd].shift;
  state_next[j] = S_DONE;
}

}  // namespace mrrr

// Eigenpairs il .. iu-1 (ascending) of the symmetric tridiagonal T (diagonal a,
// or zeros when a is null; off-diagonal b, or -b when bse_form) by the
// representation tree. Z: row-major m x ldz, column j = eigenvector il + j.
int tdeig_mrrr(int m, const double* a, const double* b, int bse_form, int il, int iu, double gaptol, double* lam,
               double* Z, long ldz, int bse_signs, void* work, DevStatus* st, cudaStream_t s) {
  using namespace mrrr;
  const int nz = iu - il;
  if (nz <= 0) return BSE_OK;
  Work w = carve(work, m, nz);
  const Tri t{a, b, bse_form};
  const int cap = capacity(nz);
  {
    KprofScope ks(K_TDEIG_BISECT, s, 0.0, 0.0);
    mrrr_root<<<1, 1024, 0, s>>>(m, t, w.rep[0], w.meta[0], w.scal);
    BSE_LAUNCH_CHECK();
    mrrr_init<<<ceil_div(nz, 256), 256, 0, s>>>(nz, w.scal, w.node[0], w.state[0], w.lo, w.hi);
    BSE_LAUNCH_CHECK();
  }
  for (int d = 0; d < kMaxDepth + kMaxPeels + 2; ++d) {
    const int cur = d & 1, nxt = cur ^ 1;
    {
      KprofScope ks(K_TDEIG_BISECT, s, 0.0, 0.0);
      mrrr_bisect<<<ceil_div((long)nz * kLanes, 256), 256, 0, s>>>(m, nz, il, w.rep[cur], w.node[cur], w.state[cur],
                                                                    w.lo, w.hi, w.lamloc, st);
      BSE_LAUNCH_CHECK();
      BSE_CUDA(cudaMemsetAsync(w.nchild + nxt, 0, sizeof(int), s));
      mrrr_classify<<<ceil_div(nz, 256), 256, 0, s>>>(nz, gaptol, w.node[cur], w.state[cur], w.lamloc, w.meta[cur],
                                                      w.node[nxt], w.state[nxt], w.lo, w.hi, w.meta[nxt],
                                                      w.nchild + nxt);
      BSE_LAUNCH_CHECK();
    }
    {
      KprofScope ks(K_TDEIG_VEC, s, 0.0, 0.0);
      mrrr_vectors<<<ceil_div(nz, 32), 32, 0, s>>>(m, nz, w.rep[cur], w.node[cur], w.meta[cur], w.state[nxt],
                                                    w.lamloc, lam, Z, ldz, bse_signs);
      BSE_LAUNCH_CHECK();
    }
    {
      KprofScope ks(K_TDEIG_BISECT, s, 0.0, 0.0);
      mrrr_child<<<ceil_div(cap, 32), 32, 0, s>>>(m, w.nchild + nxt, w.meta[nxt], w.rep[cur], w.rep[nxt]);
      BSE_LAUNCH_CHECK();
    }
    int more = 0;
    BSE_CUDA(cudaMemcpyAsync(&more, w.nchild + nxt, sizeof(int), cudaMemcpyDeviceToHost, s));
    BSE_CUDA(cudaStreamSynchronize(s));
    if (more == 0) break;
  }
  return BSE_OK;
}

size_t tdeig_mrrr_worksize(int m, int nz) { return mrrr::worksize(m, nz); }

}  // namespace bse

extern "C" size_t bse_stage_tdeig_mrrr_worksize(int m, int il, int iu) {
  if (m < 1 || il < 0 || iu > m || iu <= il) return 0;
  return bse::tdeig_mrrr_worksize(m, iu - il);
}

extern "C" int bse_stage_tdeig_mrrr(int m, const double* a, const double* b, int bse_form, int il, int iu,
                                    double gaptol, double* lam, double* Z, int ldz, int bse_signs, void* work,
                                    int* dev_status, void* stream) {
  if (m < 1 || (!b && m > 1) || il < 0 || iu > m || iu <= il || !lam || !Z || ldz < iu - il || !work || !dev_status)
    return BSE_ERR_ARG;
  if (!(gaptol > 0.0 && gaptol < 1.0)) gaptol = 1e-3;
  return bse::tdeig_mrrr(m, a, b, bse_form, il, iu, gaptol, lam, Z, ldz, bse_signs, work,
                         reinterpret_cast<bse::DevStatus*>(dev_status), (cudaStream_t)stream);
}
