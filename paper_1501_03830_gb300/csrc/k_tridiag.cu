// Algorithm 3 step 1: W = U T U^T, skew-symmetric Householder tridiagonalization
// (Section 3.3, remark 1: a modified symmetric tridiagonal reduction with
// skew-symmetric level-2/level-3 kernels), blocked by NB = 64 columns.
//
// Column j (trailing matrix A_j = rows/cols j+1..m-1, skew):
//   w   = column j of A_j              (pending panel updates applied: K1)
//   H_j = I - tau v v^T, H_j w = beta e_1   (dlarfg convention: K2)
//   p   = tau A_j v                    (skew SYMV on the stored lower triangle
//                                       of the panel-start matrix A0: K3, plus
//                                       the panel's V (P^T v) - P (V^T v): K4)
//   A_{j+1} = H_j A_j H_j = A_j + v p^T - p v^T
// (for skew A, v^T A v = 0, so the symmetric algorithm's correction term
// vanishes). After NB columns the trailing lower triangle gets the rank-2NB
// update A0 <- A0 + V P^T - P V^T (a GEMM).
//
// Outputs: beta_j (the sub-diagonal T[j+1, j]) in e[j], tau_j in tau[j], and
// v_j in W[j+1:m, j] (with the explicit leading 1), j = 0..m-2.
//
// K3 is the HBM-bound kernel. One warp processes 32x32 sub-tiles of one
// 32-row strip: lane l owns row r; the direct product sum_c A[r,c] v[c]
// accumulates in a register, the transposed product -sum_r A[r,c] v[r] is
// reduced across lanes with a 31-shuffle butterfly (lane l ends with column
// c0 + l). Each stored element is read once per column (4m^3/3 bytes in
// FP64 over the whole reduction). Partial sums go to two small buffers that
// K4 reduces.
#include "common.cuh"
#include "gemm_simt.cuh"
#include "../../include/bse_stages.h"

namespace bse {

constexpr int TRD_NB = 64;   // panel width (the paper's n_b)
constexpr int TRD_TB = 32;   // sub-tile edge = warp width
constexpr int TRD_QC = 16;   // sub-tiles per warp work item

template <typename T>
struct TrdWork {
  T* VP;        // m x 2NB: [V | P]
  T* PV;        // m x 2NB: [P | -V]
  T* Dpart;     // direct partials   [ns][maxQ][32]
  T* Tpart;     // transposed partials [ns][ns][32]
  double* norm2; // m
  double* dots;  // m x 2NB: V^T v, P^T v per column
};

static inline size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

template <typename T>
size_t trd_worksize(int m) {
  size_t ns = ceil_div(m, TRD_TB);
  size_t maxQ = ceil_div((long)ns, TRD_QC);
  size_t b = 0;
  b += 2 * align256(sizeof(T) * (size_t)m * 2 * TRD_NB);
  b += align256(sizeof(T) * ns * maxQ * TRD_TB);
  b += align256(sizeof(T) * ns * ns * TRD_TB);
  b += align256(sizeof(double) * (size_t)m);
  b += align256(sizeof(double) * (size_t)m * 2 * TRD_NB);
  return b;
}

template <typename T>
static TrdWork<T> carve(void* work, int m) {
  size_t ns = ceil_div(m, TRD_TB);
  size_t maxQ = ceil_div((long)ns, TRD_QC);
  char* p = reinterpret_cast<char*>(work);
  TrdWork<T> w;
  w.VP = reinterpret_cast<T*>(p); p += align256(sizeof(T) * (size_t)m * 2 * TRD_NB);
  w.PV = reinterpret_cast<T*>(p); p += align256(sizeof(T) * (size_t)m * 2 * TRD_NB);
  w.Dpart = reinterpret_cast<T*>(p); p += align256(sizeof(T) * ns * maxQ * TRD_TB);
  w.Tpart = reinterpret_cast<T*>(p); p += align256(sizeof(T) * ns * ns * TRD_TB);
  w.norm2 = reinterpret_cast<double*>(p); p += align256(sizeof(double) * (size_t)m);
  w.dots = reinterpret_cast<double*>(p);
  return w;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// K1: apply the panel's pending updates to column j, accumulate ||w[1:]||^2.
template <typename T>
__global__ void __launch_bounds__(256) trd_colupdate(int m, int j, int c, T* __restrict__ W, long ldw,
                                                     const T* __restrict__ VP, double* __restrict__ norm2) {
  __shared__ double red[8];
  const int r = j + 1 + blockIdx.x * 256 + threadIdx.x;
  double sq = 0.0;
  if (r < m) {
    T w = W[r + (long)j * ldw];
    for (int t = 0; t < c; ++t) {
      const T vr = VP[r + (long)t * m], pr = VP[r + (long)(TRD_NB + t) * m];
      const T vj = VP[j + (long)t * m], pj = VP[j + (long)(TRD_NB + t) * m];
      w = fma(vr, pj, w);
      w = fma(-pr, vj, w);
    }
    W[r + (long)j * ldw] = w;
    if (r >= j + 2) sq = (double)w * (double)w;
  }
  sq = warp_sum(sq);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sq;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < 8; ++k) s += red[k];
    if (s != 0.0) atomicAdd(norm2 + j, s);
  }
}

struct House {
  double beta, tau, scal;
};

__device__ __forceinline__ House make_house(double alpha, double sigma) {
  House h;
  if (sigma == 0.0) {
    h.beta = alpha; h.tau = 0.0; h.scal = 0.0;
  } else {
    const double nrm = sqrt(alpha * alpha + sigma);
    h.beta = alpha >= 0.0 ? -nrm : nrm;
    h.tau = (h.beta - alpha) / h.beta;
    h.scal = 1.0 / (alpha - h.beta);
  }
  return h;
}

// K2: Householder vector v (scaled in place), tau, beta; V^T v and P^T v.
template <typename T>
__global__ void __launch_bounds__(256) trd_house(int m, int j, int c, T* __restrict__ W, long ldw, T* VP,
                                                 T* PV, const double* __restrict__ norm2,
                                                 double* __restrict__ dots, double* __restrict__ e,
                                                 T* __restrict__ tau_out) {
  __shared__ double red[8][2 * TRD_NB];
  const double alpha = (double)W[(j + 1) + (long)j * ldw];
  const House h = make_house(alpha, norm2[j]);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    e[j] = h.beta;
    tau_out[j] = (T)h.tau;
  }
  const int r = j + 1 + blockIdx.x * 256 + threadIdx.x;
  double v = 0.0;
  if (r < m) {
    v = (r == j + 1) ? 1.0 : (double)W[r + (long)j * ldw] * h.scal;
    const T vt = (T)v;
    VP[r + (long)c * m] = vt;
    PV[r + (long)(TRD_NB + c) * m] = -vt;
    if (r > j + 1) W[r + (long)j * ldw] = vt;
    v = (double)vt;
  }
  if (c == 0) return;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int t = 0; t < c; ++t) {
    double a = 0.0, b = 0.0;
    if (r < m) {
      a = (double)VP[r + (long)t * m] * v;
      b = (double)VP[r + (long)(TRD_NB + t) * m] * v;
    }
    a = warp_sum(a);
    b = warp_sum(b);
    if (lane == 0) {
      red[wid][t] = a;
      red[wid][TRD_NB + t] = b;
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < 2 * TRD_NB; q += 256) {
    if ((q % TRD_NB) >= c) continue;
    double s = 0.0;
    for (int k = 0; k < 8; ++k) s += red[k][q];
    if (s != 0.0) atomicAdd(dots + (long)j * 2 * TRD_NB + q, s);
  }
}

// K3: skew SYMV partials over the trailing matrix rows/cols [s, m) of A0 (the
// stored strict lower triangle of W). 4 warps per CTA, one work item per warp.
template <typename T>
__global__ void __launch_bounds__(128) trd_symv(int m, int s, const T* __restrict__ W, long ldw,
                                                const T* __restrict__ v, T* __restrict__ Dpart,
                                                T* __restrict__ Tpart, int ns, int maxQ) {
  const int lane = threadIdx.x & 31;
  const long item = (long)blockIdx.x * 4 + (threadIdx.x >> 5);
  const int Rr = (int)(item / maxQ), q = (int)(item % maxQ);
  if (Rr >= ns) return;
  const int cb0 = q * TRD_QC;
  if (cb0 > Rr) return;
  const int cb1 = min(cb0 + TRD_QC, Rr + 1);
  const int sb = s / TRD_TB;
  const int r = (sb + Rr) * TRD_TB + lane;
  const bool rok = (r >= s) && (r < m);
  const T vr = rok ? v[r] : T(0);
  const T* Wr = W + (rok ? r : s);
  T yd = T(0);
  for (int cb = cb0; cb < cb1; ++cb) {
    const int c0 = (sb + cb) * TRD_TB;
    const bool diag = (cb == Rr);
    T a[TRD_TB];
#pragma unroll
    for (int k = 0; k < TRD_TB; ++k) {
      const int cc = c0 + k;
      const bool ok = rok && cc >= s && cc < m && (!diag || cc < r);
      a[k] = ok ? Wr[(long)cc * ldw] : T(0);
    }
#pragma unroll
    for (int k = 0; k < TRD_TB; ++k) {
      const int cc = c0 + k;
      const T vc = (cc >= s && cc < m) ? v[cc] : T(0);
      yd = fma(a[k], vc, yd);
      a[k] *= vr;
    }
    // butterfly reduce-scatter: lane l ends with sum over lanes of a[l]
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
      const bool up = (lane & off) != 0;
#pragma unroll
      for (int k = 0; k < off; ++k) {
        const T send = up ? a[k] : a[k + off];
        const T keep = up ? a[k + off] : a[k];
        a[k] = keep + __shfl_xor_sync(0xffffffffu, send, off);
      }
    }
    // a[0] = sum_r A[r, c0+lane] v[r]: contributes -a[0] to y[c0+lane]
    if (diag) {
      yd -= a[0];
    } else {
      Tpart[((long)cb * ns + Rr) * TRD_TB + lane] = -a[0];
    }
  }
  Dpart[((long)Rr * maxQ + q) * TRD_TB + lane] = yd;
}

// K4: y = reduced partials; p = tau (y + V (P^T v) - P (V^T v)); store p.
template <typename T>
__global__ void __launch_bounds__(256) trd_finalize(int m, int j, int c, T* __restrict__ W, long ldw,
                                                    T* VP, T* PV, const T* __restrict__ Dpart,
                                                    const T* __restrict__ Tpart, int ns, int maxQ,
                                                    const double* __restrict__ dots,
                                                    const T* __restrict__ tau_in) {
  const int s = j + 1;
  const int r = s + blockIdx.x * 256 + threadIdx.x;
  if (blockIdx.x == 0 && threadIdx.x == 0) W[(j + 1) + (long)j * ldw] = T(1);
  if (r >= m) return;
  const int sb = s / TRD_TB;
  const int Rr = r / TRD_TB - sb, l = r % TRD_TB;
  const int nq = (Rr + TRD_QC) / TRD_QC;  // ceil((Rr+1)/QC)
  T y = T(0);
  for (int q = 0; q < nq; ++q) y += Dpart[((long)Rr * maxQ + q) * TRD_TB + l];
  for (int R2 = Rr + 1; R2 < ns; ++R2) y += Tpart[((long)Rr * ns + R2) * TRD_TB + l];
  const double* d = dots + (long)j * 2 * TRD_NB;
  for (int t = 0; t < c; ++t) {
    y = fma(VP[r + (long)t * m], (T)d[TRD_NB + t], y);
    y = fma(-VP[r + (long)(TRD_NB + t) * m], (T)d[t], y);
  }
  const T p = tau_in[j] * y;
  VP[r + (long)(TRD_NB + c) * m] = p;
  PV[r + (long)c * m] = p;
}

template <typename T>
int tridiagonalize(int m, T* W, long ldw, double* e, T* tau, void* work, cudaStream_t st) {
  TrdWork<T> w = carve<T>(work, m);
  BSE_CUDA(cudaMemsetAsync(w.norm2, 0, sizeof(double) * (size_t)m, st));
  BSE_CUDA(cudaMemsetAsync(w.dots, 0, sizeof(double) * (size_t)m * 2 * TRD_NB, st));
  const int ncols = m - 1;  // columns 0..m-2 carry a reflector (the last one is trivial)
  for (int j0 = 0; j0 < ncols; j0 += TRD_NB) {
    const int nbp = min(TRD_NB, ncols - j0);
    // zero rows [j0, m) of the panel buffers
    BSE_CUDA(cudaMemset2DAsync(w.VP + j0, (size_t)m * sizeof(T), 0, (size_t)(m - j0) * sizeof(T), 2 * TRD_NB, st));
    BSE_CUDA(cudaMemset2DAsync(w.PV + j0, (size_t)m * sizeof(T), 0, (size_t)(m - j0) * sizeof(T), 2 * TRD_NB, st));
    for (int c = 0; c < nbp; ++c) {
      const int j = j0 + c;
      const int rows = m - j - 1;
      const int g = ceil_div(rows, 256);
      {
        KprofScope ks(K_TRD_COL, st, 0.0, 0.0);
        trd_colupdate<T><<<g, 256, 0, st>>>(m, j, c, W, ldw, w.VP, w.norm2);
      }
      {
        KprofScope ks(K_TRD_COL, st, 0.0, 0.0);
        trd_house<T><<<g, 256, 0, st>>>(m, j, c, W, ldw, w.VP, w.PV, w.norm2, w.dots, e, tau);
      }
      const int s = j + 1;
      const int ns = ceil_div(m, TRD_TB) - s / TRD_TB;
      const int maxQ = ceil_div(ns, TRD_QC);
      const long items = (long)ns * maxQ;
      {
        // algorithmic traffic: the strict lower triangle of the trailing matrix, once
        const double N = (double)(m - s);
        KprofScope ks(K_TRD_SYMV, st, N * (N - 1.0) * 0.5 * sizeof(T), 2.0 * N * (N - 1.0));
        trd_symv<T><<<(unsigned)ceil_div(items, 4), 128, 0, st>>>(m, s, W, ldw, w.VP + (long)c * m, w.Dpart,
                                                                 w.Tpart, ns, maxQ);
      }
      {
        KprofScope ks(K_TRD_COL, st, 0.0, 0.0);
        trd_finalize<T><<<g, 256, 0, st>>>(m, j, c, W, ldw, w.VP, w.PV, w.Dpart, w.Tpart, ns, maxQ, w.dots, tau);
      }
    }
    BSE_LAUNCH_CHECK();
    const int s2 = j0 + nbp;
    const int N = m - s2;
    if (N > 1 && s2 < ncols) {
      // A0[s2:, s2:] += [V P] [P -V]^T  (strict lower triangle)
      BSE_TRY(gemm<T>(N, N, 2 * TRD_NB, 1.0, w.VP + s2, m, false, w.PV + s2, m, true, 1.0,
                      W + s2 + (long)s2 * ldw, ldw, st, TRI_NONE, TRI_NONE, 2));
    }
  }
  return BSE_OK;
}

template size_t trd_worksize<double>(int);
template size_t trd_worksize<float>(int);
template int tridiagonalize<double>(int, double*, long, double*, double*, void*, cudaStream_t);
template int tridiagonalize<float>(int, float*, long, double*, float*, void*, cudaStream_t);

}  // namespace bse

extern "C" size_t bse_stage_tridiag_worksize(int m, int fp32) {
  return fp32 ? bse::trd_worksize<float>(m) : bse::trd_worksize<double>(m);
}

extern "C" int bse_stage_tridiag(int m, void* W, int ldw, double* e, void* tau, int fp32, void* work,
                                 void* stream) {
  if (m < 2 || !W || ldw < m || !e || !tau || !work) return BSE_ERR_ARG;
  if (fp32)
    return bse::tridiagonalize<float>(m, (float*)W, ldw, e, (float*)tau, work, (cudaStream_t)stream);
  return bse::tridiagonalize<double>(m, (double*)W, ldw, e, (double*)tau, work, (cudaStream_t)stream);
}
