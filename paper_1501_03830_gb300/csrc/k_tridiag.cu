// Algorithm 3 step 1: W = U T U^T, skew-symmetric Householder tridiagonalization
// (Section 3.3, remark 1: a modified symmetric tridiagonal reduction with
// skew-symmetric level-2/level-3 kernels), blocked by NB = 64 columns.
//
// Column j (trailing matrix A_j = rows/cols j+1..m-1, skew):
//   w   = column j of A_j              (pending panel updates applied)
//   H_j = I - tau v v^T, H_j w = beta e_1   (dlarfg convention)
//   p   = tau A_j v                    (skew SYMV on the stored lower triangle
//                                       of the panel-start matrix A0, plus the
//                                       panel's V (P^T v) - P (V^T v))
//   A_{j+1} = H_j A_j H_j = A_j + v p^T - p v^T
// (for skew A, v^T A v = 0, so the symmetric algorithm's correction term
// vanishes). After NB columns the trailing lower triangle gets the rank-2NB
// update A0 <- A0 + V P^T - P V^T (a GEMM).
//
// Outputs: beta_j (the sub-diagonal T[j+1, j]) in e[j], tau_j in tau[j], and
// v_j in W[j+1:m, j] (with the explicit leading 1), j = 0..m-2.
//
// All NB columns of a panel run in one persistent cooperative launch with two
// grid barriers per column (see trd_panel_kernel). The skew SYMV is the
// HBM-bound part: warps take equal ranges of the 32x32 sub-tiles of the
// trailing lower triangle (see symv_item); each stored element is read once per
// column (4m^3/3 bytes in FP64 over the whole reduction). Partial sums go to two
// small buffers that the owners of the rows reduce after the barrier.
#include "common.cuh"
#include "gemm_simt.cuh"
#include "../../include/bse_stages.h"

namespace bse {

constexpr int TRD_NB = 64;   // panel width (the paper's n_b)
constexpr int TRD_TB = 32;   // sub-tile edge = warp width

template <typename T>
struct TrdWork {
  T* VP;        // m x 2NB: [V | P]
  T* PV;        // m x 2NB: [P | -V]
  T* Dpart;     // direct partials   [ns][ns][32]: strip, piece, row
  T* Tpart;     // transposed partials [ns][ns][32]
  double* normpart;  // [2][kMaxGrid] per-block partial squared norms of the next column (by column parity)
  double* alpha;     // [2] the next column's leading entry (by column parity)
  T* dotpart;   // [2][kMaxGrid][2NB] per-block partial V^T w, P^T w (by column parity)
  T* dotpart2;  // [kMaxGrid / kDotL1][2NB] sums of kDotL1 blocks' partials
  unsigned* bar;     // grid barrier words
};

constexpr int kMaxGrid = 1024;  // upper bound on the panel kernel's grid
constexpr int kDotL1 = 16;      // blocks whose dot-product partials one first-level sum adds

static inline size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }
// VP / PV leading dimension: m rounded up to 32 (aligned panels for the tensor-core update)
static inline long vp_ld(int m) { return ((long)m + 31) / 32 * 32; }

template <typename T>
size_t trd_worksize(int m) {
  size_t ns = ceil_div(m, TRD_TB);
  size_t maxQ = ns;  // work items hold >= 1 sub-tile
  size_t b = 0;
  b += 2 * align256(sizeof(T) * (size_t)vp_ld(m) * 2 * TRD_NB);
  b += align256(sizeof(T) * ns * maxQ * TRD_TB);
  b += align256(sizeof(T) * ns * ns * TRD_TB);
  b += align256(sizeof(double) * 2 * kMaxGrid);
  b += align256(sizeof(double) * 2);
  b += align256(sizeof(double) * 2 * kMaxGrid * 2 * TRD_NB);
  b += align256(sizeof(double) * (kMaxGrid / kDotL1) * 2 * TRD_NB);
  b += align256(64);
  return b;
}

template <typename T>
static TrdWork<T> carve(void* work, int m) {
  size_t ns = ceil_div(m, TRD_TB);
  size_t maxQ = ns;
  char* p = reinterpret_cast<char*>(work);
  TrdWork<T> w;
  w.VP = reinterpret_cast<T*>(p); p += align256(sizeof(T) * (size_t)vp_ld(m) * 2 * TRD_NB);
  w.PV = reinterpret_cast<T*>(p); p += align256(sizeof(T) * (size_t)vp_ld(m) * 2 * TRD_NB);
  w.Dpart = reinterpret_cast<T*>(p); p += align256(sizeof(T) * ns * maxQ * TRD_TB);
  w.Tpart = reinterpret_cast<T*>(p); p += align256(sizeof(T) * ns * ns * TRD_TB);
  w.normpart = reinterpret_cast<double*>(p); p += align256(sizeof(double) * 2 * kMaxGrid);
  w.alpha = reinterpret_cast<double*>(p); p += align256(sizeof(double) * 2);
  w.dotpart = reinterpret_cast<T*>(p); p += align256(sizeof(double) * 2 * kMaxGrid * 2 * TRD_NB);
  w.dotpart2 = reinterpret_cast<T*>(p); p += align256(sizeof(double) * (kMaxGrid / kDotL1) * 2 * TRD_NB);
  w.bar = reinterpret_cast<unsigned*>(p);
  return w;
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

template <typename T>
struct PanelArgs {
  int m, j0, nbp;
  T* W;
  long ldw;
  long ldvp;    // leading dimension of VP and PV
  T* VP;
  T* PV;
  T* Dpart;
  T* Tpart;
  double* normpart;
  double* alpha;
  T* dotpart;
  T* dotpart2;
  double* e;
  T* tau;
  unsigned* bar;  // [0] arrivals (monotonic within a launch)
  DevStatus* st;
  int vec;  // 16-byte vector loads of W are aligned (ldw multiple of 16 B / sizeof(T), W 16-B aligned)
  unsigned long long* trace;  // optional: [column][kTracePoints][trace_stride] globaltimer stamps
  int trace_cols;
  int trace_stride;  // the largest grid of any panel launch (the buffer's block dimension)
  long spin;  // polls before a grid-barrier wait gives up
};

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

constexpr int kTracePoints = 8;  // per column: see trd_panel_kernel

template <typename T>
__device__ __forceinline__ void trace_point(const PanelArgs<T>& a, int col, int point) {
  if (a.trace && threadIdx.x == 0 && col < a.trace_cols)
    a.trace[((long)col * kTracePoints + point) * a.trace_stride + blockIdx.x] = gtimer();
}

// Grid-wide barrier for a cooperative launch on a monotonic arrival counter
// (bar[0], zeroed before every launch): the k-th barrier of the launch is passed
// once the counter reaches k * gridDim.x, so the last block's arrival itself
// releases the others (no reset, no second word). The arrival is a release atomic
// (it publishes the block's writes, which __syncthreads ordered before it) and the
// poll an acquire load. The wait is bounded: after `spin` polls (2^25, about 2 s,
// unless a test lowers it) it records BSE_ERR_TIMEOUT and every block returns at
// its next barrier. A failure recorded by any block (or an earlier stage) also
// makes all blocks return.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned& epoch, DevStatus* st, long spin) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ++epoch;
    const unsigned target = epoch * gridDim.x;
    unsigned v;
    asm volatile("atom.add.release.gpu.u32 %0, [%1], 1;" : "=r"(v) : "l"(bar) : "memory");
    ++v;
    int ok = 1;
    long it = 0;
    while ((int)(v - target) < 0) {
      if (++it > spin) {
        set_status(st, BSE_ERR_TIMEOUT, 1);
        ok = 0;
        break;
      }
      // spin tightly first (the release usually comes within a few us), then back off
      if (it > 256) __nanosleep(40);
      asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
    }
    if (*(volatile int*)&st->code != 0) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

template <typename T>
__device__ __forceinline__ T ldcg(const T* p) {
  return __ldcg(p);
}

__device__ __forceinline__ double block_sum(double v, double* red8) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red8[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) t += red8[k];
  return t;
}

// Butterfly reduce-scatter across the warp: on return a[0] of lane l holds the
// sum over lanes of the input a[l].
template <typename T>
__device__ __forceinline__ void warp_reduce_scatter32(T (&a)[32], int lane) {
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
}

// SYMV work split: the T = ns (ns + 1) / 2 sub-tiles of the trailing lower
// triangle, numbered strip by strip (strip R holds sub-tiles R (R+1)/2 ..
// R (R+1)/2 + R, one per column block cb <= R), are cut into nw = min(warps, T)
// contiguous non-empty ranges of equal size (+-1): warp w < nw takes
// [floor(w T / nw), floor((w+1) T / nw)).
// A range covers parts ("pieces") of one or a few strips; piece q of strip R is
// the part owned by warp owner(first sub-tile of R) + q, which indexes its
// direct partial sums.
__device__ __forceinline__ int symv_owner(long t, int nw, long T) { return (int)(((t + 1) * nw - 1) / T); }

// strip R with R (R+1) / 2 <= t < (R+1)(R+2) / 2
__device__ __forceinline__ int symv_strip_of(long t) {
  int R = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while ((long)(R + 1) * (R + 2) / 2 <= t) ++R;
  while (R > 0 && (long)R * (R + 1) / 2 > t) --R;
  return R;
}

// pieces (direct partial sums) of strip R
__device__ __forceinline__ int symv_pieces(int R, int nw, long T) {
  const long S = (long)R * (R + 1) / 2;
  return symv_owner(S + R, nw, T) - symv_owner(S, nw, T) + 1;
}

template <typename T>
struct Vec;
template <>
struct Vec<float> {
  using V = float4;
  static constexpr int W = 4;
  __device__ static void split(const V& x, float* o) { o[0] = x.x; o[1] = x.y; o[2] = x.z; o[3] = x.w; }
};
template <>
struct Vec<double> {
  using V = double2;
  static constexpr int W = 2;
  __device__ static void split(const V& x, double* o) { o[0] = x.x; o[1] = x.y; }
};

// Skew SYMV partials for one work item (strip Rr, column blocks cb0..cb1-1 of
// the trailing matrix), processed by one warp. Lane (rg, cg) holds a VW x CPL
// block of every 32x32 sub-tile: rows r0 + rg*VW + [0, VW) (one 16-byte vector
// load per column) and columns c0 + cg*CPL + [0, CPL). Per element: one FMA for
// A v and one for A^T v. The v values of a sub-tile's 32 columns are one
// coalesced load (lane l: column c0 + l) shuffled to their users, and both the
// tile and its v values are prefetched one sub-tile ahead. The transposed sums
// are reduce-scattered over the RG lanes of a column group per sub-tile; the
// direct sums stay in registers for the whole item and are reduce-scattered
// over the CG lanes of a row group at its end. Sub-tiles that cross the matrix
// edge take a masked scalar-load path; the diagonal ones and those that cross
// row/column s load whole vectors and zero what lies outside.
template <typename T>
__device__ __forceinline__ void symv_item(const PanelArgs<T>& a, int j, int s, int sb, int ns, int Rr,
                                          int cb0, int cb1, int q, int lane) {
  constexpr int VW = Vec<T>::W;   // rows per lane
  constexpr int RG = 32 / VW;     // lanes along the rows of a sub-tile
  constexpr int CG = VW;          // column groups
  constexpr int CPL = 32 / CG;    // columns per lane (= RG)
  using V = typename Vec<T>::V;
  const int m = a.m;
  const long ldw = a.ldw;
  const T* __restrict__ W = a.W;
  const int rg = lane % RG, cg = lane / RG;
  const int r0 = (sb + Rr) * TRD_TB;
  const int rbase = r0 + rg * VW;
  // the unscaled column below row s (zero at s and outside)
  auto vval = [&](int idx) -> T { return (idx > s && idx < m) ? ldcg(W + idx + (long)j * ldw) : T(0); };
  T vr[VW];
#pragma unroll
  for (int i = 0; i < VW; ++i) vr[i] = vval(rbase + i);
  const bool rows_full = (r0 >= s) && (r0 + TRD_TB <= m);
  T yd[VW];
#pragma unroll
  for (int i = 0; i < VW; ++i) yd[i] = T(0);
  T cur[CPL][VW], nxt[CPL][VW];
  auto load_tile = [&](T (&dst)[CPL][VW], int cb) {
    const int c0 = (sb + cb) * TRD_TB;
    const int cbase = c0 + cg * CPL;
    const bool diag = (cb == Rr);
    // a sub-tile that lies inside the stored m x m array is read with vector
    // loads even where it is not wholly inside the trailing lower triangle (the
    // diagonal sub-tile, the strip and column block that contain row/column s):
    // the entries outside are then replaced by zeros (a select, so whatever the
    // strict upper triangle or the earlier columns hold never enters a sum)
    const bool inmem = a.vec && (r0 + TRD_TB <= m) && (c0 + TRD_TB <= m);
    if (inmem) {
#pragma unroll
      for (int k = 0; k < CPL; ++k) {
        const V x = *reinterpret_cast<const V*>(W + rbase + (long)(cbase + k) * ldw);
        Vec<T>::split(x, dst[k]);
      }
      if (diag || !rows_full || c0 < s) {
#pragma unroll
        for (int k = 0; k < CPL; ++k) {
          const int cc = cbase + k;
#pragma unroll
          for (int i = 0; i < VW; ++i) {
            const int r = rbase + i;
            const bool ok = r >= s && cc >= s && (!diag || cc < r);
            dst[k][i] = ok ? dst[k][i] : T(0);
          }
        }
      }
    } else {
#pragma unroll
      for (int k = 0; k < CPL; ++k) {
        const int cc = cbase + k;
#pragma unroll
        for (int i = 0; i < VW; ++i) {
          const int r = rbase + i;
          const bool ok = r >= s && r < m && cc >= s && cc < m && (!diag || cc < r);
          dst[k][i] = ok ? W[r + (long)cc * ldw] : T(0);
        }
      }
    }
  };
  load_tile(cur, cb0);
  T vl = vval((sb + cb0) * TRD_TB + lane), vln = T(0);
  for (int cb = cb0; cb < cb1; ++cb) {
    if (cb + 1 < cb1) {
      load_tile(nxt, cb + 1);
      vln = vval((sb + cb + 1) * TRD_TB + lane);
    }
    T t[CPL];
#pragma unroll
    for (int k = 0; k < CPL; ++k) {
      const T vc = __shfl_sync(0xffffffffu, vl, cg * CPL + k);
      T tk = T(0);
#pragma unroll
      for (int i = 0; i < VW; ++i) {
        yd[i] = fma(cur[k][i], vc, yd[i]);
        tk = fma(cur[k][i], vr[i], tk);
      }
      t[k] = tk;
    }
    // reduce-scatter over the RG lanes of this column group: lane rg ends with column cbase + rg
#pragma unroll
    for (int off = RG / 2; off >= 1; off >>= 1) {
      const bool up = (rg & off) != 0;
#pragma unroll
      for (int k = 0; k < off; ++k) {
        const T send = up ? t[k] : t[k + off];
        const T keep = up ? t[k + off] : t[k];
        t[k] = keep + __shfl_xor_sync(0xffffffffu, send, off);
      }
    }
    // transposed contribution -sum_r A[r, c] v[r] to y[c]; the diagonal sub-tile's
    // goes to the strip's own slot (cb == Rr), read back by the row owners
    a.Tpart[((long)cb * ns + Rr) * TRD_TB + cg * CPL + rg] = -t[0];
    if (cb + 1 < cb1) {
      vl = vln;
#pragma unroll
      for (int k = 0; k < CPL; ++k)
#pragma unroll
        for (int i = 0; i < VW; ++i) cur[k][i] = nxt[k][i];
    }
  }
  // direct sums: reduce-scatter over the CG lanes of a row group (shuffle
  // distance RG): lane (rg, cg) ends with row rbase + cg
#pragma unroll
  for (int off = CG / 2; off >= 1; off >>= 1) {
    const bool up = (cg & off) != 0;
#pragma unroll
    for (int i = 0; i < off; ++i) {
      const T send = up ? yd[i] : yd[i + off];
      const T keep = up ? yd[i + off] : yd[i];
      yd[i] = keep + __shfl_xor_sync(0xffffffffu, send, off * RG);
    }
  }
  a.Dpart[((long)Rr * ns + q) * TRD_TB + rg * VW + cg] = yd[0];
}

// One panel of the reduction (columns j0 .. j0+nbp-1) in one cooperative launch.
// Per column j (panel index c), two grid barriers separate
//   phase B/C: the skew SYMV partials of A0 w^ on the unscaled column below its
//              leading entry (no reflector scalars needed yet) and the first
//              level of the panel dot products;
//   phase D+A: every block forms the reflector (beta, tau, scal) from the
//              column's norm partials, then p = tau (A0 v + V (P^T v) - P (V^T v))
//              for its rows, v and p stored, then column j+1 updated with all
//              pending panel terms and its squared norm and panel dot products
//              accumulated.
// Blocks own groups of 32 rows counted from j+1 (see phase D); data written by
// other blocks during the launch is read with __ldcg (L2) so no stale L1 line is
// used. Trace points (bse_debug_trace_tridiag): 0 column start, 1 after the first
// barrier, 2 SYMV start, 3 SYMV share and first dot level done, 4 after the second
// barrier, 5 reflector formed, 6 p at row s known, 7 rows updated.
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 1) trd_panel_kernel(PanelArgs<T> a) {
  __shared__ double red8[16];
  __shared__ double sh_house[3];
  __shared__ double sh_ps[2];           // SYMV sum of w^ at row s, then p at row s
  __shared__ T s_acc[2 * TRD_NB];       // w^T V, w^T P over rows > s (all blocks)
  __shared__ T s_vec[4][TRD_NB];        // V^T v, P^T v, row s of V, row s of P
  __shared__ T wdots[8][2 * TRD_NB];
  const int m = a.m;
  const long ldw = a.ldw;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int nwarps = gridDim.x * 8;
  const int gwarp = blockIdx.x * 8 + wid;
  const int G = gridDim.x;
  T* __restrict__ W = a.W;
  T* VP = a.VP;
  T* PV = a.PV;
  const long ldvp = a.ldvp;
  unsigned epoch = 0;  // barriers passed in this launch (thread 0)
  T* sdV = s_vec[0];
  T* sdP = s_vec[1];
  T* sVs = s_vec[2];
  T* sPs = s_vec[3];

  // phase A for the first panel column: its norm and leading entry (no pending
  // updates yet)
  {
    const int j = a.j0;
    const int r = j + 1 + blockIdx.x * 256 + tid;
    double sq = 0.0;
    if (r < m && r >= j + 2) {
      const double w = (double)W[r + (long)j * ldw];
      sq = w * w;
    }
    sq = block_sum(sq, red8);
    if (tid == 0) a.normpart[blockIdx.x] = sq;
    if (blockIdx.x == 0 && tid == 0) a.alpha[0] = (double)W[(j + 1) + (long)j * ldw];
  }

  for (int c = 0; c < a.nbp; ++c) {
    const int j = a.j0 + c;
    const int s = j + 1;
    const int par = c & 1;
    trace_point(a, j, 0);
    // column j (updated by the previous column's phase D) is complete
    if (!grid_barrier(a.bar, epoch, a.st, a.spin)) return;
    trace_point(a, j, 1);

    // ---------------- phase B/C ----------------
    // skew SYMV partials of A0[s:, s:] w^ with w^ = the unscaled column below row
    // s (w^[s] = 0). With v = e_s + scal w^ (dlarfg: v[s] = 1), A0 v =
    // A0 e_s + scal A0 w^, and A0 e_s is column s of A0 below the diagonal; phase
    // D adds that column and the scaling once the reflector's scalars are known,
    // so the SYMV does not wait for the column's norm.
    trace_point(a, j, 2);
    {
      const int sb = s / TRD_TB;
      const int ns = ceil_div(m, TRD_TB) - sb;
      const long nsub = (long)ns * (ns + 1) / 2;
      const int nw = (int)min((long)nwarps, nsub);  // every range non-empty
      const long t0 = (long)gwarp * nsub / nw, t1 = (long)(gwarp + 1) * nsub / nw;
      if (gwarp < nw) {
        int R = symv_strip_of(t0);
        for (long t = t0; t < t1; ++R) {
          const long S = (long)R * (R + 1) / 2;
          const int c0 = (int)(t - S);
          const int c1 = (int)min((long)R + 1, t1 - S);
          const int q = gwarp - symv_owner(S, nw, nsub);
          symv_item<T>(a, j, s, sb, ns, R, c0, c1, q, lane);
          t = S + R + 1;
        }
      }
    }
    // first level of the dot-product reduction: block b < ceil(G/16) adds the
    // partials of blocks 16b .. 16b+15 (written by the previous column's phase D);
    // 2c <= 126 slots, one per thread. It runs after the block's SYMV share (it is
    // needed only after the second barrier), so the SYMV of these blocks starts
    // with the others'.
    if (c > 0 && blockIdx.x * kDotL1 < G && tid < 2 * c) {
      const int d1slot = tid < c ? tid : TRD_NB + (tid - c);
      const T* d1 = a.dotpart + (long)par * kMaxGrid * 2 * TRD_NB;
      const int b0 = blockIdx.x * kDotL1, b1 = min(b0 + kDotL1, G);
      T pv[kDotL1];
#pragma unroll
      for (int k = 0; k < kDotL1; ++k) pv[k] = (b0 + k < b1) ? ldcg(d1 + (long)(b0 + k) * 2 * TRD_NB + d1slot) : T(0);
      T t = T(0);
#pragma unroll
      for (int k = 0; k < kDotL1; ++k) t += pv[k];
      a.dotpart2[(long)blockIdx.x * 2 * TRD_NB + d1slot] = t;
    }
    trace_point(a, j, 3);
    if (!grid_barrier(a.bar, epoch, a.st, a.spin)) return;
    trace_point(a, j, 4);

    // ---------------- phase D (+ A of the next column) ----------------
    {
      const int sb = s / TRD_TB;
      const int ns = ceil_div(m, TRD_TB) - sb;
      const long Ttot = (long)ns * (ns + 1) / 2;
      const int nwp = (int)min((long)nwarps, Ttot);  // the SYMV split's warp count
      const bool next = (c + 1 < a.nbp);
      // D1: every block gathers, in one round of independent loads, the column's
      // squared norm (G partials), its leading entry, the panel dot products
      // (ceil(G/16) first-level sums per slot), row s of V and P, and the SYMV
      // partial sums of row s; then forms the reflector (every block alike: the
      // sums run in a fixed order) and p at row s. Every load is unrolled and
      // predicated so that all are in flight at once.
      double nrm = 0.0;
      {
        double v[kMaxGrid / 256];
#pragma unroll
        for (int k = 0; k < kMaxGrid / 256; ++k)
          v[k] = (tid + 256 * k < G) ? __ldcg(a.normpart + (long)par * kMaxGrid + tid + 256 * k) : 0.0;
#pragma unroll
        for (int k = 0; k < kMaxGrid / 256; ++k) nrm += v[k];
      }
      const double alpha = (tid == 0) ? __ldcg(a.alpha + par) : 0.0;
      // row s of [V | P] (stored to shared memory after the other loads are issued)
      const bool vps_ok = tid < c || (tid >= TRD_NB && tid - TRD_NB < c);
      const T vpsv = vps_ok ? ldcg(VP + s + (long)tid * ldvp) : T(0);
      // SYMV sum at row s: the transposed partials of its column block over all
      // strips, and the one direct piece of the first strip (its only sub-tile is
      // the diagonal one)
      T psum = T(0);
      {
        const int l = s % TRD_TB;
        T pp[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) pp[k] = (tid + 256 * k < ns) ? ldcg(a.Tpart + (long)(tid + 256 * k) * TRD_TB + l) : T(0);
        for (int R2 = tid + 2048; R2 < ns; R2 += 256) pp[0] += ldcg(a.Tpart + (long)R2 * TRD_TB + l);
        if (tid == 0) pp[1] += ldcg(a.Dpart + l);
        psum = ((pp[0] + pp[1]) + (pp[2] + pp[3])) + ((pp[4] + pp[5]) + (pp[6] + pp[7]));
      }
      // dot products: TP threads per slot (a power of two, TP * 2c <= 256)
      const int nslot = 2 * c;
      int TP = 16;
      while (TP > 1 && TP * nslot > 256) TP >>= 1;
      const int dq = tid / TP, dsub = tid % TP;
      const int nblk = ceil_div(G, kDotL1);
      T dacc = T(0);
      if (dq < nslot) {
        // nblk <= kMaxGrid / kDotL1 = 64 first-level sums, at most 32 per thread (TP >= 2)
        const int slot = dq < c ? dq : TRD_NB + (dq - c);
        T pa[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const int b = dsub + k * TP;
          pa[k] = b < nblk ? ldcg(a.dotpart2 + (long)b * 2 * TRD_NB + slot) : T(0);
        }
        for (int b = dsub + 16 * TP; b < nblk; b += TP) pa[0] += ldcg(a.dotpart2 + (long)b * 2 * TRD_NB + slot);
#pragma unroll
        for (int k = 0; k < 8; ++k) pa[k] += pa[k + 8];
        dacc = ((pa[0] + pa[1]) + (pa[2] + pa[3])) + ((pa[4] + pa[5]) + (pa[6] + pa[7]));
      }
      if (vps_ok) {
        if (tid < c) sVs[tid] = vpsv;
        else sPs[tid - TRD_NB] = vpsv;
      }
      // reductions: the norm and the row-s sum over the block, the dot products
      // over the TP threads of their slot
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) {
        nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
        psum += __shfl_xor_sync(0xffffffffu, psum, o);
      }
      for (int o = TP >> 1; o >= 1; o >>= 1) dacc += __shfl_xor_sync(0xffffffffu, dacc, o);
      if (lane == 0) {
        red8[wid] = nrm;
        red8[8 + wid] = (double)psum;
      }
      if (dq < nslot && dsub == 0) s_acc[dq] = dacc;
      // this warp's partial dot products of the next column with V, P (t <= c)
      T* wd = &wdots[wid][0];
      for (int t = lane; t < 2 * TRD_NB; t += 32) wd[t] = T(0);
      __syncthreads();
      if (tid == 0) {
        double sigma = 0.0, ps = 0.0;
        for (int w = 0; w < 8; ++w) {
          sigma += red8[w];
          ps += red8[8 + w];
        }
        const House h = make_house(alpha, sigma);
        sh_house[0] = h.beta;
        sh_house[1] = h.tau;
        sh_house[2] = h.scal;
        sh_ps[0] = ps;
        if (blockIdx.x == 0) {
          a.e[j] = h.beta;
          a.tau[j] = (T)h.tau;
        }
      }
      __syncthreads();
      trace_point(a, j, 5);
      const T scal = (T)sh_house[2];
      const T tauj = (T)sh_house[1];
      // V^T v and P^T v: v = e_s + scal w^, so each is row s of V (P) plus scal
      // times the dot products with w^
      if (tid < nslot) {
        const T lead = tid < c ? sVs[tid] : sPs[tid - c];
        const T d = fma(scal, s_acc[tid], lead);
        if (tid < c) sdV[tid] = d;
        else sdP[tid - c] = d;
      }
      __syncthreads();
      // p at row s (= j+1): every block needs it for the next column's update
      T p_s = T(0);
      if (next) {
        if (wid == 0) {
          T y = T(0);
          for (int t = lane; t < c; t += 32) y += sVs[t] * sdP[t] - sPs[t] * sdV[t];
#pragma unroll
          for (int o = 16; o >= 1; o >>= 1) y += __shfl_xor_sync(0xffffffffu, y, o);
          // (A0 e_s)[s] = 0
          if (lane == 0) sh_ps[1] = (double)(tauj * fma(scal, (T)sh_ps[0], y));
        }
        __syncthreads();
        p_s = (T)sh_ps[1];
      }
      trace_point(a, j, 6);
      // rows: 8 lanes per row, in groups of 32 rows from s. Group g goes to block
      // g mod G in a boustrophedon order (blocks 0, 1, .., G-1, then G-1, .., 0,
      // ...): the reduction of a row's transposed partials gets shorter down the
      // matrix (strips Rr .. ns-1), so each block pairs a long group with a short one
      const int l8 = tid & 7;
      const int sbD = s / TRD_TB;
      const int j1 = j + 1;
      double sq = 0.0;
      // the loop runs on a warp-uniform group index so every lane reaches the shuffles
      for (int k = 0;; ++k) {
        const int g = (k & 1) ? (k + 1) * G - 1 - (int)blockIdx.x : k * G + (int)blockIdx.x;
        if (s + g * 32 >= m) break;
        const int r = s + g * 32 + wid * 4 + (lane >> 3);
        const bool valid = r < m;
        const int Rr = r / TRD_TB - sbD, l = r % TRD_TB;
        const int nq = valid ? symv_pieces(Rr, nwp, Ttot) : 0;
        const int nsv = valid ? ns : 0;
        // the row's panel entries V[r, t], P[r, t] (t = l8 + 8k < c), column s of
        // A0 and the unscaled reflector, loaded up front so their latency overlaps
        // the partial-sum loads below
        T vvk[8], ppk[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int t = l8 + 8 * k;
          const bool ok = valid && t < c;
          vvk[k] = ok ? ldcg(VP + r + (long)t * ldvp) : T(0);
          ppk[k] = ok ? ldcg(VP + r + (long)(TRD_NB + t) * ldvp) : T(0);
        }
        const T w0 = (valid && r > s) ? ldcg(W + r + (long)j1 * ldw) : T(0);
        const T wj = (valid && r > s) ? ldcg(W + r + (long)j * ldw) : T(0);
        T acc[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] = T(0);
        const T* dp = a.Dpart + (long)Rr * ns * TRD_TB + l;
        acc[0] = (l8 < nq) ? ldcg(dp + (long)l8 * TRD_TB) : T(0);
        for (int q = l8 + 8; q < nq; q += 8) acc[0] += ldcg(dp + (long)q * TRD_TB);
        const T* tp = a.Tpart + (long)Rr * ns * TRD_TB + l;
        int R2 = Rr + l8;
        // up to 32 independent loads in flight per lane (unrolled and predicated):
        // the rows near the top have many strips to add
        for (; R2 < nsv; R2 += 256) {
          T t4[32];
#pragma unroll
          for (int k = 0; k < 32; ++k) t4[k] = (R2 + 8 * k < nsv) ? ldcg(tp + (long)(R2 + 8 * k) * TRD_TB) : T(0);
#pragma unroll
          for (int k = 0; k < 8; ++k) acc[k] += (t4[k] + t4[k + 8]) + (t4[k + 16] + t4[k + 24]);
        }
        T y = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
        const bool upd = next && r >= s + 1;
        T w = T(0), yp = T(0);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int t = l8 + 8 * k;
          if (valid && t < c) {
            yp = fma(vvk[k], sdP[t], yp);
            yp = fma(-ppk[k], sdV[t], yp);
            w = fma(vvk[k], sPs[t], w);
            w = fma(-ppk[k], sVs[t], w);
          }
        }
#pragma unroll
        for (int o = 4; o >= 1; o >>= 1) {
          y += __shfl_xor_sync(0xffffffffu, y, o);
          yp += __shfl_xor_sync(0xffffffffu, yp, o);
          w += __shfl_xor_sync(0xffffffffu, w, o);
        }
        // every lane of the row's group finishes the row (the sums are replicated by
        // the butterfly); lane l8 == 0 stores. (A0 v)[r] = A0[r, s] + scal (A0 w^)[r]
        const T vr = !valid ? T(0) : (r == s) ? T(1) : wj * scal;
        // row s takes the p_s every block formed (the same value the next column's
        // update uses)
        const T p = (next && r == s) ? p_s : tauj * (fma(scal, y, w0) + yp);
        T wf = T(0);
        if (valid && upd) {
          // column j+1 with all panel terms t <= c; t = c: V[j1, c] = 1, P[j1, c] = p_s
          w += w0;
          w = fma(vr, p_s, w);
          w = fma(-p, T(1), w);
          wf = w;
        }
        if (valid && l8 == 0) {
          VP[r + (long)c * ldvp] = vr;
          VP[r + (long)(TRD_NB + c) * ldvp] = p;
          PV[r + (long)c * ldvp] = p;
          PV[r + (long)(TRD_NB + c) * ldvp] = -vr;
          W[r + (long)j * ldw] = vr;  // the reflector, leading 1 included
          if (upd) {
            W[r + (long)j1 * ldw] = wf;
            if (r >= j1 + 2) sq += (double)wf * (double)wf;
            // the next column's leading entry, for its reflector
            if (r == j1 + 1) a.alpha[par ^ 1] = (double)wf;
          }
        }
        if (next) {
          // next column's dot products with the panel, rows below its leading entry:
          // lane l8 takes t = l8 + 8k (t < c from the prefetched entries, t = c the
          // new column v, p); the 4 rows of the warp are summed by shuffles
          const T wd_r = (valid && upd && r >= j1 + 2) ? wf : T(0);
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const int t = l8 + 8 * k;
            T dv = (t < c ? vvk[k] : (t == c ? vr : T(0))) * wd_r;
            T dq = (t < c ? ppk[k] : (t == c ? p : T(0))) * wd_r;
            dv += __shfl_xor_sync(0xffffffffu, dv, 8);
            dq += __shfl_xor_sync(0xffffffffu, dq, 8);
            dv += __shfl_xor_sync(0xffffffffu, dv, 16);
            dq += __shfl_xor_sync(0xffffffffu, dq, 16);
            if (lane < 8 && t <= c) {
              wd[t] += dv;
              wd[TRD_NB + t] += dq;
            }
          }
        }
      }
      trace_point(a, j, 7);
      if (next) {
        sq = block_sum(sq, red8);  // also orders the warps' dot partials before their sum
        if (tid == 0) a.normpart[(long)(par ^ 1) * kMaxGrid + blockIdx.x] = sq;
        T* dnext = a.dotpart + (long)(par ^ 1) * kMaxGrid * 2 * TRD_NB + (long)blockIdx.x * 2 * TRD_NB;
        for (int q = tid; q < 2 * (c + 1); q += 256) {
          const int slot = q <= c ? q : TRD_NB + (q - c - 1);
          T t = T(0);
#pragma unroll
          for (int k = 0; k < 8; ++k) t += wdots[k][slot];
          dnext[slot] = t;
        }
      }
      __syncthreads();  // the staged vectors are rewritten for the next column
    }
  }
}


// ---- small problems: the whole reduction in one CTA --------------------------
// For m <= TRD_SMALL_MAX the panel scheme's fixed costs per column (two grid
// barriers, partial-sum buffers) outweigh the work, so one CTA of 512 threads
// reduces the matrix alone, with only CTA barriers, and many such problems run
// side by side on the GPU. Unblocked form of the same recurrence: for column
// j+1, first its own update with (v_j, p_j), then its reflector, then ONE pass
// over the trailing lower triangle (rows/cols >= j+2, L2-resident at these
// sizes) that applies A += v_j p_j^T - p_j v_j^T and accumulates the skew SYMV
// y = A v_{j+1} for the next p = tau y. Warps take 32x32 tiles; lane = row, the
// row sums accumulate in a register and the column sums (skew: -A^T v) are
// reduced across the warp by the reduce-scatter butterfly; both go to the
// warp's own partial vector in shared memory, and the warps' partials are
// added in a fixed order, so results are reproducible bit for bit.
constexpr int TRD_SMALL_MAX = 512;  // FP64
#ifndef BSE_TRD_SMALL_MAX_F32
#define BSE_TRD_SMALL_MAX_F32 512
#endif
template <typename T>
constexpr int trd_small_max() { return sizeof(T) == 4 ? BSE_TRD_SMALL_MAX_F32 : TRD_SMALL_MAX; }

template <typename T>
__device__ __forceinline__ double cta_sum(double v, double* red32) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red32[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red32[k];
  return t;
}

// One pass over the tiles of rows/cols [s, m): optional update with (va, pa),
// then this warp's share of y = A vb (skew, lower triangle stored) added into
// its own partial vector `part` (summed over the warps in a fixed order
// afterwards, so the result does not depend on scheduling). A tile's 32 loads
// are all issued before any of its stores.
template <typename T, bool UPDATE>
__device__ __forceinline__ void small_pass(int m, int s, T* __restrict__ W, long ldw, const T* __restrict__ va,
                                           const T* __restrict__ pa, const T* __restrict__ vb, T* __restrict__ part) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int N = m - s;
  const int nb = (N + 31) / 32;
  const int tiles = nb * (nb + 1) / 2;
  for (int t = warp; t < tiles; t += nwarp) {
    int I = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while (I * (I + 1) / 2 > t) --I;
    while ((I + 1) * (I + 2) / 2 <= t) ++I;
    const int K = t - I * (I + 1) / 2;
    const int i = s + 32 * I + lane;
    const int k0 = s + 32 * K;
    const bool row_ok = i < m;
    T* col = W + i;
    T w[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) w[c] = (row_ok && k0 + c < i) ? col[(long)(k0 + c) * ldw] : T(0);
    const T vbi = row_ok ? vb[i] : T(0);
    if (UPDATE) {
      const T vai = row_ok ? va[i] : T(0);
      const T pai = row_ok ? pa[i] : T(0);
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        const int k = k0 + c;
        if (row_ok && k < i) {
          w[c] = w[c] + vai * pa[k] - pai * va[k];
          col[(long)k * ldw] = w[c];
        }
      }
    }
    T dir = T(0);
#pragma unroll
    for (int c = 0; c < 32; ++c) {
      dir += w[c] * vb[min(k0 + c, m - 1)];
      w[c] = -w[c] * vbi;  // column c's term of -A^T vb from this row
    }
    warp_reduce_scatter32<T>(w, lane);
    if (row_ok) part[i] += dir;
    if (k0 + lane < m) part[k0 + lane] += w[0];
  }
}

template <typename T>
__global__ void __launch_bounds__(512) trd_small_kernel(int m, T* __restrict__ W, long ldw, double* __restrict__ e,
                                                        T* __restrict__ tau, DevStatus* st) {
  extern __shared__ __align__(16) unsigned char trd_small_smem[];
  T* va = reinterpret_cast<T*>(trd_small_smem);  // v_j (global row index)
  T* pa = va + m;                                // p_j
  T* vb = pa + m;                                // v_{j+1}
  T* parts = vb + m;                             // [warps][m] partial sums of A v_{j+1}
  __shared__ double red32[32];
  __shared__ double s_alpha;
  if (st->code) return;
  const int tid = threadIdx.x, nt = blockDim.x, nwarp = nt >> 5;
  T* mypart = parts + (long)(tid >> 5) * m;
  for (int r = tid; r < nwarp * m; r += nt) parts[r] = T(0);
  // p = tau * (sum of the warps' partials), in warp order; partials cleared
  auto gather_p = [&](double tauv) {
    for (int r = tid; r < m; r += nt) {
      T y = T(0);
      for (int w = 0; w < nwarp; ++w) {
        y += parts[(long)w * m + r];
        parts[(long)w * m + r] = T(0);
      }
      pa[r] = (T)tauv * y;
    }
  };
  // column 0: its reflector, then p_0 = tau_0 A v_0 over rows/cols >= 1
  {
    double sq = 0.0;
    for (int r = 2 + tid; r < m; r += nt) {
      const double w = (double)W[r];
      sq += w * w;
    }
    const double sigma = cta_sum<T>(sq, red32);
    const House h = make_house((double)W[1], sigma);
    for (int r = tid; r < m; r += nt) {
      T v = T(0);
      if (r >= 1) v = (r == 1) ? T(1) : W[r] * (T)h.scal;
      va[r] = v;
      if (r >= 1) W[r] = v;
    }
    if (tid == 0) {
      e[0] = h.beta;
      tau[0] = (T)h.tau;
    }
    __syncthreads();
    small_pass<T, false>(m, 1, W, ldw, va, va, va, mypart);
    __syncthreads();
    gather_p(h.tau);
    __syncthreads();
  }
  for (int j = 0; j + 2 < m; ++j) {
    // (i) column j+1 gets its update from (v_j, p_j); v_j[j+1] = 1
    T* cj = W + (long)(j + 1) * ldw;
    const T pj1 = pa[j + 1];
    double sq = 0.0;
    for (int r = j + 2 + tid; r < m; r += nt) {
      const T w = cj[r] + va[r] * pj1 - pa[r];
      cj[r] = w;
      if (r == j + 2) s_alpha = (double)w;
      else sq += (double)w * (double)w;
    }
    const double sigma = cta_sum<T>(sq, red32);  // its barriers also publish s_alpha
    // (ii) reflector of column j+1
    const House h = make_house(s_alpha, sigma);
    for (int r = tid; r < m; r += nt) {
      T v = T(0);
      if (r >= j + 2) {
        v = (r == j + 2) ? T(1) : cj[r] * (T)h.scal;
        cj[r] = v;
      }
      vb[r] = v;
    }
    if (tid == 0) {
      e[j + 1] = h.beta;
      tau[j + 1] = (T)h.tau;
    }
    __syncthreads();
    // (iii) update + SYMV over rows/cols >= j+2
    small_pass<T, true>(m, j + 2, W, ldw, va, pa, vb, mypart);
    __syncthreads();
    // (iv) p_{j+1} = tau y; v_{j+1} becomes the current reflector
    gather_p(h.tau);
    for (int r = tid; r < m; r += nt) va[r] = vb[r];
    __syncthreads();
  }
}

static unsigned long long* g_trace = nullptr;
static int g_trace_cols = 0;
constexpr long kBarrierSpin = 1L << 25;
static long g_barrier_spin = kBarrierSpin;

template <typename T>
int tridiagonalize(int m, T* W, long ldw, double* e, T* tau, void* work, cudaStream_t st, DevStatus* status) {
  StatusScope ss(status);
  if (m <= trd_small_max<T>()) {
    double bytes = 0.0, flops = 0.0;
    for (int c = 0; c + 1 < m; ++c) {
      const double N = (double)(m - c - 1);
      bytes += N * (N - 1.0) * 0.5 * sizeof(T);
      flops += 2.0 * N * (N - 1.0);
    }
    const size_t smem = (3 + 16) * sizeof(T) * (size_t)m;  // v_j, p_j, v_{j+1}, 16 warp partials
    static cudaError_t attr_err = cudaFuncSetAttribute(trd_small_kernel<T>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                       (int)((3 + 16) * sizeof(T) * trd_small_max<T>()));
    if (attr_err != cudaSuccess) {
      record_error("cudaFuncSetAttribute(trd_small_kernel)", attr_err, __FILE__, __LINE__);
      return BSE_ERR_CUDA;
    }
    KprofScope ks(K_TRD_SYMV, st, bytes, flops);
    trd_small_kernel<T><<<1, 512, smem, st>>>(m, W, ldw, e, tau, status);
    BSE_LAUNCH_CHECK();
    return BSE_OK;
  }
  TrdWork<T> w = carve<T>(work, m);
  int dev = 0, nsm = 0, per_sm = 0;
  BSE_CUDA(cudaGetDevice(&dev));
  BSE_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  BSE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, trd_panel_kernel<T>, 256, 0));
  if (per_sm < 1) {
    record_message("tridiagonal panel kernel cannot be resident");
    return BSE_ERR_CUDA;
  }
  per_sm = min(per_sm, 2);
  if (nsm * per_sm > kMaxGrid) per_sm = max(1, kMaxGrid / nsm);
  const int ncols = m - 1;  // columns 0..m-2 carry a reflector (the last one is trivial)
  const long ldvp = vp_ld(m);
  for (int j0 = 0; j0 < ncols; j0 += TRD_NB) {
    const int nbp = min(TRD_NB, ncols - j0);
    // zero rows [j0, m) of the panel buffers
    BSE_CUDA(cudaMemset2DAsync(w.VP + j0, (size_t)ldvp * sizeof(T), 0, (size_t)(m - j0) * sizeof(T), 2 * TRD_NB, st));
    BSE_CUDA(cudaMemset2DAsync(w.PV + j0, (size_t)ldvp * sizeof(T), 0, (size_t)(m - j0) * sizeof(T), 2 * TRD_NB, st));
    // enough blocks for the owned rows and the SYMV items, at most per_sm per SM
    const int rows = m - j0 - 1;
    const long sub = (long)ceil_div(rows, TRD_TB);
    const long want = max((long)ceil_div(rows, 256), (sub * (sub + 1) / 2 + 7) / 8);
    const int grid = (int)max(1L, min((long)nsm * per_sm, want));
    PanelArgs<T> pa;
    pa.m = m; pa.j0 = j0; pa.nbp = nbp; pa.W = W; pa.ldw = ldw; pa.VP = w.VP; pa.PV = w.PV; pa.ldvp = ldvp;
    pa.Dpart = w.Dpart; pa.Tpart = w.Tpart; pa.normpart = w.normpart; pa.alpha = w.alpha;
    pa.dotpart = w.dotpart; pa.dotpart2 = w.dotpart2; pa.e = e; pa.tau = tau;
    pa.bar = w.bar; pa.st = status;
    pa.vec = ((ldw * (long)sizeof(T)) % 16 == 0) && ((reinterpret_cast<uintptr_t>(W) % 16) == 0);
    pa.trace = g_trace;
    pa.trace_cols = g_trace_cols;
    pa.trace_stride = nsm * per_sm;
    pa.spin = g_barrier_spin;
    if (grid * 256 < rows + 1 && grid < nsm * per_sm) {
      record_message("tridiagonal panel grid too small");
      return BSE_ERR_CUDA;
    }
    {
      // charged: the strict lower triangles of the nbp trailing matrices, once each
      double bytes = 0.0, flops = 0.0;
      for (int c = 0; c < nbp; ++c) {
        const double N = (double)(m - j0 - c - 1);
        bytes += N * (N - 1.0) * 0.5 * sizeof(T);
        flops += 2.0 * N * (N - 1.0);
      }
      // every launch counts its barriers from zero
      BSE_CUDA(cudaMemsetAsync(w.bar, 0, 64, st));
      KprofScope ks(K_TRD_SYMV, st, bytes, flops);
      void* args[] = {&pa};
      BSE_CUDA(cudaLaunchCooperativeKernel((const void*)trd_panel_kernel<T>, dim3(grid), dim3(256), args, 0, st));
    }
    const int s2 = j0 + nbp;
    const int N = m - s2;
    if (N > 1 && s2 < ncols) {
      // A0[s2:, s2:] += [V P] [P -V]^T  (strict lower triangle)
      BSE_TRY(gemm<T>(N, N, 2 * TRD_NB, 1.0, w.VP + s2, ldvp, false, w.PV + s2, ldvp, true, 1.0,
                      W + s2 + (long)s2 * ldw, ldw, st, TRI_NONE, TRI_NONE, 2));
    }
  }
  return BSE_OK;
}

template size_t trd_worksize<double>(int);
template size_t trd_worksize<float>(int);
template int tridiagonalize<double>(int, double*, long, double*, double*, void*, cudaStream_t, DevStatus*);
template int tridiagonalize<float>(int, float*, long, double*, float*, void*, cudaStream_t, DevStatus*);

}  // namespace bse

extern "C" int bse_debug_trace_tridiag(void* dev_buffer, int columns) {
  bse::g_trace = reinterpret_cast<unsigned long long*>(dev_buffer);
  bse::g_trace_cols = dev_buffer ? columns : 0;
  return BSE_OK;
}

extern "C" int bse_debug_barrier_spin(long polls) {
  if (polls < 0) return BSE_ERR_ARG;
  bse::g_barrier_spin = polls == 0 ? bse::kBarrierSpin : polls;
  return BSE_OK;
}

extern "C" int bse_stage_tridiag_grid(int m, int fp32) {
  int dev = 0, nsm = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (fp32) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, bse::trd_panel_kernel<float>, 256, 0);
  else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, bse::trd_panel_kernel<double>, 256, 0);
  return nsm * (per < 2 ? per : 2);
}

extern "C" size_t bse_stage_tridiag_worksize(int m, int fp32) {
  return fp32 ? bse::trd_worksize<float>(m) : bse::trd_worksize<double>(m);
}

extern "C" int bse_stage_tridiag(int m, void* W, int ldw, double* e, void* tau, int fp32, void* work,
                                 int* dev_status, void* stream) {
  if (m < 2 || !W || ldw < m || !e || !tau || !work || !dev_status) return BSE_ERR_ARG;
  auto* st = reinterpret_cast<bse::DevStatus*>(dev_status);
  if (fp32)
    return bse::tridiagonalize<float>(m, (float*)W, ldw, e, (float*)tau, work, (cudaStream_t)stream, st);
  return bse::tridiagonalize<double>(m, (double*)W, ldw, e, (double*)tau, work, (cudaStream_t)stream, st);
}
