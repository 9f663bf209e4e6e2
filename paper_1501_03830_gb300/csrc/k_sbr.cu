// Two-stage (successive band) reduction of the skew-symmetric W to tridiagonal
// form for the FP32 bulk of the mixed path -- Section 3.3's closing remark names
// band reduction as the way past the memory-bound skew SYMV of Algorithm 3's
// one-stage reduction (step 1, remark 1).
//
// Stage 1, dense -> band of half-bandwidth b = SBR_B. For the panels of b columns
// j0 = 0, b, 2b, ...: the block P = W[r0:m, j0:j0+b] (r0 = j0 + b) below the band
// is QR-factored, P = Q [R; 0] with Q = I - V T V^T (Householder, LAPACK
// conventions), and the trailing skew matrix A = W[r0:m, r0:m] is transformed,
//     A <- Q^T A Q = A + V Y^T - Y V^T,
//     X = A V T,   Z = T^T V^T X (skew),   Y = X - V Z / 2
// (A^T = -A gives V^T A = -(A V)^T and V^T A V skew, which folds the two-sided
// product into one rank-2b update). X and the update are tensor-core GEMMs; the
// trailing matrix is kept in full (both triangles) so that A V is a plain
// product. R goes into the band, V (unit diagonal implicit) below it, tau[j]
// per column: reflector j acts on rows j+b .. m-1.
//
// Stage 2, band -> tridiagonal (bulge chasing). Sweep j annihilates column j
// below its first sub-diagonal entry with a reflector on rows/columns
// I_0 = [j+1, j+b]; the right-hand application to the block below creates a
// bulge whose first column the next reflector (rows I_1 = I_0 + b) annihilates,
// and so on down the band: step k of sweep j uses H_{j,k} on I_k = [j+1+kb,
// j+(k+1)b]. Step k of sweep j touches matrix entries that step k+1 of sweep j-1
// also touches, and nothing of later steps of earlier sweeps, so sweep j may run
// step k once sweep j-1 has finished step k+1: the sweeps proceed as a pipeline,
// one thread block per sweep, synchronised by per-sweep progress counters
// (bounded waits). The band and its bulges live in a compact lower band array.
// Q2 = prod_j prod_k H_{j,k} (in the sequential order) is kept as (v, tau) per
// (j, k) for the back-transform.
//
// Both stages are orthogonal similarities that leave index 0 alone, so
// W = Q T Q^T with Q = Q1 Q2 and Q e_1 = e_1; T's sub-diagonal goes to e (the
// one-stage convention: e[j] = T[j+1, j]).
#include "common.cuh"
#include "gemm_simt.cuh"
#include "internal.cuh"
#include "../../include/bse_stages.h"

namespace bse {

constexpr int SBR_B = 64;     // half-bandwidth after stage 1
constexpr int QR_RB = 128;    // panel rows per thread block of the panel QR
constexpr int GRAM_RB = 64;   // rows per thread block of the tall-skinny Gram kernel
constexpr int SBR_LDB = 2 * SBR_B + 1;  // compact band: rows j .. j+2b of column j
constexpr long kSbrSpin = 1L << 25;     // polls before a wait gives up (~2 s)

static inline size_t al256s(size_t b) { return (b + 255) & ~(size_t)255; }
static inline long ld32(long x) { return (x + 31) / 32 * 32; }

// steps of sweep j: blocks I_k = [j+1+kb, j+(k+1)b] that start inside the matrix
__host__ __device__ inline int sbr_steps(int m, int j) { return (m - 1 - j + SBR_B - 1) / SBR_B; }

struct SbrWork {
  float* VY;      // ldv x 2b: [V | Y]
  float* YV;      // ldv x 2b: [Y | -V]
  float* X;       // ldv x b
  float *G, *S, *Z, *Tf;  // b x b
  double* Gpart;  // ceil(m / GRAM_RB) x b x b partial Gram matrices
  double* qpart;  // [2][grid][b + 1] panel-QR partial sums
  double* rowq;   // [2][b] pivot rows of the panel QR
  unsigned* bar;  // grid barrier words (panel QR)
  float* band;    // SBR_LDB x m compact lower band (stage 2)
  float* V2;      // Kmax x m x b reflectors of stage 2
  float* tau2;    // Kmax x m
  int* progress;  // m: completed steps per sweep
  float* Tq;      // b x b triangular factor per back-transform block of stage 2
  long ldv;
  int kmax;
};

size_t sbr_q2_blocks(int m);
static_assert(SBR_B == kSbrBand, "band width");

size_t sbr_worksize(int m) {
  const size_t ldv = ld32(m), kmax = sbr_steps(m, 0) + 1, grid = (m + QR_RB - 1) / QR_RB + 1;
  const size_t gparts = (m + GRAM_RB - 1) / GRAM_RB + 1;
  size_t b = 0;
  b += 2 * al256s(4 * ldv * 2 * SBR_B) + al256s(4 * ldv * SBR_B);
  b += 4 * al256s(4 * SBR_B * SBR_B);
  b += al256s(8 * gparts * SBR_B * SBR_B);
  b += al256s(8 * 2 * grid * (SBR_B + 1)) + al256s(8 * 2 * SBR_B) + al256s(64);
  b += al256s(4 * (size_t)SBR_LDB * m);
  b += al256s(4 * kmax * (size_t)m * SBR_B) + al256s(4 * kmax * (size_t)m);
  b += al256s(4 * (size_t)m);
  b += al256s(4 * sbr_q2_blocks(m) * SBR_B * SBR_B);
  return b;
}

static SbrWork carve_sbr(void* work, int m) {
  SbrWork w;
  w.ldv = ld32(m);
  w.kmax = sbr_steps(m, 0) + 1;
  const size_t grid = (m + QR_RB - 1) / QR_RB + 1;
  char* p = reinterpret_cast<char*>(work);
  auto take = [&](size_t sz) {
    void* r = p;
    p += al256s(sz);
    return r;
  };
  w.VY = (float*)take(4 * w.ldv * 2 * SBR_B);
  w.YV = (float*)take(4 * w.ldv * 2 * SBR_B);
  w.X = (float*)take(4 * w.ldv * SBR_B);
  w.G = (float*)take(4 * SBR_B * SBR_B);
  w.S = (float*)take(4 * SBR_B * SBR_B);
  w.Z = (float*)take(4 * SBR_B * SBR_B);
  w.Tf = (float*)take(4 * SBR_B * SBR_B);
  w.Gpart = (double*)take(8 * ((m + GRAM_RB - 1) / GRAM_RB + 1) * SBR_B * SBR_B);
  w.qpart = (double*)take(8 * 2 * grid * (SBR_B + 1));
  w.rowq = (double*)take(8 * 2 * SBR_B);
  w.bar = (unsigned*)take(64);
  w.band = (float*)take(4 * (size_t)SBR_LDB * m);
  w.V2 = (float*)take(4 * (size_t)w.kmax * m * SBR_B);
  w.tau2 = (float*)take(4 * (size_t)w.kmax * m);
  w.progress = (int*)take(4 * (size_t)m);
  w.Tq = (float*)take(4 * sbr_q2_blocks(m) * SBR_B * SBR_B);
  return w;
}

// ---- small helpers ------------------------------------------------------------

struct SbrHouse {
  double beta, tau, scal;
};
// Reflector H = I - tau v v^T with v[0] = 1, H x = beta e_1, for x[0] = alpha and
// sigma = ||x[1:]||^2 (dlarfg convention: beta = -sign(alpha) ||x||).
__device__ __forceinline__ SbrHouse sbr_house(double alpha, double sigma) {
  SbrHouse h;
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

// Grid barrier of a cooperative launch, bounded like the tridiagonal panel's.
__device__ __forceinline__ bool sbr_grid_barrier(unsigned* bar, DevStatus* st, long spin) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = bar + 1;
    const unsigned g = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u);
    int ok = 1;
    if (arrived == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long it = 0;
      while (*vgen == g) {
        if (++it > spin) {
          set_status(st, BSE_ERR_TIMEOUT, 2);
          ok = 0;
          break;
        }
        __nanosleep(40);
      }
    }
    __threadfence();
    if (*(volatile int*)&st->code != 0) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// W[i, j] = -W[j, i] for i < j (the upper triangle from the stored lower one),
// zero diagonal: the trailing matrices of stage 1 are kept in full.
__global__ void sbr_mirror(int m, float* __restrict__ W, long ldw) {
  __shared__ float t[32][33];
  const int bi = blockIdx.x * 32, bj = blockIdx.y * 32;  // upper tile: rows bi.., columns bj..
  if (bi > bj) return;
  // the mirrored lower tile W[bj + x, bi + y], read along its columns
  for (int y = threadIdx.y; y < 32; y += 8) {
    const int row = bj + threadIdx.x, c = bi + y;
    t[y][threadIdx.x] = (row < m && c < m && row > c) ? W[row + (long)c * ldw] : 0.f;
  }
  __syncthreads();
  // W[bi + x, bj + y] = -W[bj + y, bi + x] above the diagonal, 0 on it
  for (int y = threadIdx.y; y < 32; y += 8) {
    const int row = bi + threadIdx.x, c = bj + y;
    if (row < m && c < m && row <= c) W[row + (long)c * ldw] = (row == c) ? 0.f : -t[threadIdx.x][y];
  }
}

// Partial A^T B over GRAM_RB-row blocks (A, B: rows x b, FP32; FP32 sums of 64
// terms per block); sbr_gram_sum adds the partials in FP64 in block order
// (deterministic).
__global__ void __launch_bounds__(256) sbr_gram_part(int rows, const float* __restrict__ A, long lda,
                                                     const float* __restrict__ B, long ldb,
                                                     double* __restrict__ part) {
  __shared__ float sA[GRAM_RB][SBR_B + 1];
  __shared__ float sB[GRAM_RB][SBR_B + 1];
  const int r0 = blockIdx.x * GRAM_RB;
  for (int e = threadIdx.x; e < GRAM_RB * SBR_B; e += 256) {
    const int r = e % GRAM_RB, c = e / GRAM_RB;
    const bool ok = r0 + r < rows;
    sA[r][c] = ok ? A[r0 + r + (long)c * lda] : 0.f;
    sB[r][c] = ok ? B[r0 + r + (long)c * ldb] : 0.f;
  }
  __syncthreads();
  const int i = threadIdx.x & 63, jb = threadIdx.x >> 6;  // output (i, jb + 4q)
  float acc[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) acc[q] = 0.f;
  for (int r = 0; r < GRAM_RB; ++r) {
    const float a = sA[r][i];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = fmaf(a, sB[r][jb + 4 * q], acc[q]);
  }
  double* out = part + (size_t)blockIdx.x * SBR_B * SBR_B;
#pragma unroll
  for (int q = 0; q < 16; ++q) out[i + (jb + 4 * q) * SBR_B] = (double)acc[q];
}

__global__ void sbr_gram_sum(int parts, const double* __restrict__ part, float* __restrict__ G) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= SBR_B * SBR_B) return;
  double s = 0.0;
  for (int b = 0; b < parts; ++b) s += part[(size_t)b * SBR_B * SBR_B + e];
  G[e] = (float)s;
}

static int gram(int rows, const float* A, long lda, const float* B, long ldb, double* part, float* G,
                cudaStream_t s) {
  const int parts = ceil_div(rows, GRAM_RB);
  KprofScope ks(K_ELEMENTWISE, s, 8.0 * rows * (double)SBR_B, 4.0 * rows * (double)SBR_B * SBR_B);
  sbr_gram_part<<<parts, 256, 0, s>>>(rows, A, lda, B, ldb, part);
  BSE_LAUNCH_CHECK();
  sbr_gram_sum<<<ceil_div(SBR_B * SBR_B, 256), 256, 0, s>>>(parts, part, G);
  BSE_LAUNCH_CHECK();
  return BSE_OK;
}

// VY[:, 0:b] = V with explicit unit diagonal and zeros above it, from the panel
// of W (rows r0.., columns j0..j0+b-1); columns nr.. are zero.
__global__ void sbr_copy_v(int N, int nr, const float* __restrict__ P, long ldw, float* __restrict__ V, long ldv) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x, q = blockIdx.y;
  if (r >= N) return;
  float v = 0.f;
  if (q < nr) v = (r == q) ? 1.f : (r > q ? P[r + (long)q * ldw] : 0.f);
  V[r + (long)q * ldv] = v;
}

// YV = [Y | -V] from VY = [V | Y].
__global__ void sbr_make_yv(int N, const float* __restrict__ VY, float* __restrict__ YV, long ldv) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x, q = blockIdx.y;
  if (r >= N) return;
  YV[r + (long)q * ldv] = VY[r + (long)(SBR_B + q) * ldv];
  YV[r + (long)(SBR_B + q) * ldv] = -VY[r + (long)q * ldv];
}

// ---- stage 1: panel QR ------------------------------------------------------------
// Householder QR of the N x nc panel P (nc <= b), one cooperative launch: block g
// keeps rows [g QR_RB, (g+1) QR_RB) in shared memory. For reflector q, every
// block adds up, over its rows i > q, sigma = sum P[i,q]^2 and d_c = sum P[i,q] P[i,c]
// (c > q) (FP32 over 32 rows, FP64 beyond: FP64 arithmetic is scarce on this
// GPU); the owner of row q publishes it. After one grid barrier every
// block sums the partials in block order (the same numbers everywhere), forms the
// reflector (beta, tau, 1/(alpha - beta)) and w_c = v^T P[:, c] = P[q,c] +
// d_c / (alpha - beta), and updates its rows: P[i,c] -= tau v_i w_c, P[i,q] = v_i.
// Partials and pivot rows are double-buffered by the parity of q, so one barrier
// per reflector suffices.
struct QrArgs {
  int N, nc, nr;
  float* P;
  long ld;
  float* tau;
  double* part;  // [2][gridDim.x][SBR_B + 1]
  double* rowq;  // [2][SBR_B]
  unsigned* bar;
  DevStatus* st;
  long spin;
};

__global__ void __launch_bounds__(256) sbr_panel_qr(QrArgs a) {
  __shared__ float sP[QR_RB][SBR_B + 1];
  __shared__ double sred[4][SBR_B];
  __shared__ double sdot[SBR_B];
  __shared__ double srow[SBR_B];
  __shared__ float sw[SBR_B];
  __shared__ double sh[3];
  const int tid = threadIdx.x;
  const int i0 = blockIdx.x * QR_RB;
  const int rows = min(QR_RB, a.N - i0);
  const int G = gridDim.x;
  for (int e = tid; e < QR_RB * SBR_B; e += 256) {
    const int r = e % QR_RB, c = e / QR_RB;
    sP[r][c] = (r < rows && c < a.nc) ? a.P[i0 + r + (long)c * a.ld] : 0.f;
  }
  __syncthreads();
  const int c = tid & 63, rg = tid >> 6;  // column c, rows rg*32 .. rg*32+31 of the block
  for (int q = 0; q < a.nr; ++q) {
    const int par = q & 1;
    double* part = a.part + (size_t)par * G * (SBR_B + 1);
    // partial sums over this block's rows i > q
    float acc = 0.f;
    if (c >= q && c < a.nc) {
      const int rbeg = max(rg * 32, q + 1 - i0), rend = min(rg * 32 + 32, rows);
      for (int r = rbeg; r < rend; ++r) acc = fmaf(sP[r][q], sP[r][c], acc);
    }
    sred[rg][c] = (double)acc;
    __syncthreads();
    if (tid < SBR_B) {
      const double t = (sred[0][tid] + sred[1][tid]) + (sred[2][tid] + sred[3][tid]);
      part[(size_t)blockIdx.x * (SBR_B + 1) + tid] = t;
      if (q >= i0 && q < i0 + rows) a.rowq[par * SBR_B + tid] = (double)sP[q - i0][tid];
    }
    if (!sbr_grid_barrier(a.bar, a.st, a.spin)) return;
    // every block: the same sums, in block order
    if (tid < SBR_B) {
      double t = 0.0;
      if (tid >= q && tid < a.nc)
        for (int b = 0; b < G; ++b) t += __ldcg(part + (size_t)b * (SBR_B + 1) + tid);
      sdot[tid] = t;
      srow[tid] = __ldcg(a.rowq + par * SBR_B + tid);
    }
    __syncthreads();
    if (tid == 0) {
      const SbrHouse h = sbr_house(srow[q], sdot[q]);
      sh[0] = h.beta;
      sh[1] = h.tau;
      sh[2] = h.scal;
      if (blockIdx.x == 0) a.tau[q] = (float)h.tau;
    }
    __syncthreads();
    const float tau = (float)sh[1], scal = (float)sh[2];
    if (tid < SBR_B) sw[tid] = (tid > q && tid < a.nc) ? (float)(srow[tid] + sh[2] * sdot[tid]) : 0.f;
    __syncthreads();
    // update: rows i > q of this block (v_i = P[i,q] scal), and row q if owned
    for (int e = tid; e < rows * SBR_B; e += 256) {
      const int r = e % rows, cc = e / rows;
      const int i = i0 + r;
      if (cc < q || cc >= a.nc || i < q) continue;
      if (i == q) {
        if (cc == q) sP[r][cc] = (float)sh[0];
        else sP[r][cc] = fmaf(-tau, sw[cc], sP[r][cc]);
      } else {
        if (cc == q) continue;  // scaled after every column of this row is updated
        const float v = sP[r][q] * scal;
        sP[r][cc] = fmaf(-tau * v, sw[cc], sP[r][cc]);
      }
    }
    __syncthreads();
    for (int r = tid; r < rows; r += 256)
      if (i0 + r > q) sP[r][q] *= scal;
    __syncthreads();
  }
  for (int e = tid; e < rows * SBR_B; e += 256) {
    const int r = e % rows, cc = e / rows;
    if (cc < a.nc) a.P[i0 + r + (long)cc * a.ld] = sP[r][cc];
  }
  if (blockIdx.x == 0)
    for (int q = a.nr + tid; q < a.nc; q += 256) a.tau[q] = 0.f;
}

// Triangular factor T (upper, k x k in a b x b array) of H_0 ... H_{k-1} = I - V T V^T
// from G = V^T V and the tau: column i is T[0:i, i] = -tau_i T[0:i, 0:i] G[0:i, i],
// T[i, i] = tau_i (forward, column-wise accumulation).
__global__ void sbr_larft(int k, const float* __restrict__ G, const float* __restrict__ tau, float* __restrict__ Tf) {
  __shared__ double Ts[SBR_B][SBR_B + 1];
  __shared__ double g[SBR_B];
  const int t = threadIdx.x;  // blockDim = SBR_B
  for (int r = 0; r < SBR_B; ++r) Ts[r][t] = 0.0;
  __syncthreads();
  for (int i = 0; i < k; ++i) {
    const double ti = tau[i];
    g[t] = (t < i) ? -ti * (double)G[t + i * SBR_B] : 0.0;
    __syncthreads();
    if (t < i) {
      double s = 0.0;
      for (int l = t; l < i; ++l) s += Ts[t][l] * g[l];
      Ts[t][i] = s;
    }
    if (t == 0) Ts[i][i] = ti;
    __syncthreads();
  }
  for (int r = 0; r < SBR_B; ++r) Tf[r + t * SBR_B] = (float)Ts[r][t];
}

// Stage 1 on W (FP32, lower triangle given, leading dimension ldw, m x m):
// afterwards W's band (0 < i - j <= b) holds the band matrix, W[j+b+1:, j] the
// reflector j below its implicit unit entry at row j+b, tau[j] its scalar.
static int sbr_stage1(int m, float* W, long ldw, float* tau, const SbrWork& w, DevStatus* st, cudaStream_t s) {
  const long ldv = w.ldv;
  {
    KprofScope ks(K_ELEMENTWISE, s, 4.0 * (double)m * m, 0.0);
    sbr_mirror<<<dim3(ceil_div(m, 32), ceil_div(m, 32)), dim3(32, 8), 0, s>>>(m, W, ldw);
  }
  BSE_LAUNCH_CHECK();
  BSE_CUDA(cudaMemsetAsync(w.bar, 0, 64, s));
  BSE_CUDA(cudaMemsetAsync(tau, 0, sizeof(float) * (size_t)m, s));
  int dev = 0, nsm = 0, per_sm = 0;
  BSE_CUDA(cudaGetDevice(&dev));
  BSE_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  BSE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sbr_panel_qr, 256, 0));
  float* V = w.VY;
  float* Yp = w.VY + SBR_B * ldv;
  for (int j0 = 0;; j0 += SBR_B) {
    const int r0 = j0 + SBR_B;
    if (r0 >= m - 1) break;
    const int N = m - r0;
    const int nc = min(SBR_B, m - j0);
    const int nr = min(nc, N - 1);
    float* P = W + r0 + (long)j0 * ldw;
    float* A = W + r0 + (long)r0 * ldw;
    QrArgs qa;
    qa.N = N; qa.nc = nc; qa.nr = nr; qa.P = P; qa.ld = ldw; qa.tau = tau + j0;
    qa.part = w.qpart; qa.rowq = w.rowq; qa.bar = w.bar; qa.st = st; qa.spin = kSbrSpin;
    const int grid = ceil_div(N, QR_RB);
    if (grid > nsm * per_sm) {
      record_message("band reduction: panel QR grid exceeds the co-resident blocks");
      return BSE_ERR_CUDA;
    }
    {
      KprofScope ks(K_SBR_QR, s, 8.0 * N * (double)nc, 4.0 * N * (double)nc * nc);
      void* args[] = {&qa};
      BSE_CUDA(cudaLaunchCooperativeKernel((const void*)sbr_panel_qr, dim3(grid), dim3(256), args, 0, s));
    }
    {
      KprofScope ks(K_ELEMENTWISE, s, 8.0 * N * (double)SBR_B, 0.0);
      sbr_copy_v<<<dim3(ceil_div(N, 256), SBR_B), 256, 0, s>>>(N, nr, P, ldw, V, ldv);
    }
    BSE_LAUNCH_CHECK();
    BSE_TRY(gram(N, V, ldv, V, ldv, w.Gpart, w.G, s));
    {
      KprofScope ks(K_ELEMENTWISE, s, 0.0, 0.0);
      sbr_larft<<<1, SBR_B, 0, s>>>(nr, w.G, tau + j0, w.Tf);
    }
    BSE_LAUNCH_CHECK();
    // X = A V T into the Y half of VY; Z = T^T V^T X; Y = X - V Z / 2
    BSE_TRY(gemm<float>(N, SBR_B, N, 1.0, A, ldw, false, V, ldv, false, 0.0, w.X, ldv, s));
    BSE_TRY(gemm<float>(N, SBR_B, SBR_B, 1.0, w.X, ldv, false, w.Tf, SBR_B, false, 0.0, Yp, ldv, s));
    BSE_TRY(gram(N, V, ldv, Yp, ldv, w.Gpart, w.S, s));
    BSE_TRY(gemm<float>(SBR_B, SBR_B, SBR_B, 1.0, w.Tf, SBR_B, true, w.S, SBR_B, false, 0.0, w.Z, SBR_B, s));
    BSE_TRY(gemm<float>(N, SBR_B, SBR_B, -0.5, V, ldv, false, w.Z, SBR_B, false, 1.0, Yp, ldv, s));
    {
      KprofScope ks(K_ELEMENTWISE, s, 16.0 * N * (double)SBR_B, 0.0);
      sbr_make_yv<<<dim3(ceil_div(N, 256), SBR_B), 256, 0, s>>>(N, w.VY, w.YV, ldv);
    }
    BSE_LAUNCH_CHECK();
    // A += [V Y] [Y -V]^T, both triangles
    BSE_TRY(gemm<float>(N, N, 2 * SBR_B, 1.0, w.VY, ldv, false, w.YV, ldv, true, 1.0, A, ldw, s));
  }
  return BSE_OK;
}

// ---- stage 2: bulge chasing -------------------------------------------------------

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// entry (r, c), r >= c, r - c <= 2b, of the compact lower band
__device__ __forceinline__ long bidx(int r, int c) { return (long)(r - c) + (long)c * SBR_LDB; }

// band[d + c LDB] = W[c + d, c] for 1 <= d <= b, zero elsewhere (diagonal, bulge room)
__global__ void sbr_extract_band(int m, const float* __restrict__ W, long ldw, float* __restrict__ band) {
  const int c = blockIdx.x;
  for (int d = threadIdx.x; d < SBR_LDB; d += blockDim.x)
    band[d + (long)c * SBR_LDB] = (d >= 1 && d <= SBR_B && c + d < m) ? W[c + d + (long)c * ldw] : 0.f;
}

// explicit unit entries of the stage-1 reflectors, W[j + b, j] = 1 (after the
// band has been copied out)
__global__ void sbr_unit_diag(int m, float* __restrict__ W, long ldw) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j + SBR_B < m) W[j + SBR_B + (long)j * ldw] = 1.f;
}

__global__ void sbr_subdiag(int m, const float* __restrict__ band, double* __restrict__ e) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < m - 1) e[j] = (double)band[1 + (long)j * SBR_LDB];
  if (j == m - 1) e[j] = 0.0;
}

struct ChaseArgs {
  int m;
  float* band;
  float* V2;    // [k][j][b]
  float* tau2;  // [k][j]
  int* progress;
  DevStatus* st;
  long spin;
};

// One block per sweep at a time (sweeps j = blockIdx.x, + gridDim.x, ...), the
// step's blocks in shared memory: D = B[I_k, I_k] (skew, both triangles) and, for
// k >= 1, O = B[I_k, I_{k-1}] (in the first column, for k = 0, column j's entries
// on rows I_0). Thread t works on row (or column) t / 4 and a quarter of the
// other index, the quarters combined by two shuffles.
__global__ void __launch_bounds__(256) sbr_chase(ChaseArgs a) {
  __shared__ float O[SBR_B][SBR_B + 1];
  __shared__ float D[SBR_B][SBR_B + 1];
  __shared__ float vprev[SBR_B], vcur[SBR_B], pv[SBR_B];
  __shared__ double sh[3];
  __shared__ int s_ok;
  const int tid = threadIdx.x, m = a.m;
  const int r4 = tid >> 2, q4 = (tid & 3) * (SBR_B / 4);  // row / column r4, quarter [q4, q4 + 16)
  float* band = a.band;
  for (int j = blockIdx.x; j < m - 2; j += gridDim.x) {
    const int K = sbr_steps(m, j);
    float tau_prev = 0.f;
    for (int k = 0; k < K; ++k) {
      if (tid == 0) {
        int ok = 1;
        if (j > 0) {
          const int need = min(k + 2, sbr_steps(m, j - 1));
          long it = 0;
          while (ld_acquire(a.progress + j - 1) < need) {
            if (*(volatile int*)&a.st->code != 0) {
              ok = 0;
              break;
            }
            if (++it > a.spin) {
              set_status(a.st, BSE_ERR_TIMEOUT, 3);
              ok = 0;
              break;
            }
            __nanosleep(32);
          }
        }
        s_ok = ok;
      }
      __syncthreads();
      if (!s_ok) return;
      const int rk = j + 1 + k * SBR_B;  // first row of I_k
      const int nk = min(SBR_B, m - rk);
      const int ck = (k >= 1) ? rk - SBR_B : j;  // first column of the O block
      for (int e = tid; e < SBR_B * SBR_B; e += 256) {
        const int r = e % SBR_B, c = e / SBR_B;
        if (r >= c) {  // lower triangle, read along columns; the upper one is its mirror
          const float d = (r > c && r < nk) ? __ldcg(band + bidx(rk + r, rk + c)) : 0.f;
          D[r][c] = d;
          D[c][r] = -d;
        }
        float o = 0.f;
        if (r < nk && (k >= 1 || c == 0)) o = __ldcg(band + bidx(rk + r, ck + c));
        O[r][c] = o;
      }
      __syncthreads();
      if (k >= 1) {
        // (a) right-hand application of the previous reflector: O <- O (I - tau v v^T)
        float s = 0.f;
#pragma unroll
        for (int c = 0; c < SBR_B / 4; ++c) s = fmaf(O[r4][q4 + c], vprev[q4 + c], s);
        s += __shfl_xor_sync(0xffffffffu, s, 1);
        s += __shfl_xor_sync(0xffffffffu, s, 2);
        const float tw = tau_prev * s;
#pragma unroll
        for (int c = 0; c < SBR_B / 4; ++c) O[r4][q4 + c] = fmaf(-tw, vprev[q4 + c], O[r4][q4 + c]);
        __syncthreads();
      }
      // (b) reflector annihilating O[1:nk, 0]
      if (tid < 32) {
        double sg = 0.0;
        for (int r = 1 + tid; r < nk; r += 32) sg += (double)O[r][0] * (double)O[r][0];
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) sg += __shfl_xor_sync(0xffffffffu, sg, o);
        if (tid == 0) {
          const SbrHouse h = sbr_house((double)O[0][0], sg);
          sh[0] = h.beta;
          sh[1] = h.tau;
          sh[2] = h.scal;
        }
      }
      __syncthreads();
      const float tau = (float)sh[1];
      if (tid < SBR_B) vcur[tid] = (tid == 0) ? 1.f : (tid < nk ? (float)((double)O[tid][0] * sh[2]) : 0.f);
      __syncthreads();
      if (tid < SBR_B) O[tid][0] = (tid == 0) ? (float)sh[0] : 0.f;
      if (k >= 1) {
        // (c) left-hand application to the other columns of O
        float s = 0.f;
#pragma unroll
        for (int r = 0; r < SBR_B / 4; ++r) s = fmaf(vcur[q4 + r], O[q4 + r][r4], s);
        s += __shfl_xor_sync(0xffffffffu, s, 1);
        s += __shfl_xor_sync(0xffffffffu, s, 2);
        if (r4 >= 1) {
          const float ts = tau * s;
#pragma unroll
          for (int r = 0; r < SBR_B / 4; ++r) O[q4 + r][r4] = fmaf(-ts, vcur[q4 + r], O[q4 + r][r4]);
        }
      }
      // (d) two-sided application to D: p = tau D v, D += v p^T - p v^T
      {
        float s = 0.f;
#pragma unroll
        for (int c = 0; c < SBR_B / 4; ++c) s = fmaf(D[r4][q4 + c], vcur[q4 + c], s);
        s += __shfl_xor_sync(0xffffffffu, s, 1);
        s += __shfl_xor_sync(0xffffffffu, s, 2);
        if ((tid & 3) == 0) pv[r4] = tau * s;
      }
      __syncthreads();
      {
        const float vr = vcur[r4], pr = pv[r4];
#pragma unroll
        for (int c = 0; c < SBR_B / 4; ++c)
          D[r4][q4 + c] = fmaf(vr, pv[q4 + c], fmaf(-pr, vcur[q4 + c], D[r4][q4 + c]));
      }
      __syncthreads();
      // store: D's lower triangle, O (its first column only on step 0), the reflector
      for (int e = tid; e < SBR_B * SBR_B; e += 256) {
        const int r = e % SBR_B, c = e / SBR_B;
        if (r < nk && c < r) __stcg(band + bidx(rk + r, rk + c), D[r][c]);
        if (r < nk && (k >= 1 || c == 0)) __stcg(band + bidx(rk + r, ck + c), O[r][c]);
      }
      if (tid < SBR_B) {
        a.V2[((long)k * m + j) * SBR_B + tid] = vcur[tid];
        vprev[tid] = vcur[tid];
      }
      if (tid == 0) a.tau2[(long)k * m + j] = tau;
      tau_prev = tau;
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        st_release(a.progress + j, k + 1);
      }
    }
  }
}

// ---- back-transform of stage 2: Phi <- Phi Q2 ---------------------------------------
// The reflectors H_{j,k} of QG = b consecutive sweeps j in [g b, g b + b) at one
// step k act on the windows [j+1+kb, j+(k+1)b], shifted by one per sweep: as a
// block they are I - V T V^T with V the (2b-1) x b "parallelogram" (column t is
// v_{gb+t,k} at rows t .. t+b-1 of the block's window [gb+1+kb, gb+(k+2)b-1)).
// H_{j,k} must follow H_{j-1,k} and H_{j-1,k+1} (they overlap) and commutes with
// everything it does not overlap, so applying the blocks group by group
// (g ascending) with k descending inside a group reproduces the product Q2 of the
// sequential order. The rows of Phi are independent: one thread block per slab of
// QR_RB rows applies every block to its slab, window columns in shared memory.
constexpr int Q2_RS = 128;  // rows of Phi per slab

__host__ __device__ inline int q2_groups(int m) { return (m - 2 + SBR_B - 1) / SBR_B; }
__host__ __device__ inline int q2_kmax(int m, int g) { return (g * SBR_B <= m - 3) ? sbr_steps(m, g * SBR_B) : 0; }

size_t sbr_q2_blocks(int m) {
  size_t t = 0;
  for (int g = 0; g < q2_groups(m); ++g) t += q2_kmax(m, g);
  return t;
}

// T factor of block (g, k) (grid: groups x Kmax; blocks with k >= kmax_g exit)
__global__ void __launch_bounds__(SBR_B) sbr_q2_prep(int m, const float* __restrict__ V2,
                                                     const float* __restrict__ tau2, float* __restrict__ Tq) {
  __shared__ float Vc[SBR_B][SBR_B + 1];  // Vc[t][i] = v_{gb+t,k}[i] (window row t + i)
  __shared__ float Ts[SBR_B][SBR_B + 1];
  __shared__ float tau[SBR_B], gcol[SBR_B];
  const int g = blockIdx.x, k = blockIdx.y, t = threadIdx.x;
  if (k >= q2_kmax(m, g)) return;
  long off = 0;
  for (int h = 0; h < g; ++h) off += q2_kmax(m, h);
  off += k;
  {
    const int j = g * SBR_B + t;
    const bool has = j <= m - 3 && k < sbr_steps(m, j);
    for (int i = 0; i < SBR_B; ++i) Vc[t][i] = has ? V2[((long)k * m + j) * SBR_B + i] : 0.f;
    tau[t] = has ? tau2[(long)k * m + j] : 0.f;
  }
  for (int r = 0; r < SBR_B; ++r) Ts[r][t] = 0.f;
  __syncthreads();
  // column i of T: T[0:i, i] = -tau_i T[0:i, 0:i] (V^T v_i)[0:i]; v_t^T v_i over the
  // common window rows i .. t+b-1 (t < i)
  for (int i = 0; i < SBR_B; ++i) {
    if (t < i) {
      double acc = 0.0;
      for (int q = i - t; q < SBR_B; ++q) acc = fma((double)Vc[t][q], (double)Vc[i][q - (i - t)], acc);
      gcol[t] = (float)(-(double)tau[i] * acc);
    }
    __syncthreads();
    if (t < i) {
      float sacc = 0.f;
      for (int l = t; l < i; ++l) sacc = fmaf(Ts[t][l], gcol[l], sacc);
      Ts[t][i] = sacc;
    }
    if (t == 0) Ts[i][i] = tau[i];
    __syncthreads();
  }
  float* out = Tq + off * SBR_B * SBR_B;
  for (int r = 0; r < SBR_B; ++r) out[r + t * SBR_B] = Ts[r][t];
}

constexpr int Q2_LDR = Q2_RS + 4;  // shared row pitch of the window and Z buffers
constexpr int Q2_SLOTS = 128;      // window columns held (a block window is at most 2b - 1 wide)
constexpr size_t Q2_SMEM = sizeof(float) * ((size_t)Q2_SLOTS * Q2_LDR + 2 * SBR_B * (SBR_B + 1) + 2 * SBR_B * Q2_LDR);

__device__ __forceinline__ void q2_move(int m, float* __restrict__ Phi, long ldp, float* ring, int r0, int rows,
                                        int c_lo, int c_hi, bool store) {
  // columns [c_lo, c_hi) between Phi[r0 .. r0+rows) and their ring slots
  const int ncol = c_hi - c_lo;
  for (int e = threadIdx.x; e < ncol * Q2_RS; e += blockDim.x) {
    const int r = e % Q2_RS, c = c_lo + e / Q2_RS;
    if (r >= rows) continue;
    float* sp = ring + (size_t)(c % Q2_SLOTS) * Q2_LDR + r;
    float* gp = Phi + r0 + r + (long)c * ldp;
    if (store) *gp = *sp;
    else *sp = *gp;
  }
}

__global__ void __launch_bounds__(256) sbr_q2_apply(int m, float* __restrict__ Phi, long ldp,
                                                    const float* __restrict__ V2, const float* __restrict__ Tq) {
  extern __shared__ __align__(16) float q2s[];
  float* ring = q2s;                                   // [slot][row]
  float (*Vc)[SBR_B + 1] = reinterpret_cast<float (*)[SBR_B + 1]>(ring + (size_t)Q2_SLOTS * Q2_LDR);
  float (*Ts)[SBR_B + 1] = Vc + SBR_B;
  float* Zs = reinterpret_cast<float*>(Ts + SBR_B);    // [t][row]
  float* Z2s = Zs + SBR_B * Q2_LDR;
  const int tid = threadIdx.x;
  const int r0 = blockIdx.x * Q2_RS, rows = min(Q2_RS, m - r0);
  const int rt = tid & 15, tt = tid >> 4;  // 8-row tile, 4-column (Z) or 8-column (update) tile
  int lo = 0, hi = 0;                       // window columns held in the ring
  long off = 0;
  const int NG = q2_groups(m);
  for (int g = 0; g < NG; ++g) {
    const int K = q2_kmax(m, g);
    for (int k = K - 1; k >= 0; --k) {
      const int s0 = g * SBR_B + 1 + k * SBR_B;
      const int wc = min(2 * SBR_B - 1, m - s0);
      // ring: write back what leaves, read what enters
      q2_move(m, Phi, ldp, ring, r0, rows, max(lo, s0 + wc), hi, true);
      q2_move(m, Phi, ldp, ring, r0, rows, lo, min(hi, s0), true);
      __syncthreads();
      const int keep_lo = max(lo, s0), keep_hi = min(hi, s0 + wc);
      if (keep_lo < keep_hi) {
        q2_move(m, Phi, ldp, ring, r0, rows, s0, keep_lo, false);
        q2_move(m, Phi, ldp, ring, r0, rows, keep_hi, s0 + wc, false);
      } else {
        q2_move(m, Phi, ldp, ring, r0, rows, s0, s0 + wc, false);
      }
      lo = s0;
      hi = s0 + wc;
      // the block's reflectors and T
      for (int e = tid; e < SBR_B * SBR_B; e += 256) {
        const int t = e / SBR_B, i = e % SBR_B;
        const int j = g * SBR_B + t;
        const bool has = j <= m - 3 && k < sbr_steps(m, j);
        Vc[t][i] = has ? __ldg(V2 + ((long)k * m + j) * SBR_B + i) : 0.f;
        Ts[i][t] = __ldg(Tq + (off + k) * SBR_B * SBR_B + i + t * SBR_B);
      }
      __syncthreads();
      // Z = Phi_w V (rows x b): column t of V is v_t at window rows t .. t+b-1
      {
        float acc[8][4];
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[u][q] = 0.f;
        const int t0 = 4 * tt;
        const int cend = min(t0 + 3 + SBR_B, wc);
        for (int c = t0; c < cend; ++c) {
          const float* col = ring + (size_t)((s0 + c) % Q2_SLOTS) * Q2_LDR + 8 * rt;
          float ph[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) ph[u] = col[u];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int i = c - (t0 + q);
            const float vv = (i >= 0 && i < SBR_B) ? Vc[t0 + q][i] : 0.f;
#pragma unroll
            for (int u = 0; u < 8; ++u) acc[u][q] = fmaf(ph[u], vv, acc[u][q]);
          }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int u = 0; u < 8; ++u) Zs[(t0 + q) * Q2_LDR + 8 * rt + u] = acc[u][q];
      }
      __syncthreads();
      // Z2 = Z T (T upper triangular)
      {
        float acc[8][4];
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[u][q] = 0.f;
        const int t0 = 4 * tt;
        for (int s = 0; s < t0 + 4; ++s) {
          float z[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) z[u] = Zs[s * Q2_LDR + 8 * rt + u];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float tv = (s <= t0 + q) ? Ts[s][t0 + q] : 0.f;
#pragma unroll
            for (int u = 0; u < 8; ++u) acc[u][q] = fmaf(z[u], tv, acc[u][q]);
          }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int u = 0; u < 8; ++u) Z2s[(t0 + q) * Q2_LDR + 8 * rt + u] = acc[u][q];
      }
      __syncthreads();
      // Phi_w -= Z2 V^T: window column c gets sum over t with 0 <= c - t < b
      {
        float acc[8][8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
          for (int v = 0; v < 8; ++v) acc[u][v] = 0.f;
        const int c0 = 8 * tt;
        const int tlo = max(0, c0 - SBR_B + 1), thi = min(SBR_B - 1, c0 + 7);
        for (int t = tlo; t <= thi; ++t) {
          float z[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) z[u] = Z2s[t * Q2_LDR + 8 * rt + u];
#pragma unroll
          for (int v = 0; v < 8; ++v) {
            const int i = c0 + v - t;
            const float vv = (i >= 0 && i < SBR_B) ? Vc[t][i] : 0.f;
#pragma unroll
            for (int u = 0; u < 8; ++u) acc[u][v] = fmaf(z[u], vv, acc[u][v]);
          }
        }
#pragma unroll
        for (int v = 0; v < 8; ++v) {
          const int c = c0 + v;
          if (c < wc) {
            float* col = ring + (size_t)((s0 + c) % Q2_SLOTS) * Q2_LDR + 8 * rt;
#pragma unroll
            for (int u = 0; u < 8; ++u) col[u] -= acc[u][v];
          }
        }
      }
      __syncthreads();
    }
    off += K;
  }
  q2_move(m, Phi, ldp, ring, r0, rows, lo, hi, true);
}

// ---- host drivers ---------------------------------------------------------------------

static long g_sbr_spin = kSbrSpin;

int sbr_reduce(int m, float* W, long ldw, double* e, float* tau, void* work, DevStatus* st, cudaStream_t s) {
  StatusScope ss(st);
  if (m < 3) {
    record_message("band reduction needs m >= 3");
    return BSE_ERR_ARG;
  }
  SbrWork w = carve_sbr(work, m);
  BSE_TRY(sbr_stage1(m, W, ldw, tau, w, st, s));
  {
    KprofScope ks(K_ELEMENTWISE, s, 4.0 * (SBR_B + SBR_LDB) * (double)m, 0.0);
    sbr_extract_band<<<m, 128, 0, s>>>(m, W, ldw, w.band);
  }
  BSE_LAUNCH_CHECK();
  {
    KprofScope ks(K_ELEMENTWISE, s, 8.0 * m, 0.0);
    sbr_unit_diag<<<ceil_div(m, 256), 256, 0, s>>>(m, W, ldw);
  }
  BSE_LAUNCH_CHECK();
  BSE_CUDA(cudaMemsetAsync(w.progress, 0, sizeof(int) * (size_t)m, s));
  BSE_CUDA(cudaMemsetAsync(w.V2, 0, sizeof(float) * (size_t)w.kmax * m * SBR_B, s));
  BSE_CUDA(cudaMemsetAsync(w.tau2, 0, sizeof(float) * (size_t)w.kmax * m, s));
  int dev = 0, nsm = 0, per_sm = 0;
  BSE_CUDA(cudaGetDevice(&dev));
  BSE_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  BSE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sbr_chase, 256, 0));
  if (per_sm < 1) {
    record_message("bulge-chasing kernel cannot be resident");
    return BSE_ERR_CUDA;
  }
  ChaseArgs ca;
  ca.m = m; ca.band = w.band; ca.V2 = w.V2; ca.tau2 = w.tau2; ca.progress = w.progress; ca.st = st;
  ca.spin = g_sbr_spin;
  const int grid = max(1, min(nsm, m - 2));
  {
    // charged: the steps' 16 b^2 flops (left, right and two-sided applications), no HBM bytes
    double steps = 0.0;
    for (int j = 0; j + 2 < m; ++j) steps += sbr_steps(m, j);
    KprofScope ks(K_SBR_CHASE, s, 0.0, 16.0 * SBR_B * SBR_B * steps);
    void* args[] = {&ca};
    BSE_CUDA(cudaLaunchCooperativeKernel((const void*)sbr_chase, dim3(grid), dim3(256), args, 0, s));
  }
  {
    KprofScope ks(K_ELEMENTWISE, s, 12.0 * m, 0.0);
    sbr_subdiag<<<ceil_div(m, 256), 256, 0, s>>>(m, w.band, e);
  }
  BSE_LAUNCH_CHECK();
  return BSE_OK;
}

int sbr_apply_q2(int m, float* Phi, long ldp, void* work, cudaStream_t s) {
  SbrWork w = carve_sbr(work, m);
  const int NG = q2_groups(m);
  {
    KprofScope ks(K_ELEMENTWISE, s, 0.0, 0.0);
    sbr_q2_prep<<<dim3(NG, w.kmax), SBR_B, 0, s>>>(m, w.V2, w.tau2, w.Tq);
  }
  BSE_LAUNCH_CHECK();
  static cudaError_t attr_err =
      cudaFuncSetAttribute(sbr_q2_apply, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Q2_SMEM);
  if (attr_err != cudaSuccess) {
    record_error("cudaFuncSetAttribute(sbr_q2_apply)", attr_err, __FILE__, __LINE__);
    return BSE_ERR_CUDA;
  }
  {
    // charged: 2 m^3-type flops of the reflectors (4 b flops per reflector and row), Phi read and written once
    double refl = 0.0;
    for (int j = 0; j + 2 < m; ++j) refl += sbr_steps(m, j);
    KprofScope ks(K_SBR_Q2, s, 8.0 * (double)m * m, 4.0 * SBR_B * (double)m * refl);
    sbr_q2_apply<<<ceil_div(m, Q2_RS), 256, Q2_SMEM, s>>>(m, Phi, ldp, w.V2, w.Tq);
  }
  BSE_LAUNCH_CHECK();
  return BSE_OK;
}

}  // namespace bse

extern "C" size_t bse_stage_sbr_worksize(int m) { return m >= 3 ? bse::sbr_worksize(m) : 0; }

extern "C" int bse_stage_sbr(int m, float* W, int ldw, double* e, float* tau, void* work, int* dev_status,
                             void* stream) {
  if (m < 3 || !W || ldw < m || !e || !tau || !work || !dev_status) return BSE_ERR_ARG;
  if ((ldw % 32) != 0 || (reinterpret_cast<uintptr_t>(W) % 16) != 0) {
    bse::record_message("bse_stage_sbr: W needs a 16-byte aligned base and a leading dimension divisible by 32");
    return BSE_ERR_ARG;
  }
  return bse::sbr_reduce(m, W, ldw, e, tau, work, reinterpret_cast<bse::DevStatus*>(dev_status),
                         (cudaStream_t)stream);
}

extern "C" int bse_stage_sbr_apply_q2(int m, float* Phi, int ldp, void* work, void* stream) {
  if (m < 3 || !Phi || ldp < m || !work) return BSE_ERR_ARG;
  return bse::sbr_apply_q2(m, Phi, ldp, work, (cudaStream_t)stream);
}

extern "C" int bse_stage_sbr_backtransform(int m, float* L, int ldl, const float* W, int ldw, const float* tau,
                                           const double* Vs, const double* lam, double* X, double* Y, int ldx,
                                           void* bt_work, void* sbr_work, void* stream) {
  if (m < 4 || (m & 1) || !L || !W || !tau || !Vs || !lam || ldl < m || ldw < m || ldx < m || !bt_work || !sbr_work)
    return BSE_ERR_ARG;
  return bse::backtransform<float>(m, L, ldl, W, ldw, tau, Vs, lam, X, Y, ldx, bt_work, (cudaStream_t)stream,
                                   bse::kSbrBand, sbr_work);
}
