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
  double* Gpart;  // ceil(m / QR_RB) x b x b partial Gram matrices
  double* qpart;  // [2][grid][b + 1] panel-QR partial sums
  double* rowq;   // [2][b] pivot rows of the panel QR
  unsigned* bar;  // grid barrier words (panel QR)
  float* band;    // SBR_LDB x m compact lower band (stage 2)
  float* V2;      // Kmax x m x b reflectors of stage 2
  float* tau2;    // Kmax x m
  int* progress;  // m: completed steps per sweep
  long ldv;
  int kmax;
};

size_t sbr_worksize(int m) {
  const size_t ldv = ld32(m), kmax = sbr_steps(m, 0) + 1, grid = (m + QR_RB - 1) / QR_RB + 1;
  size_t b = 0;
  b += 2 * al256s(4 * ldv * 2 * SBR_B) + al256s(4 * ldv * SBR_B);
  b += 4 * al256s(4 * SBR_B * SBR_B);
  b += al256s(8 * grid * SBR_B * SBR_B);
  b += al256s(8 * 2 * grid * (SBR_B + 1)) + al256s(8 * 2 * SBR_B) + al256s(64);
  b += al256s(4 * (size_t)SBR_LDB * m);
  b += al256s(4 * kmax * (size_t)m * SBR_B) + al256s(4 * kmax * (size_t)m);
  b += al256s(4 * (size_t)m);
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
  w.Gpart = (double*)take(8 * grid * SBR_B * SBR_B);
  w.qpart = (double*)take(8 * 2 * grid * (SBR_B + 1));
  w.rowq = (double*)take(8 * 2 * SBR_B);
  w.bar = (unsigned*)take(64);
  w.band = (float*)take(4 * (size_t)SBR_LDB * m);
  w.V2 = (float*)take(4 * (size_t)w.kmax * m * SBR_B);
  w.tau2 = (float*)take(4 * (size_t)w.kmax * m);
  w.progress = (int*)take(4 * (size_t)m);
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

// Partial A^T B over 128-row blocks (A, B: rows x b, FP32), in FP64 per block;
// sbr_gram_sum adds the partials in block order (deterministic).
__global__ void __launch_bounds__(256) sbr_gram_part(int rows, const float* __restrict__ A, long lda,
                                                     const float* __restrict__ B, long ldb,
                                                     double* __restrict__ part) {
  __shared__ float sA[QR_RB][SBR_B + 1];
  __shared__ float sB[QR_RB][SBR_B + 1];
  const int r0 = blockIdx.x * QR_RB;
  for (int e = threadIdx.x; e < QR_RB * SBR_B; e += 256) {
    const int r = e % QR_RB, c = e / QR_RB;
    const bool ok = r0 + r < rows;
    sA[r][c] = ok ? A[r0 + r + (long)c * lda] : 0.f;
    sB[r][c] = ok ? B[r0 + r + (long)c * ldb] : 0.f;
  }
  __syncthreads();
  const int i = threadIdx.x & 63, jb = threadIdx.x >> 6;  // output (i, jb + 4q)
  double acc[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) acc[q] = 0.0;
  for (int r = 0; r < QR_RB; ++r) {
    const double a = sA[r][i];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = fma(a, (double)sB[r][jb + 4 * q], acc[q]);
  }
  double* out = part + (size_t)blockIdx.x * SBR_B * SBR_B;
#pragma unroll
  for (int q = 0; q < 16; ++q) out[i + (jb + 4 * q) * SBR_B] = acc[q];
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
  const int parts = ceil_div(rows, QR_RB);
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
// (c > q) in FP64; the owner of row q publishes it. After one grid barrier every
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
  __shared__ double sw[SBR_B];
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
    double acc = 0.0;
    if (c >= q && c < a.nc) {
      const int rbeg = max(rg * 32, q + 1 - i0), rend = min(rg * 32 + 32, rows);
      for (int r = rbeg; r < rend; ++r) acc = fma((double)sP[r][q], (double)sP[r][c], acc);
    }
    sred[rg][c] = acc;
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
    const double tau = sh[1], scal = sh[2];
    if (tid < SBR_B) sw[tid] = (tid > q && tid < a.nc) ? srow[tid] + scal * sdot[tid] : 0.0;
    __syncthreads();
    // update: rows i > q of this block (v_i = P[i,q] scal), and row q if owned
    for (int e = tid; e < rows * SBR_B; e += 256) {
      const int r = e % rows, cc = e / rows;
      const int i = i0 + r;
      if (cc < q || cc >= a.nc || i < q) continue;
      if (i == q) {
        if (cc == q) sP[r][cc] = (float)sh[0];
        else sP[r][cc] = (float)((double)sP[r][cc] - tau * sw[cc]);
      } else {
        const double v = (double)sP[r][q] * scal;
        if (cc == q) continue;  // stored after every column of this row is updated
        sP[r][cc] = (float)((double)sP[r][cc] - tau * v * sw[cc]);
      }
    }
    __syncthreads();
    for (int r = tid; r < rows; r += 256)
      if (i0 + r > q) sP[r][q] = (float)((double)sP[r][q] * scal);
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
        float d = 0.f;
        if (r < nk && c < nk) {
          if (r > c) d = __ldcg(band + bidx(rk + r, rk + c));
          else if (r < c) d = -__ldcg(band + bidx(rk + c, rk + r));
        }
        D[r][c] = d;
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
