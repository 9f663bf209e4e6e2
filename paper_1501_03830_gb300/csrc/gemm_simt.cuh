// Register-tiled SIMT GEMM used by the dense updates of the FP64 path and as
// the generic fallback shape of the FP32 path:
//
//   C = alpha * op(A) * op(B) + beta * C        (column-major, strided batches)
//
// op(A) is M x K, op(B) is K x N. Triangular structure is exploited at tile
// granularity and masked exactly on load, so the unused triangle of a
// triangular operand may hold anything:
//   a_tri = TRI_LOWER : op(A)(i,k) = 0 for k > i      a_tri = TRI_UPPER : 0 for k < i
//   b_tri = TRI_LOWER : op(B)(k,j) = 0 for k < j      b_tri = TRI_UPPER : 0 for k > j
// and the output can be restricted to the lower triangle (c_uplo = 1: i >= j,
// c_uplo = 2: i > j), where only tiles touching it are launched.
#pragma once

#include "common.cuh"

namespace bse {

enum { TRI_NONE = 0, TRI_LOWER = 1, TRI_UPPER = 2 };

struct GemmArgs {
  int M, N, K;
  const void* A;
  long lda, strideA;
  const void* B;
  long ldb, strideB;
  void* C;
  long ldc, strideC;
  double alpha, beta;
  int transA, transB;
  int a_tri, b_tri, c_uplo;
  int batch;
};

template <typename T, int BM, int BN, int BK, int TM, int TN>
struct GemmCfg {
  static constexpr int THREADS = (BM / TM) * (BN / TN);
};

template <typename T, int BM, int BN, int BK, int TM, int TN, bool TA, bool TB>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
    gemm_simt_kernel(GemmArgs g) {
  constexpr int NT = (BM / TM) * (BN / TN);
  constexpr int A_PER = BM * BK / NT;
  constexpr int B_PER = BN * BK / NT;
  static_assert(A_PER * NT == BM * BK, "A tile split");
  static_assert(B_PER * NT == BN * BK, "B tile split");
  __shared__ T As[2][BK][BM + 4];
  __shared__ T Bs[2][BK][BN + 4];

  const int tilesM = (g.M + BM - 1) / BM;
  const int ti = blockIdx.x % tilesM;
  const int tj = blockIdx.x / tilesM;
  const int i0 = ti * BM, j0 = tj * BN;
  if (i0 >= g.M || j0 >= g.N) return;
  if (g.c_uplo && i0 + BM - 1 < j0) return;  // tile strictly above the diagonal

  const long bz = blockIdx.z;
  const T* A = reinterpret_cast<const T*>(g.A) + bz * g.strideA;
  const T* B = reinterpret_cast<const T*>(g.B) + bz * g.strideB;
  T* C = reinterpret_cast<T*>(g.C) + bz * g.strideC;

  int kbeg = 0, kend = g.K;
  if (g.a_tri == TRI_LOWER) kend = min(kend, i0 + BM);
  if (g.a_tri == TRI_UPPER) kbeg = max(kbeg, i0);
  if (g.b_tri == TRI_LOWER) kbeg = max(kbeg, j0);
  if (g.b_tri == TRI_UPPER) kend = min(kend, j0 + BN);

  const int tid = threadIdx.x;
  // tx indexes rows (consecutive threads -> consecutive rows: coalesced C
  // stores), ty indexes columns.
  const int tx = tid % (BM / TM);
  const int ty = tid / (BM / TM);

  T acc[TM][TN];
#pragma unroll
  for (int r = 0; r < TM; ++r)
#pragma unroll
    for (int c = 0; c < TN; ++c) acc[r][c] = T(0);

  T ra[A_PER], rb[B_PER];

  auto load_global = [&](int k0) {
#pragma unroll
    for (int u = 0; u < A_PER; ++u) {
      int e = tid + u * NT;
      int ii, kk;
      if (!TA) { ii = e % BM; kk = e / BM; } else { kk = e % BK; ii = e / BK; }
      int gi = i0 + ii, gk = k0 + kk;
      T v = T(0);
      bool ok = gi < g.M && gk < kend && gk >= kbeg;
      if (g.a_tri == TRI_LOWER) ok = ok && gk <= gi;
      if (g.a_tri == TRI_UPPER) ok = ok && gk >= gi;
      if (ok) v = TA ? A[gk + (long)gi * g.lda] : A[gi + (long)gk * g.lda];
      ra[u] = v;
    }
#pragma unroll
    for (int u = 0; u < B_PER; ++u) {
      int e = tid + u * NT;
      int jj, kk;
      if (!TB) { kk = e % BK; jj = e / BK; } else { jj = e % BN; kk = e / BN; }
      int gj = j0 + jj, gk = k0 + kk;
      T v = T(0);
      bool ok = gj < g.N && gk < kend && gk >= kbeg;
      if (g.b_tri == TRI_LOWER) ok = ok && gk >= gj;
      if (g.b_tri == TRI_UPPER) ok = ok && gk <= gj;
      if (ok) v = TB ? B[gj + (long)gk * g.ldb] : B[gk + (long)gj * g.ldb];
      rb[u] = v;
    }
  };
  auto store_smem = [&](int buf) {
#pragma unroll
    for (int u = 0; u < A_PER; ++u) {
      int e = tid + u * NT;
      int ii, kk;
      if (!TA) { ii = e % BM; kk = e / BM; } else { kk = e % BK; ii = e / BK; }
      As[buf][kk][ii] = ra[u];
    }
#pragma unroll
    for (int u = 0; u < B_PER; ++u) {
      int e = tid + u * NT;
      int jj, kk;
      if (!TB) { kk = e % BK; jj = e / BK; } else { jj = e % BN; kk = e / BN; }
      Bs[buf][kk][jj] = rb[u];
    }
  };

  int k0 = kbeg - (kbeg % BK);
  if (k0 < kend) {
    load_global(k0);
    store_smem(0);
    __syncthreads();
    int buf = 0;
    for (; k0 < kend; k0 += BK) {
      const bool more = k0 + BK < kend;
      if (more) load_global(k0 + BK);
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        T a[TM], b[TN];
#pragma unroll
        for (int r = 0; r < TM; ++r) a[r] = As[buf][kk][tx + r * (BM / TM)];
#pragma unroll
        for (int c = 0; c < TN; ++c) b[c] = Bs[buf][kk][ty + c * (BN / TN)];
#pragma unroll
        for (int r = 0; r < TM; ++r)
#pragma unroll
          for (int c = 0; c < TN; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
      }
      if (more) {
        store_smem(buf ^ 1);
        __syncthreads();
        buf ^= 1;
      }
    }
  }

  const T alpha = T(g.alpha), beta = T(g.beta);
#pragma unroll
  for (int c = 0; c < TN; ++c) {
    int gj = j0 + ty + c * (BN / TN);
    if (gj >= g.N) continue;
#pragma unroll
    for (int r = 0; r < TM; ++r) {
      int gi = i0 + tx + r * (BM / TM);
      if (gi >= g.M) continue;
      if (g.c_uplo == 1 && gi < gj) continue;
      if (g.c_uplo == 2 && gi <= gj) continue;
      T* cp = C + gi + (long)gj * g.ldc;
      T v = alpha * acc[r][c];
      if (g.beta != 0.0) v = fma(beta, *cp, v);
      *cp = v;
    }
  }
}

// Host launcher (defined in gemm_simt.cu for T = float, double).
template <typename T>
int gemm(const GemmArgs& g, cudaStream_t s);

// Convenience wrapper: C = alpha op(A) op(B) + beta C.
template <typename T>
inline int gemm(int M, int N, int K, double alpha, const T* A, long lda, bool transA, const T* B,
                long ldb, bool transB, double beta, T* C, long ldc, cudaStream_t s, int a_tri = TRI_NONE,
                int b_tri = TRI_NONE, int c_uplo = 0) {
  GemmArgs g{};
  g.M = M; g.N = N; g.K = K;
  g.A = A; g.lda = lda; g.B = B; g.ldb = ldb; g.C = C; g.ldc = ldc;
  g.alpha = alpha; g.beta = beta; g.transA = transA; g.transB = transB;
  g.a_tri = a_tri; g.b_tri = b_tri; g.c_uplo = c_uplo; g.batch = 1;
  return gemm<T>(g, s);
}

}  // namespace bse
