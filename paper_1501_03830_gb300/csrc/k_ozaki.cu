// FP64-accurate GEMM on the bf16 tensor cores by error-free digit splitting
// (the Ozaki scheme: Ozaki, Ogita, Oishi, Rump, Numer. Algorithms 59, 2012).
//
//   C = A B,   A_ik = sigma_i sum_p a^(p)_ik 2^{-beta (p+1)},
//              B_kj = tau_j   sum_q b^(q)_kj 2^{-beta (q+1)}
//
// sigma_i, tau_j are powers of two bounding row i of A and column j of B, and
// the digits a^(p), b^(q) are integers with |digit| <= 2^beta, exactly
// representable in bf16. beta is chosen so that K * 2^(2 beta) <= 2^24: every
// dot product of two digit vectors is then an integer below 2^24, which the
// tensor cores' FP32 accumulation holds exactly whatever the summation order.
// Each digit pair (p, q) with p + q < s is one tensor-core pass; the epilogue
// accumulates sigma_i tau_j 2^{-beta (p+q+2)} x (exact integer) in FP64. With s
// digits per operand the result carries about beta*s bits relative to
// sigma_i tau_j.
//
// Layout: A is given K-major (row i of A is A[i * lda + k], k contiguous; for a
// symmetric matrix stored column-major that is the matrix itself), B column-
// major (column j is B[j * ldb + k]). Digit matrices are stored K-major with
// the K pitch rounded up to 64 and zero padding.
#include <cuda_bf16.h>
#include <math.h>

#include "common.cuh"
#include "tcgemm.cuh"

namespace bse {

static inline size_t al256o(size_t b) { return (b + 255) & ~(size_t)255; }

struct OzakiPlan {
  int M, N, K, ldk, beta, s;
};

static OzakiPlan plan(int M, int N, int K, int s) {
  OzakiPlan p;
  p.M = M; p.N = N; p.K = K;
  p.ldk = (K + 63) / 64 * 64;
  // K * 2^(2 beta) <= 2^24
  int lk = 0;
  while ((1L << lk) < (long)p.ldk) ++lk;
  p.beta = (24 - lk) / 2;
  if (p.beta > 7) p.beta = 7;
  if (p.beta < 1) p.beta = 1;
  p.s = s;
  return p;
}

int ozaki_digits(int K) {
  const OzakiPlan p = plan(1, 1, K, 1);
  return (50 + p.beta - 1) / p.beta;
}

size_t ozaki_worksize(int M, int N, int K, int s) {
  OzakiPlan p = plan(M, N, K, s);
  return al256o((size_t)2 * s * M * p.ldk) + al256o((size_t)2 * s * N * p.ldk) + al256o(8 * (size_t)M) +
         al256o(8 * (size_t)N);
}

// One block per K-vector (row of A or column of B): power-of-two scale and digits.
__global__ void __launch_bounds__(256) ozaki_split(const double* __restrict__ X, long ldx, int K, int ldk, int beta,
                                                   int s, long digit_stride, __nv_bfloat16* __restrict__ D,
                                                   double* __restrict__ scale) {
  __shared__ double red[8];
  const long v = blockIdx.x;
  const double* x = X + v * ldx;
  double mx = 0.0;
  for (int k = threadIdx.x; k < K; k += 256) mx = fmax(mx, fabs(x[k]));
  for (int o = 16; o >= 1; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  mx = 0.0;
  for (int w = 0; w < 8; ++w) mx = fmax(mx, red[w]);
  int e = 0;
  if (mx > 0.0) frexp(mx, &e);  // mx = f 2^e, f in [0.5, 1): |x| / 2^e < 1
  if (threadIdx.x == 0) scale[v] = ldexp(1.0, e);
  __nv_bfloat16* dv = D + v * (long)ldk;
  for (int k = threadIdx.x; k < ldk; k += 256) {
    double r = (k < K && mx > 0.0) ? ldexp(x[k], -e) : 0.0;
    for (int p = 0; p < s; ++p) {
      const double t = ldexp(r, beta);
      const double d = rint(t);
      r = t - d;  // exact
      dv[p * digit_stride + k] = __float2bfloat16_rn((float)d);
    }
  }
}

// C (M x N, column-major, ldc) = A B to FP64 accuracy. work: ozaki_worksize bytes.
int ozaki_gemm(int M, int N, int K, const double* A, long lda, const double* B, long ldb, double* C, long ldc, int s,
               void* work, bool split_A, int* status, cudaStream_t st) {
  if (M <= 0 || N <= 0) return BSE_OK;
  if (s < 1 || s * (s + 1) / 2 > tc::kMaxUnits) return BSE_ERR_ARG;
  const OzakiPlan p = plan(M, N, K, s);
  char* w = reinterpret_cast<char*>(work);
  __nv_bfloat16* dA = reinterpret_cast<__nv_bfloat16*>(w);
  w += al256o((size_t)2 * s * M * p.ldk);
  __nv_bfloat16* dB = reinterpret_cast<__nv_bfloat16*>(w);
  w += al256o((size_t)2 * s * N * p.ldk);
  double* rs = reinterpret_cast<double*>(w);
  w += al256o(8 * (size_t)M);
  double* cs = reinterpret_cast<double*>(w);
  if (split_A) {
    KprofScope ks(K_ELEMENTWISE, st, 8.0 * M * (double)K + 2.0 * s * M * (double)p.ldk, 0.0);
    ozaki_split<<<M, 256, 0, st>>>(A, lda, K, p.ldk, p.beta, s, (long)M * p.ldk, dA, rs);
  }
  BSE_LAUNCH_CHECK();
  {
    KprofScope ks(K_ELEMENTWISE, st, 8.0 * N * (double)K + 2.0 * s * N * (double)p.ldk, 0.0);
    ozaki_split<<<N, 256, 0, st>>>(B, ldb, K, p.ldk, p.beta, s, (long)N * p.ldk, dB, cs);
  }
  BSE_LAUNCH_CHECK();
  BSE_CUDA(cudaMemset2DAsync(C, ldc * sizeof(double), 0, (size_t)M * sizeof(double), N, st));
  tc::TcProblem pb{};
  pb.M = M; pb.N = N; pb.K = K; pb.ldk = p.ldk;
  pb.A = dA; pb.B = dB; pb.a_rows = M; pb.b_rows = N; pb.a_digits = s; pb.b_digits = s;
  int u = 0;
  for (int a = 0; a < s; ++a)
    for (int b = 0; a + b < s; ++b) {
      pb.a_digit[u] = a;
      pb.b_digit[u] = b;
      pb.unit_scale[u] = ldexp(1.0, -p.beta * (a + b + 2));
      ++u;
    }
  pb.units = u;
  pb.mode = 1; pb.Cd = C; pb.ldc = ldc; pb.rs = rs; pb.cs = cs; pb.status = status;
  return tc::tc_gemm(pb, st);
}

}  // namespace bse

extern "C" size_t bse_ozaki_worksize(int M, int N, int K, int s) { return bse::ozaki_worksize(M, N, K, s); }

// C (M x N FP64, column-major, ldc) = A B with A K-major (row i at A + i*lda),
// B column-major (column j at B + j*ldb), to about 5*s bits beyond the row/column
// scales, on the tensor cores. work: bse_ozaki_worksize(M, N, K, s) bytes.
extern "C" int bse_ozaki_gemm(int M, int N, int K, const double* A, int lda, const double* B, int ldb, double* C,
                              int ldc, int s, void* work, int* dev_status, void* stream) {
  if (M < 1 || N < 1 || K < 1 || !A || !B || !C || lda < K || ldb < K || ldc < M || !work || !dev_status)
    return BSE_ERR_ARG;
  return bse::ozaki_gemm(M, N, K, A, lda, B, ldb, C, ldc, s, work, true, dev_status, (cudaStream_t)stream);
}
