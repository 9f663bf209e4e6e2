// FP64-accurate GEMM on the bf16 tensor cores by error-free digit splitting
// (the Ozaki scheme: Ozaki, Ogita, Oishi, Rump, Numer. Algorithms 59, 2012).
//
//   C = A B,   A_ik = sigma_i sum_p a^(p)_ik 2^{-beta (p+1)},
//              B_kj = tau_j   sum_q b^(q)_kj 2^{-beta (q+1)}
//
// sigma_i, tau_j are powers of two (one above the magnitude of row i of A and
// column j of B), and the digits a^(p), b^(q) are integers with
// |digit| <= 2^(beta-1), exactly representable in bf16. The tensor cores
// accumulate a digit pair's products in FP32 over chunks of Kc = 256 (kTcChunkK)
// reduction steps; beta is chosen so that Kc * 2^(2 beta - 2) <= 2^22: every
// chunk sum is then an integer the FP32 accumulation holds exactly whatever its
// summation order, and the epilogue adds the chunk sums in 32-bit integers (which
// bounds the whole-K sum of one anti-diagonal of pairs below 2^31, a second
// condition on beta). Each digit pair (p, q) with p + q < s is one tensor-core
// pass; the pairs of one anti-diagonal p + q = d share their scale and their
// integer sum, and the epilogue adds sigma_i tau_j 2^{-beta (d+2)} x (exact
// integer) to C in FP64. With s digits per operand the result carries about
// beta*s - 1 bits relative to the magnitudes of the row and column (beta = 8 for
// K = 16384 up to 7 digits: 55 bits with 28 pairs).
//
// Layout: A is given K-major (row i of A is A[i * lda + k], k contiguous; for a
// symmetric matrix stored column-major that is the matrix itself), B column-
// major (column j is B[j * ldb + k]). Digit matrices are stored K-major with
// the K pitch rounded up to 64 and zero padding.
#include <cuda_bf16.h>
#include <math.h>

#include "common.cuh"
#include "internal.cuh"
#include "tcgemm.cuh"

namespace bse {

static inline size_t al256o(size_t b) { return (b + 255) & ~(size_t)255; }

struct OzakiPlan {
  int M, N, K, ldk, beta, s;
};

constexpr int kTcChunkK = 256;  // reduction steps per exact FP32 chunk (4 blocks of 64)
constexpr int kMaxDigits = 11;  // s (s + 1) / 2 <= kMaxUnits

static int ceil_log2(long x) {
  int l = 0;
  while ((1L << l) < x) ++l;
  return l;
}

// Exactness conditions for beta with s digits per operand (every digit bounded by
// 2^(beta-1), so every digit product by 2^(2 beta - 2)): a chunk of Kc products
// sums to at most Kc 2^(2 beta - 2) <= 2^22 (exact in FP32 and convertible by the
// 1.5 * 2^23 shift), and one anti-diagonal's integer sum over the whole K (at
// most s pairs) stays below 2^31. bf16 holds every |digit| <= 2^8 exactly.
static bool beta_ok(int ldk, int beta, int s) {
  const int lkc = ceil_log2(ldk < kTcChunkK ? ldk : kTcChunkK);
  if (2 * beta - 2 > 22 - lkc) return false;
  return (double)ldk * ldexp(1.0, 2 * beta - 2) * (double)s < 2147483648.0;
}

static OzakiPlan plan(int M, int N, int K, int s) {
  OzakiPlan p;
  p.M = M; p.N = N; p.K = K;
  p.ldk = (K + 63) / 64 * 64;
  p.beta = 8;
  while (p.beta > 1 && !beta_ok(p.ldk, p.beta, s)) --p.beta;
  p.s = s;
  return p;
}

// s digits of beta bits carry beta s - 1 bits (the leading digit is bounded by
// 2^(beta-1) like the others, see ozaki_split): the fewest digits for `bits`
int ozaki_digits(int K, int bits) {
  const int ldk = (K + 63) / 64 * 64;
  for (int beta = 8; beta >= 1; --beta) {
    const int s = (bits + 1 + beta - 1) / beta;
    if (beta_ok(ldk, beta, s)) return s;
  }
  return bits + 1;
}

// digits of A and B, their scales, and one int32 M x N plane per anti-diagonal
size_t ozaki_worksize(int M, int N, int K, int s) {
  OzakiPlan p = plan(M, N, K, s);
  return al256o((size_t)2 * s * M * p.ldk) + al256o((size_t)2 * s * N * p.ldk) + al256o(8 * (size_t)M) +
         al256o(8 * (size_t)N) + al256o((size_t)4 * s * M * N);
}

// Digits on the integer pipe (FP64 arithmetic is slow on this GPU): x / 2^e is
// first written as a 62-bit fixed-point integer X (bits below 2^-62 of the vector
// scale are dropped, far below the s*beta - 1 <= 63 bits kept), then digit p is X
// rounded at bit 62 - beta (p+1) and subtracted:
// X = sum_p d_p 2^(62 - beta (p+1)) + remainder, the balanced digits of the
// scheme with |d_p| <= 2^(beta-1) for p > 0. The scale 2^e is one power of two
// above the vector's magnitude (|x| / 2^e < 1/2, so |X| < 2^61), which bounds the
// leading digit by 2^(beta-1) too: every digit product is then <= 2^(2 beta - 2),
// and beta = 8 keeps the 256-long chunk sums within 2^22.
__device__ __forceinline__ long long fixed62(double x, int e) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7ff);
  if (ex == 0) return 0;  // zero or subnormal: below every digit
  const long long mant = (long long)((b & 0xfffffffffffffULL) | 0x10000000000000ULL);
  // x = mant 2^(ex - 1075), so X = x 2^(62 - e) = mant 2^(ex - 1013 - e), shift <= 9
  const int sh = ex - 1013 - e;
  long long X = sh >= 0 ? (mant << sh) : (sh > -63 ? (mant >> -sh) : 0);
  return (b >> 63) ? -X : X;
}
__device__ __forceinline__ long long fixed62(float x, int e) { return fixed62((double)x, e); }

__device__ __forceinline__ void put_digits(long long X, int beta, int s, long digit_stride,
                                           __nv_bfloat16* __restrict__ d) {
  for (int p = 0; p < s; ++p) {
    const int sh = 62 - beta * (p + 1);
    long long q = 0;  // digits past the 62 fixed-point bits are zero
    if (sh > 0) {
      q = (X + (1LL << (sh - 1))) >> sh;  // round to nearest (ties up)
      X -= q << sh;
    }
    d[p * digit_stride] = __int2bfloat16_rn((int)q);
  }
}

// exponent e with max |x| < 2^e (frexp convention), from the largest magnitude's bits
__device__ __forceinline__ int scale_exp(unsigned long long maxbits) {
  if (maxbits == 0) return 0;
  int e = 0;
  frexp(__longlong_as_double((long long)maxbits), &e);
  return e;
}

// One block per K-vector (row of A or column of B): power-of-two scale and digits.
// Vector v is X[v * ldx + k] (k contiguous).
template <typename TI>
__global__ void __launch_bounds__(256) ozaki_split(const TI* __restrict__ X, long ldx, int K, int ldk, int beta,
                                                   int s, long digit_stride, __nv_bfloat16* __restrict__ D,
                                                   double* __restrict__ scale) {
  __shared__ unsigned long long red[8];
  const long v = blockIdx.x;
  const TI* x = X + v * ldx;
  // max |x| on the bit patterns (non-negative doubles order like their bits)
  unsigned long long mx = 0;
  for (int k = threadIdx.x; k < K; k += 256) {
    const unsigned long long b = (unsigned long long)__double_as_longlong((double)x[k]) & 0x7fffffffffffffffULL;
    mx = b > mx ? b : mx;
  }
  for (int o = 16; o >= 1; o >>= 1) {
    const unsigned long long y = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = y > mx ? y : mx;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  mx = 0;
  for (int w = 0; w < 8; ++w) mx = red[w] > mx ? red[w] : mx;
  const int e = scale_exp(mx) + 1;  // |x| / 2^e < 1/2
  if (threadIdx.x == 0) scale[v] = ldexp(1.0, e);
  __nv_bfloat16* dv = D + v * (long)ldk;
  for (int k = threadIdx.x; k < ldk; k += 256) {
    const long long F = (k < K && mx) ? fixed62(x[k], e) : 0;
    put_digits(F, beta, s, digit_stride, dv + k);
  }
}

// Same for vectors stored with stride: vector v is X[v + k * ldx] (rows of a
// column-major matrix). 32 vectors per block, staged through shared memory so
// reads and digit writes are both coalesced.
template <typename TI>
__global__ void __launch_bounds__(256) ozaki_split_rows(const TI* __restrict__ X, long ldx, int V, int K, int ldk,
                                                        int beta, int s, long digit_stride,
                                                        __nv_bfloat16* __restrict__ D, double* __restrict__ scale) {
  __shared__ double tile[64][33];
  __shared__ unsigned long long vmax[8][32];
  __shared__ int vexp[32];
  const int v0 = blockIdx.x * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 8 x 32
  // pass 1: per-vector max on the bit patterns
  unsigned long long mx = 0;
  if (v0 + tx < V)
    for (int k = ty; k < K; k += 8) {
      const unsigned long long b =
          (unsigned long long)__double_as_longlong((double)X[(v0 + tx) + (long)k * ldx]) & 0x7fffffffffffffffULL;
      mx = b > mx ? b : mx;
    }
  vmax[ty][tx] = mx;
  __syncthreads();
  if (ty == 0) {
    unsigned long long m2 = 0;
    for (int w = 0; w < 8; ++w) m2 = vmax[w][tx] > m2 ? vmax[w][tx] : m2;
    const int e = scale_exp(m2) + 1;  // |x| / 2^e < 1/2
    vexp[tx] = m2 ? e : 1000000;  // 1e6 marks an all-zero vector
    if (v0 + tx < V) scale[v0 + tx] = ldexp(1.0, m2 ? e : 0);
  }
  __syncthreads();
  // pass 2: digits, 64 k at a time
  for (int k0 = 0; k0 < ldk; k0 += 64) {
    for (int kk = ty; kk < 64; kk += 8) {
      const int k = k0 + kk;
      tile[kk][tx] = (v0 + tx < V && k < K) ? (double)X[(v0 + tx) + (long)k * ldx] : 0.0;
    }
    __syncthreads();
    // thread (ty, tx) writes vectors ty, ty+8, ... at k = k0 + 2 tx, k0 + 2 tx + 1
    for (int vv = ty; vv < 32; vv += 8) {
      if (v0 + vv >= V) continue;
      const int e = vexp[vv];
      __nv_bfloat16* dv = D + (long)(v0 + vv) * ldk + k0;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int kk = 2 * tx + h;
        const long long F = (e == 1000000) ? 0 : fixed62(tile[kk][vv], e);
        put_digits(F, beta, s, digit_stride, dv + kk);
      }
    }
    __syncthreads();
  }
}

// C (+)= sigma_i tau_j sum_d 2^{-beta (d+2)} S_d(i, j): the G anti-diagonal
// integer sums S_d (int32 planes, M x N column-major, ld M) scaled and added in
// FP64, smallest terms first (Horner in 2^-beta, exact power-of-two steps).
__global__ void __launch_bounds__(256) ozaki_combine(int M, int N, int G, const int* __restrict__ S, long plane,
                                                     const double* __restrict__ rs, const double* __restrict__ cs,
                                                     int beta, double* __restrict__ C, long ldc, int accumulate) {
  const int i = blockIdx.x * 256 + threadIdx.x;
  if (i >= M) return;
  const double step = __longlong_as_double((long long)(1023 - beta) << 52);       // 2^-beta
  const double tail = __longlong_as_double((long long)(1023 - 2 * beta) << 52);   // 2^-2 beta
  const double ri = rs[i] * tail;
  for (int j = blockIdx.y; j < N; j += gridDim.y) {
    const int* sp = S + i + (long)j * M;
    double t = 0.0;
    for (int g = G - 1; g >= 0; --g) t = fma(t, step, (double)sp[g * plane]);
    const double v = t * (ri * cs[j]);
    double* cp = C + i + (long)j * ldc;
    *cp = accumulate ? *cp + v : v;
  }
}

// Generic digit-split product C (M x N, column-major, ldc) (+)= A B on the
// tensor cores. Operand descriptions: A rows are K-vectors at A + i*lda
// (a_rows_strided: A[i + k*lda] instead), B columns are K-vectors at B + j*ldb
// (b_strided: B[j + k*ldb]); element types double or float (a_f32 / b_f32).
// accumulate: add to C instead of overwriting it. split_A = false reuses the A
// digits already in the workspace (same A, same K, same s).
int ozaki_gemm_ex(const OzOperand& A, const OzOperand& B, int M, int N, int K, double* C, long ldc, int s,
                  bool accumulate, void* work, bool split_A, int* status, cudaStream_t st, int s_use) {
  if (M <= 0 || N <= 0) return BSE_OK;
  if (s < 1 || s > kMaxDigits || s * (s + 1) / 2 > tc::kMaxUnits) return BSE_ERR_ARG;
  if (s_use <= 0 || s_use > s) s_use = s;
  const OzakiPlan p = plan(M, N, K, s);
  char* w = reinterpret_cast<char*>(work);
  __nv_bfloat16* dA = reinterpret_cast<__nv_bfloat16*>(w);
  w += al256o((size_t)2 * s * M * p.ldk);
  __nv_bfloat16* dB = reinterpret_cast<__nv_bfloat16*>(w);
  w += al256o((size_t)2 * s * N * p.ldk);
  double* rs = reinterpret_cast<double*>(w);
  w += al256o(8 * (size_t)M);
  double* cs = reinterpret_cast<double*>(w);
  auto split = [&](const OzOperand& X, int V, __nv_bfloat16* D, double* scl, int s) -> int {
    const double bytes = (X.f32 ? 4.0 : 8.0) * V * (double)K + 2.0 * s * V * (double)p.ldk;
    KprofScope ks(K_ELEMENTWISE, st, bytes, 0.0);
    const long dstride = (long)V * p.ldk;
    if (!X.strided) {
      if (X.f32)
        ozaki_split<float><<<V, 256, 0, st>>>((const float*)X.ptr, X.ld, K, p.ldk, p.beta, s, dstride, D, scl);
      else
        ozaki_split<double><<<V, 256, 0, st>>>((const double*)X.ptr, X.ld, K, p.ldk, p.beta, s, dstride, D, scl);
    } else {
      const int blocks = ceil_div(V, 32);
      if (X.f32)
        ozaki_split_rows<float><<<blocks, 256, 0, st>>>((const float*)X.ptr, X.ld, V, K, p.ldk, p.beta, s, dstride, D,
                                                        scl);
      else
        ozaki_split_rows<double><<<blocks, 256, 0, st>>>((const double*)X.ptr, X.ld, V, K, p.ldk, p.beta, s, dstride,
                                                         D, scl);
    }
    BSE_LAUNCH_CHECK();
    return BSE_OK;
  };
  // A keeps all s digits (later calls may reuse them with more digits); B only
  // needs the s_use digits this product pairs
  if (split_A) BSE_TRY(split(A, M, dA, rs, s));
  BSE_TRY(split(B, N, dB, cs, s_use));
  int* planes = reinterpret_cast<int*>(w + al256o(8 * (size_t)N));
  tc::TcProblem pb{};
  pb.M = M; pb.N = N; pb.K = K; pb.ldk = p.ldk;
  pb.A = dA; pb.B = dB; pb.a_rows = M; pb.b_rows = N; pb.a_digits = s; pb.b_digits = s;
  pb.chunk_kb = kTcChunkK / 64;
  // pairs ordered by anti-diagonal d = a + b; the last pair of each closes plane d
  int u = 0;
  for (int d = 0; d < s_use; ++d)
    for (int a = 0; a <= d; ++a) {
      pb.a_digit[u] = a;
      pb.b_digit[u] = d - a;
      pb.fold[u] = a == d;
      ++u;
    }
  pb.units = u;
  pb.mode = 1; pb.Si = planes; pb.plane = (long)M * N; pb.ldc = M; pb.status = status;
  BSE_TRY(tc::tc_gemm(pb, st));
  {
    KprofScope ks(K_ELEMENTWISE, st, 4.0 * s_use * M * (double)N + (accumulate ? 16.0 : 8.0) * M * (double)N, 0.0);
    const dim3 grid((unsigned)ceil_div(M, 256), (unsigned)(N < 65535 ? N : 65535));
    ozaki_combine<<<grid, 256, 0, st>>>(M, N, s_use, planes, (long)M * N, rs, cs, p.beta, C, ldc, accumulate ? 1 : 0);
    BSE_LAUNCH_CHECK();
  }
  return BSE_OK;
}

// C (M x N, column-major, ldc) = A B to FP64 accuracy. work: ozaki_worksize bytes.
int ozaki_gemm(int M, int N, int K, const double* A, long lda, const double* B, long ldb, double* C, long ldc, int s,
               void* work, bool split_A, int* status, cudaStream_t st, int s_use) {
  OzOperand a{A, lda, false, false}, b{B, ldb, false, false};
  return ozaki_gemm_ex(a, b, M, N, K, C, ldc, s, false, work, split_A, status, st, s_use);
}

}  // namespace bse

extern "C" size_t bse_ozaki_worksize(int M, int N, int K, int s) { return bse::ozaki_worksize(M, N, K, s); }

extern "C" int bse_ozaki_digit_bits(int K) { return K < 1 ? BSE_ERR_ARG : bse::plan(1, 1, K, 1).beta; }

// C (M x N FP64, column-major, ldc) = A B with A K-major (row i at A + i*lda),
// B column-major (column j at B + j*ldb), to about beta*s - 1 bits beyond the
// row/column magnitudes (beta = bse_ozaki_digit_bits(K) for s up to the bound
// that keeps one anti-diagonal's integer sum below 2^31), on the tensor cores.
// work: bse_ozaki_worksize(M, N, K, s) bytes.
extern "C" int bse_ozaki_gemm(int M, int N, int K, const double* A, int lda, const double* B, int ldb, double* C,
                              int ldc, int s, void* work, int* dev_status, void* stream) {
  if (M < 1 || N < 1 || K < 1 || !A || !B || !C || lda < K || ldb < K || ldc < M || !work || !dev_status)
    return BSE_ERR_ARG;
  return bse::ozaki_gemm(M, N, K, A, lda, B, ldb, C, ldc, s, work, true, dev_status, (cudaStream_t)stream);
}
