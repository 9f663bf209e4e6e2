// Algorithm 3 steps 3-6 (with the Lambda+^{-1/2} of Algorithm 1 step 5):
//
//   Phi = L U,  U = H_0 H_1 ... H_{m-2}        (step 3: reflectors applied to L
//                                               from the right in compact-WY
//                                               blocks I - V T V^T, in place)
//   Y+  = Q Phi D V+                            (steps 4-5)
//   X   = diag(I,-I) Y+ Lambda+^{-1/2},  Y = diag(I,-I) X   (step 6, Theorem 3)
//
// Remark 3 (Q and D applied in O(n^2)) and remark 4 (real GEMMs instead of a
// complex one) are taken one step further: D V+ has purely real even rows and
// purely imaginary odd rows (0-based), so
//   Phi D V+ = Phi[:, even] Vs[even, :] + i Phi[:, odd] Vs[odd, :]
// with Vs the sign-folded V+ from the tridiagonal eigensolver: two m x n x n
// GEMMs (8n^3 flops) instead of 16n^3. Q, the signs and the Lambda scaling are
// one elementwise epilogue that writes X and Y as interleaved complex128.
#include "common.cuh"
#include "gemm_simt.cuh"
#include "internal.cuh"
#include "../../include/bse_stages.h"

namespace bse {

constexpr int BT_NB = 64;
// rows of V per block of the Gram kernel (33 KiB of shared memory either way)
template <typename T>
constexpr int gram_rows() { return sizeof(T) == 4 ? 128 : 64; }

// Panel buffers (Vb, Z, Z2) have a leading dimension of m rounded up to 32 and the
// FP32 copy of Vs a row pitch of n rounded up to 32, so that every operand of the
// tensor-core products starts on a 16-byte boundary with a pitch divisible by 4.
static inline long bt_ld(long x) { return (x + 31) / 32 * 32; }

template <typename T>
struct BtWork {
  T *Vb, *Z, *Z2, *G, *Gpart, *Tf, *Fre, *Fim, *Vsf;
  void* oz;  // digit-split product workspace (FP64 path)
  long ldv, ldvs;
};

static inline size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

// The FP64 path's two m x n x n eigenvector products run FP64-accurate on the
// bf16 tensor cores (digit-split product) from this size on; below it, and for
// every FP32 product, the GEMM kernels.
constexpr int BT_OZAKI_MIN_N = 256;

template <typename T>
size_t bt_worksize(int m) {
  const size_t n = m / 2;
  const size_t ldv = bt_ld(m), parts = (size_t)ceil_div(m, gram_rows<T>());
  size_t b = 3 * al256(sizeof(T) * ldv * BT_NB) + 2 * al256(sizeof(T) * BT_NB * BT_NB);
  b += al256(sizeof(double) * parts * BT_NB * BT_NB);
  b += 2 * al256(sizeof(T) * (size_t)m * n);
  if (sizeof(T) == 4) b += al256(sizeof(T) * (size_t)m * bt_ld(n));
  if (sizeof(T) == 8 && (int)n >= BT_OZAKI_MIN_N) b += al256(ozaki_worksize(m, (int)n, (int)n, ozaki_digits((int)n)));
  return b;
}

template <typename T>
static BtWork<T> carve_bt(void* work, int m) {
  const size_t n = m / 2;
  BtWork<T> w;
  w.ldv = bt_ld(m);
  w.ldvs = sizeof(T) == 4 ? bt_ld(n) : (long)n;
  const size_t parts = (size_t)ceil_div(m, gram_rows<T>());
  char* p = reinterpret_cast<char*>(work);
  w.Vb = (T*)p; p += al256(sizeof(T) * w.ldv * BT_NB);
  w.Z = (T*)p; p += al256(sizeof(T) * w.ldv * BT_NB);
  w.Z2 = (T*)p; p += al256(sizeof(T) * w.ldv * BT_NB);
  w.G = (T*)p; p += al256(sizeof(T) * BT_NB * BT_NB);
  w.Tf = (T*)p; p += al256(sizeof(T) * BT_NB * BT_NB);
  w.Gpart = (T*)p; p += al256(sizeof(double) * parts * BT_NB * BT_NB);
  w.Fre = (T*)p; p += al256(sizeof(T) * (size_t)m * n);
  w.Fim = (T*)p; p += al256(sizeof(T) * (size_t)m * n);
  w.Vsf = (sizeof(T) == 4) ? (T*)p : nullptr;
  if (sizeof(T) == 4) p += al256(sizeof(T) * (size_t)m * bt_ld(n));
  w.oz = p;
  return w;
}

// Panel of reflectors j0 .. j0+nbp-1 restricted to rows j0+off .. m-1 (reflector j
// starts at row j+off with its explicit unit entry; off = 1 for Algorithm 3's
// reduction, b for the band reduction's first stage): Vb[r, t] =
// v_{j0+t}[j0+off+r] = W[j0+off+r, j0+t] for r >= t, else 0.
template <typename T>
__global__ void bt_copy_panel(int m, int j0, int off, int nbp, const T* __restrict__ W, long ldw,
                              T* __restrict__ Vb, long ldv) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const int t = blockIdx.y;
  if (r >= ldv) return;
  T v = T(0);
  if (t < nbp && r >= t && j0 + off + r < m) v = W[j0 + off + r + (long)(j0 + t) * ldw];
  Vb[r + (long)t * ldv] = v;
}

// G = V^T V over row blocks: block b writes the partial Gram matrix of its
// gram_rows<T>() rows (accumulated in T); bt_gram_sum adds the partials in FP64.
template <typename T>
__global__ void __launch_bounds__(256) bt_gram_part(int rows, const T* __restrict__ Vb, long ldv,
                                                     double* __restrict__ Gpart) {
  constexpr int R = gram_rows<T>();
  __shared__ T sV[R][BT_NB + 1];
  const int r0 = blockIdx.x * R;
  for (int e = threadIdx.x; e < R * BT_NB; e += 256) {
    const int r = e % R, c = e / R;
    sV[r][c] = (r0 + r < rows) ? Vb[r0 + r + (long)c * ldv] : T(0);
  }
  __syncthreads();
  const int i = threadIdx.x & 63, jb = threadIdx.x >> 6;  // columns jb, jb+4, ..., jb+60
  T acc[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) acc[q] = T(0);
  for (int r = 0; r < R; ++r) {
    const T vi = sV[r][i];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = fma(vi, sV[r][jb + 4 * q], acc[q]);
  }
  double* out = Gpart + (size_t)blockIdx.x * BT_NB * BT_NB;
#pragma unroll
  for (int q = 0; q < 16; ++q) out[i + (jb + 4 * q) * BT_NB] = (double)acc[q];
}

template <typename T>
__global__ void bt_gram_sum(int parts, const double* __restrict__ Gpart, T* __restrict__ G) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= BT_NB * BT_NB) return;
  double s = 0.0;
  for (int b = 0; b < parts; ++b) s += Gpart[(size_t)b * BT_NB * BT_NB + e];
  G[e] = (T)s;
}

// Forward, column-wise triangular factor of a block of reflectors (the
// compact-WY representation H_0 ... H_{k-1} = I - V T V^T), from G = V^T V.
// Computed in the path's precision T: on the mixed path its only consumers are
// FP32 products, and FP32 latency is a small fraction of FP64's on this GPU.
template <typename T>
__global__ void bt_larft(int k, const T* __restrict__ G, const T* __restrict__ tau, T* __restrict__ Tf) {
  __shared__ T Ts[BT_NB][BT_NB + 1];
  __shared__ T w[BT_NB];
  const int tid = threadIdx.x;
  for (int e = tid; e < BT_NB * BT_NB; e += blockDim.x) Ts[e % BT_NB][e / BT_NB] = T(0);
  __syncthreads();
  for (int i = 0; i < k; ++i) {
    const T ti = tau[i];
    if (tid < i) w[tid] = -ti * G[tid + (long)i * BT_NB];
    __syncthreads();
    if (tid < i) {
      T s = T(0);
      for (int l = tid; l < i; ++l) s += Ts[tid][l] * w[l];
      Ts[tid][i] = s;
    }
    if (tid == 0) Ts[i][i] = ti;
    __syncthreads();
  }
  for (int e = tid; e < BT_NB * BT_NB; e += blockDim.x) Tf[e] = Ts[e % BT_NB][e / BT_NB];
}

// Phi starts as L: clear the strict upper triangle (it may still hold M).
template <typename T>
__global__ void bt_zero_upper(int m, T* __restrict__ L, long ldl) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i < j) L[i + (long)j * ldl] = T(0);
}

// dst (rows x cols, row pitch ldd) = src (rows x cols, row pitch cols), converted.
template <typename T>
__global__ void to_float_kernel(long rows, int cols, const double* __restrict__ src, T* __restrict__ dst, long ldd) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i < rows * cols; i += (long)gridDim.x * blockDim.x) {
    const long r = i / cols, c = i - r * cols;
    dst[r * ldd + c] = (T)src[i];
  }
}

template <typename T>
__global__ void bt_epilogue(int n, const T* __restrict__ Fre, const T* __restrict__ Fim, long ldf,
                            const double* __restrict__ lam, double2* __restrict__ X, double2* __restrict__ Y,
                            long ldx) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= n) return;
  const double f1r = (double)Fre[i + (long)j * ldf], f2r = (double)Fre[n + i + (long)j * ldf];
  const double f1i = (double)Fim[i + (long)j * ldf], f2i = (double)Fim[n + i + (long)j * ldf];
  const double sc = rsqrt(2.0 * lam[j]);
  const double2 top = make_double2((f1r + f2i) * sc, (f1i - f2r) * sc);
  const double2 bot = make_double2((f1r - f2i) * sc, (f1i + f2r) * sc);
  if (X) {
    X[i + (long)j * ldx] = top;
    X[n + i + (long)j * ldx] = make_double2(-bot.x, -bot.y);
  }
  if (Y) {
    Y[i + (long)j * ldx] = top;
    Y[n + i + (long)j * ldx] = bot;
  }
}

template <typename T>
int backtransform(int m, T* L, long ldl, const T* W, long ldw, const T* tau, const double* Vs,
                  const double* lam, double* X, double* Y, long ldx, void* work, cudaStream_t s, int off,
                  void* sbr_work) {
  const int n = m / 2;
  BtWork<T> w = carve_bt<T>(work, m);
  {
    KprofScope ks(K_ELEMENTWISE, s, 0.5 * sizeof(T) * m * (double)m, 0.0);
    bt_zero_upper<T><<<dim3(ceil_div(m, 256), m), 256, 0, s>>>(m, L, ldl);
  }
  BSE_LAUNCH_CHECK();
  const int nref = m - off;  // reflectors j = 0..m-off-1 act on rows/cols j+off..m-1
  const long ldv = w.ldv;
  for (int j0 = 0; j0 < nref; j0 += BT_NB) {
    const int nbp = min(BT_NB, nref - j0);
    const int rows = m - j0 - off;
    {
      KprofScope ks(K_ELEMENTWISE, s, 2.0 * sizeof(T) * rows * BT_NB, 0.0);
      bt_copy_panel<T><<<dim3(ceil_div(ldv, 256), BT_NB), 256, 0, s>>>(m, j0, off, nbp, W, ldw, w.Vb, ldv);
    }
    BSE_LAUNCH_CHECK();
    // G = V^T V
    const int parts = ceil_div(rows, gram_rows<T>());
    {
      KprofScope ks(K_ELEMENTWISE, s, sizeof(T) * (double)rows * BT_NB, 2.0 * rows * (double)BT_NB * BT_NB);
      bt_gram_part<T><<<parts, 256, 0, s>>>(rows, w.Vb, ldv, reinterpret_cast<double*>(w.Gpart));
    }
    BSE_LAUNCH_CHECK();
    {
      KprofScope ks(K_ELEMENTWISE, s, 8.0 * parts * BT_NB * BT_NB, 0.0);
      bt_gram_sum<T><<<ceil_div(BT_NB * BT_NB, 256), 256, 0, s>>>(parts, reinterpret_cast<double*>(w.Gpart), w.G);
    }
    BSE_LAUNCH_CHECK();
    {
      KprofScope ks(K_ELEMENTWISE, s, 0.0, 0.0);
      bt_larft<T><<<1, BT_NB, 0, s>>>(nbp, w.G, tau + j0, w.Tf);
    }
    BSE_LAUNCH_CHECK();
    T* Phi = L + (long)(j0 + off) * ldl;  // columns j0+off..m-1
    // Z = Phi V ; Z2 = Z T ; Phi -= Z2 V^T
    BSE_TRY(gemm<T>(m, nbp, rows, 1.0, Phi, ldl, false, w.Vb, ldv, false, 0.0, w.Z, ldv, s));
    BSE_TRY(gemm<T>(m, nbp, nbp, 1.0, w.Z, ldv, false, w.Tf, BT_NB, false, 0.0, w.Z2, ldv, s, TRI_NONE, TRI_UPPER));
    BSE_TRY(gemm<T>(m, rows, nbp, -1.0, w.Z2, ldv, false, w.Vb, ldv, true, 1.0, Phi, ldl, s));
  }
  // the band reduction's second stage: Phi <- Phi Q2
  if (sbr_work) BSE_TRY(sbr_apply_q2(m, reinterpret_cast<float*>(L), ldl, sbr_work, s));
  const T* Vsx;
  long ldvs = n;
  if (sizeof(T) == 4) {
    {
      KprofScope ks(K_ELEMENTWISE, s, 12.0 * m * (double)n, 0.0);
      to_float_kernel<T><<<1024, 256, 0, s>>>((long)m, n, Vs, w.Vsf, w.ldvs);
    }
    BSE_LAUNCH_CHECK();
    Vsx = w.Vsf;
    ldvs = w.ldvs;
  } else {
    Vsx = reinterpret_cast<const T*>(Vs);
  }
  // F_re = Phi[:, even] Vs[even, :],  F_im = Phi[:, odd] Vs[odd, :]
  if (sizeof(T) == 8 && n >= BT_OZAKI_MIN_N) {
    // row i of Phi[:, even] is L[i + 2k ldl] (k = 0..n-1), column j of Vs[even, :]
    // is Vs[2k n + j]: both strided K-vectors
    int* zst = reinterpret_cast<int*>(current_status());
    const int sd = ozaki_digits(n);
    for (int h = 0; h < 2; ++h) {
      OzOperand a{L + h * ldl, 2 * ldl, true, false};
      OzOperand b{Vs + h * (long)n, 2L * n, true, false};
      BSE_TRY(ozaki_gemm_ex(a, b, m, n, n, reinterpret_cast<double*>(h ? w.Fim : w.Fre), m, sd, false, w.oz, true,
                            zst, s));
    }
  } else {
    BSE_TRY(gemm<T>(m, n, n, 1.0, L, 2 * ldl, false, Vsx, 2L * ldvs, true, 0.0, w.Fre, m, s));
    BSE_TRY(gemm<T>(m, n, n, 1.0, L + ldl, 2 * ldl, false, Vsx + ldvs, 2L * ldvs, true, 0.0, w.Fim, m, s));
  }
  {
    KprofScope ks(K_ELEMENTWISE, s, 2.0 * sizeof(T) * m * (double)n + 32.0 * m * (double)n, 0.0);
    bt_epilogue<T><<<dim3(ceil_div(n, 128), n), 128, 0, s>>>(n, w.Fre, w.Fim, m, lam, reinterpret_cast<double2*>(X),
                                                              reinterpret_cast<double2*>(Y), ldx);
  }
  BSE_LAUNCH_CHECK();
  return BSE_OK;
}

template size_t bt_worksize<double>(int);
template size_t bt_worksize<float>(int);
template int backtransform<double>(int, double*, long, const double*, long, const double*, const double*,
                                   const double*, double*, double*, long, void*, cudaStream_t, int, void*);
template int backtransform<float>(int, float*, long, const float*, long, const float*, const double*,
                                  const double*, double*, double*, long, void*, cudaStream_t, int, void*);

}  // namespace bse

extern "C" size_t bse_stage_backtransform_worksize(int m, int fp32) {
  return fp32 ? bse::bt_worksize<float>(m) : bse::bt_worksize<double>(m);
}

extern "C" int bse_stage_backtransform(int m, void* L, int ldl, const void* W, int ldw, const void* tau,
                                       const double* Vs, const double* lam, double* X, double* Y, int ldx,
                                       int fp32, void* work, void* stream) {
  if (m < 2 || (m & 1) || !L || !W || !tau || !Vs || !lam || ldl < m || ldw < m || ldx < m || !work)
    return BSE_ERR_ARG;
  if (fp32)
    return bse::backtransform<float>(m, (float*)L, ldl, (const float*)W, ldw, (const float*)tau, Vs, lam, X, Y, ldx,
                                     work, (cudaStream_t)stream, 1, nullptr);
  return bse::backtransform<double>(m, (double*)L, ldl, (const double*)W, ldw, (const double*)tau, Vs, lam, X, Y,
                                    ldx, work, (cudaStream_t)stream, 1, nullptr);
}
