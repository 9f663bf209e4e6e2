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
#include "../../include/bse_stages.h"

namespace bse {

constexpr int BT_NB = 64;

template <typename T>
struct BtWork {
  T *Vb, *Z, *Z2, *G, *Tf, *Fre, *Fim, *Vsf;
};

static inline size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

template <typename T>
size_t bt_worksize(int m) {
  const size_t n = m / 2;
  size_t b = 3 * al256(sizeof(T) * (size_t)m * BT_NB) + 2 * al256(sizeof(T) * BT_NB * BT_NB);
  b += 2 * al256(sizeof(T) * (size_t)m * n);
  if (sizeof(T) == 4) b += al256(sizeof(T) * (size_t)m * n);
  return b;
}

template <typename T>
static BtWork<T> carve_bt(void* work, int m) {
  const size_t n = m / 2;
  char* p = reinterpret_cast<char*>(work);
  BtWork<T> w;
  w.Vb = (T*)p; p += al256(sizeof(T) * (size_t)m * BT_NB);
  w.Z = (T*)p; p += al256(sizeof(T) * (size_t)m * BT_NB);
  w.Z2 = (T*)p; p += al256(sizeof(T) * (size_t)m * BT_NB);
  w.G = (T*)p; p += al256(sizeof(T) * BT_NB * BT_NB);
  w.Tf = (T*)p; p += al256(sizeof(T) * BT_NB * BT_NB);
  w.Fre = (T*)p; p += al256(sizeof(T) * (size_t)m * n);
  w.Fim = (T*)p; p += al256(sizeof(T) * (size_t)m * n);
  w.Vsf = (sizeof(T) == 4) ? (T*)p : nullptr;
  return w;
}

// Vb[r, t] = v_{j0+t}[r] = W[r, j0+t] for r >= j0+t+1, else 0.
template <typename T>
__global__ void bt_copy_panel(int m, int j0, int nbp, const T* __restrict__ W, long ldw, T* __restrict__ Vb) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const int t = blockIdx.y;
  if (r >= m) return;
  T v = T(0);
  if (t < nbp && r >= j0 + t + 1) v = W[r + (long)(j0 + t) * ldw];
  Vb[r + (long)t * m] = v;
}

// Forward, column-wise triangular factor of a block of reflectors (the
// compact-WY representation H_0 ... H_{k-1} = I - V T V^T), from G = V^T V.
template <typename T>
__global__ void bt_larft(int k, const T* __restrict__ G, const T* __restrict__ tau, T* __restrict__ Tf) {
  __shared__ double Ts[BT_NB][BT_NB + 1];
  __shared__ double w[BT_NB];
  const int tid = threadIdx.x;
  for (int e = tid; e < BT_NB * BT_NB; e += blockDim.x) Ts[e % BT_NB][e / BT_NB] = 0.0;
  __syncthreads();
  for (int i = 0; i < k; ++i) {
    const double ti = (double)tau[i];
    if (tid < i) w[tid] = -ti * (double)G[tid + (long)i * BT_NB];
    __syncthreads();
    if (tid < i) {
      double s = 0.0;
      for (int l = tid; l < i; ++l) s += Ts[tid][l] * w[l];
      Ts[tid][i] = s;
    }
    if (tid == 0) Ts[i][i] = ti;
    __syncthreads();
  }
  for (int e = tid; e < BT_NB * BT_NB; e += blockDim.x) Tf[e] = (T)Ts[e % BT_NB][e / BT_NB];
}

// Phi starts as L: clear the strict upper triangle (it may still hold M).
template <typename T>
__global__ void bt_zero_upper(int m, T* __restrict__ L, long ldl) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i < j) L[i + (long)j * ldl] = T(0);
}

template <typename T>
__global__ void to_float_kernel(long count, const double* __restrict__ src, T* __restrict__ dst) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i < count; i += (long)gridDim.x * blockDim.x) dst[i] = (T)src[i];
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
                  const double* lam, double* X, double* Y, long ldx, void* work, cudaStream_t s) {
  const int n = m / 2;
  BtWork<T> w = carve_bt<T>(work, m);
  {
    KprofScope ks(K_ELEMENTWISE, s, 0.5 * sizeof(T) * m * (double)m, 0.0);
    bt_zero_upper<T><<<dim3(ceil_div(m, 256), m), 256, 0, s>>>(m, L, ldl);
  }
  BSE_LAUNCH_CHECK();
  const int nref = m - 1;  // reflectors j = 0..m-2 act on rows/cols j+1..m-1
  for (int j0 = 0; j0 < nref; j0 += BT_NB) {
    const int nbp = min(BT_NB, nref - j0);
    const int rows = m - j0 - 1;
    {
      KprofScope ks(K_ELEMENTWISE, s, 2.0 * sizeof(T) * m * BT_NB, 0.0);
      bt_copy_panel<T><<<dim3(ceil_div(m, 256), BT_NB), 256, 0, s>>>(m, j0, nbp, W, ldw, w.Vb);
    }
    BSE_LAUNCH_CHECK();
    // G = V^T V
    BSE_TRY(gemm<T>(nbp, nbp, rows, 1.0, w.Vb + j0 + 1, m, true, w.Vb + j0 + 1, m, false, 0.0, w.G, BT_NB, s));
    {
      KprofScope ks(K_ELEMENTWISE, s, 0.0, 0.0);
      bt_larft<T><<<1, BT_NB, 0, s>>>(nbp, w.G, tau + j0, w.Tf);
    }
    BSE_LAUNCH_CHECK();
    T* Phi = L + (long)(j0 + 1) * ldl;  // columns j0+1..m-1
    // Z = Phi V ; Z2 = Z T ; Phi -= Z2 V^T
    BSE_TRY(gemm<T>(m, nbp, rows, 1.0, Phi, ldl, false, w.Vb + j0 + 1, m, false, 0.0, w.Z, m, s));
    BSE_TRY(gemm<T>(m, nbp, nbp, 1.0, w.Z, m, false, w.Tf, BT_NB, false, 0.0, w.Z2, m, s, TRI_NONE, TRI_UPPER));
    BSE_TRY(gemm<T>(m, rows, nbp, -1.0, w.Z2, m, false, w.Vb + j0 + 1, m, true, 1.0, Phi, ldl, s));
  }
  const T* Vsx;
  if (sizeof(T) == 4) {
    {
      KprofScope ks(K_ELEMENTWISE, s, 12.0 * m * (double)n, 0.0);
      to_float_kernel<T><<<1024, 256, 0, s>>>((long)m * n, Vs, w.Vsf);
    }
    BSE_LAUNCH_CHECK();
    Vsx = w.Vsf;
  } else {
    Vsx = reinterpret_cast<const T*>(Vs);
  }
  // F_re = Phi[:, even] Vs[even, :],  F_im = Phi[:, odd] Vs[odd, :]
  BSE_TRY(gemm<T>(m, n, n, 1.0, L, 2 * ldl, false, Vsx, 2L * n, true, 0.0, w.Fre, m, s));
  BSE_TRY(gemm<T>(m, n, n, 1.0, L + ldl, 2 * ldl, false, Vsx + n, 2L * n, true, 0.0, w.Fim, m, s));
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
                                   const double*, double*, double*, long, void*, cudaStream_t);
template int backtransform<float>(int, float*, long, const float*, long, const float*, const double*,
                                  const double*, double*, double*, long, void*, cudaStream_t);

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
                                     work, (cudaStream_t)stream);
  return bse::backtransform<double>(m, (double*)L, ldl, (const double*)W, ldw, (const double*)tau, Vs, lam, X, Y,
                                    ldx, work, (cudaStream_t)stream);
}
