// Host side of the C ABI: contexts, workspace cache, bse_solve / bse_spectrum.
//
// bse_solve runs Algorithm 1 with Algorithm 3 for its steps 4-5, every stage a
// kernel of this library on the context's stream:
//   form M -> Cholesky -> W -> skew tridiagonal reduction -> tridiagonal
//   eigensolve -> back-transform (-> FP64 refinement) (-> weights on request)
// Inputs and outputs may live on the host or the device; host data is staged
// through the workspace with one cudaMemcpyAsync per buffer.
#include <math.h>
#include <string.h>

#include <atomic>
#include <chrono>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.cuh"
#include "solver.h"

namespace bse {

static thread_local std::string g_last_error;

void record_error(const char* what, cudaError_t err, const char* file, int line) {
  char buf[512];
  snprintf(buf, sizeof(buf), "%s failed: %s (%s:%d)", what, cudaGetErrorString(err), file, line);
  g_last_error = buf;
}
void record_message(const char* msg) { g_last_error = msg; }

static inline size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// W's leading dimension, padded to 32 elements so 16-byte vector loads of its
// columns stay aligned whatever n is.
size_t w_ld(int n) { return ((2 * (size_t)n + 31) / 32) * 32; }

static std::atomic<int> g_band_min_m{0};

bool use_band_reduction(int m, int precision) {
  const int lim = g_band_min_m.load(std::memory_order_relaxed);
  return precision != BSE_FP64 && lim > 0 && m >= lim && m >= 4;
}

static std::atomic<int> g_tdeig_method{0};

bool use_mrrr() { return g_tdeig_method.load(std::memory_order_relaxed) == 1; }

size_t workspace_bytes(int n, int precision) {
  const size_t m = 2 * (size_t)n;
  const bool f32 = precision != BSE_FP64;
  const size_t ts = f32 ? 4 : 8;
  size_t b = 0;
  b += 2 * al256(16 * (size_t)n * n);         // A, B staging
  b += al256(8 * m * m);                       // M (FP64)
  if (f32) b += al256(4 * w_ld(n) * m);        // L (FP32, leading dimension padded)
  b += al256(ts * w_ld(n) * m);                // W (leading dimension padded)
  b += al256(8 * m) + al256(ts * m) + al256(8 * (size_t)n);  // e, tau, lambda
  b += al256(8 * m * n);                       // Vs
  b += 2 * al256(16 * m * n);                  // X, Y
  b += al256(64);                              // status
  if (use_band_reduction((int)m, precision)) b += al256(sbr_worksize((int)m));
  size_t scratch = f32 ? potrf_worksize<float>((int)m) : potrf_worksize<double>((int)m);
  scratch = std::max(scratch, f32 ? trd_worksize<float>((int)m) : trd_worksize<double>((int)m));
  scratch = std::max(scratch, sizeof(double) * (m + 8));
  if (!f32) scratch = std::max(scratch, tdeig_reorth_worksize((int)m));
  if (use_mrrr()) scratch = std::max(scratch, tdeig_mrrr_worksize((int)m, n));
  scratch = std::max(scratch, f32 ? bt_worksize<float>((int)m) : bt_worksize<double>((int)m));
  if (precision == BSE_MIXED_REFINED) scratch = std::max(scratch, refine_worksize(n));
  b += al256(scratch);
  return b;
}

int Workspace::init(int n_, int precision_) {
  precision = precision_;
  bytes = workspace_bytes(n_, precision);
  cudaError_t err = cudaMalloc(&base, bytes);
  if (err != cudaSuccess) {
    cudaGetLastError();
    base = nullptr;
    record_error("cudaMalloc(workspace)", err, __FILE__, __LINE__);
    return BSE_ERR_NOMEM;
  }
  carve(n_);
  return BSE_OK;
}

void Workspace::carve(int n_) {
  n = n_;
  const size_t m = 2 * (size_t)n;
  const bool f32 = precision != BSE_FP64;
  const size_t ts = f32 ? 4 : 8;
  char* p = (char*)base;
  auto take = [&](size_t sz) {
    void* r = p;
    p += al256(sz);
    return r;
  };
  A = (double*)take(16 * (size_t)n * n);
  B = (double*)take(16 * (size_t)n * n);
  M = (double*)take(8 * m * m);
  ldw = (int)w_ld(n);
  Lf = f32 ? (float*)take(4 * (size_t)ldw * m) : nullptr;
  W = take(ts * (size_t)ldw * m);
  e = (double*)take(8 * m);
  tau = take(ts * m);
  lam = (double*)take(8 * (size_t)n);
  Vs = (double*)take(8 * m * n);
  X = (double*)take(16 * m * n);
  Y = (double*)take(16 * m * n);
  status = (DevStatus*)take(64);
  sbr = use_band_reduction((int)m, precision) ? take(sbr_worksize((int)m)) : nullptr;
  scratch = p;
}

void Workspace::release() {
  if (base) cudaFree(base);
  base = nullptr;
}

}  // namespace bse

using namespace bse;

static const char* kVersion = "bse-gb300 0.1 (sm_103a)";

extern "C" const char* bse_last_error(void) { return g_last_error.c_str(); }
extern "C" const char* bse_version(void) { return kVersion; }

extern "C" int bse_create(bse_ctx** out, int device, size_t hbm_budget) {
  if (!out) return BSE_ERR_ARG;
  *out = nullptr;
  int count = 0;
  BSE_CUDA(cudaGetDeviceCount(&count));
  if (device < 0 || device >= count) {
    record_message("bse_create: no such CUDA device");
    return BSE_ERR_ARG;
  }
  BSE_CUDA(cudaSetDevice(device));
  bse_ctx* c = new bse_ctx();
  c->device = device;
  size_t fr = 0, tot = 0;
  BSE_CUDA(cudaMemGetInfo(&fr, &tot));
  c->budget = hbm_budget ? hbm_budget : (size_t)(0.9 * (double)fr);
  if (cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete c;
    record_message("bse_create: cudaStreamCreate failed");
    return BSE_ERR_CUDA;
  }
  c->stream = c->own_stream;
  for (int i = 0; i < 12; ++i) cudaEventCreate(&c->ev[i]);
  // kept solutions and host-staging buffers come from the device's default
  // memory pool; let it cache freed blocks instead of returning them at every
  // synchronisation (a process-local setting of this library's allocations)
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
    uint64_t keep_all = ~0ULL;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep_all);
  }
  *out = c;
  return BSE_OK;
}

extern "C" int bse_destroy(bse_ctx* c) {
  if (!c) return BSE_OK;
  bse_serve_stop(c, 60.0);
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  for (auto* sc : c->batch_slots) bse_destroy(sc);
  c->batch_slots.clear();
  for (auto& w : c->ws) w.release();
  c->ws.clear();
  for (int i = 0; i < 12; ++i) cudaEventDestroy(c->ev[i]);
  cudaStreamDestroy(c->own_stream);
  delete c;
  return BSE_OK;
}

extern "C" int bse_set_stream(bse_ctx* c, void* stream) {
  if (!c) return BSE_ERR_ARG;
  c->stream = stream ? (cudaStream_t)stream : c->own_stream;
  return BSE_OK;
}

extern "C" int bse_set_tdeig_method(int method) {
  if (method < 0 || method > 1) return BSE_ERR_ARG;
  bse::g_tdeig_method.store(method);
  return BSE_OK;
}

extern "C" int bse_set_band_reduction(int min_m) {
  if (min_m < 0) return BSE_ERR_ARG;
  bse::g_band_min_m.store(min_m);
  return BSE_OK;
}

extern "C" int bse_set_timing(bse_ctx* c, int on) {
  if (!c) return BSE_ERR_ARG;
  c->timing = on != 0;
  return BSE_OK;
}

namespace bse {

size_t ctx_bytes_held(bse_ctx* c) {
  size_t s = 0;
  for (auto& w : c->ws) s += w.bytes;
  return s;
}

// A cached workspace of the same precision whose allocation holds the layout
// for n (the smallest such) is re-carved for n; otherwise a new one is
// allocated, evicting least recently used ones beyond the HBM budget.
int get_workspace(bse_ctx* c, int n, int precision, Workspace** out) {
  const size_t need = workspace_bytes(n, precision);
  Workspace* best = nullptr;
  for (auto& w : c->ws)
    if (w.precision == precision && w.bytes >= need && (!best || w.bytes < best->bytes)) best = &w;
  if (best) {
    if (best->n != n) best->carve(n);
    best->last_use = ++c->use_clock;
    *out = best;
    return BSE_OK;
  }
  if (need > c->budget) {
    record_message("workspace exceeds the context's HBM budget");
    return BSE_ERR_NOMEM;
  }
  while (ctx_bytes_held(c) + need > c->budget && !c->ws.empty()) {
    auto victim = c->ws.begin();
    for (auto i = c->ws.begin(); i != c->ws.end(); ++i)
      if (i->last_use < victim->last_use) victim = i;
    cudaStreamSynchronize(c->stream);
    victim->release();
    c->ws.erase(victim);
  }
  Workspace w;
  int rc = w.init(n, precision);
  if (rc != BSE_OK) return rc;
  w.last_use = ++c->use_clock;
  c->ws.push_back(w);
  *out = &c->ws.back();
  return BSE_OK;
}

static int copy_in(const double* src, int ld, int n, double* dst, cudaStream_t s, const double** used, int* ldu) {
  if (is_device_ptr(src)) {
    *used = src;
    *ldu = ld;
    return BSE_OK;
  }
  if (ld == n)  // contiguous: one linear copy (runs at the full pinned-memory rate)
    BSE_CUDA(cudaMemcpyAsync(dst, src, (size_t)n * n * 16, cudaMemcpyHostToDevice, s));
  else
    BSE_CUDA(cudaMemcpy2DAsync(dst, (size_t)n * 16, src, (size_t)ld * 16, (size_t)n * 16, n, cudaMemcpyHostToDevice,
                               s));
  *used = dst;
  *ldu = n;
  return BSE_OK;
}

__global__ void negate_bottom_kernel(int n, double2* Y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= n) return;
  double2* p = Y + n + i + (long)j * 2 * n;
  double2 v = *p;
  *p = make_double2(-v.x, -v.y);
}

int negate_bottom(int n, double* Y, cudaStream_t s) {
  kcount(1);
  negate_bottom_kernel<<<dim3(ceil_div(n, 256), n), 256, 0, s>>>(n, reinterpret_cast<double2*>(Y));
  BSE_LAUNCH_CHECK();
  return BSE_OK;
}

// Phase convention of the returned eigenvectors (eigenvectors are unique up to a
// unit factor; this fixes one for display and reproducibility): in each column
// the largest-modulus entry of the top half of x_j (the first of equal ones) is
// made real and positive. x_j and y_j are multiplied by the same unit factor,
// which keeps y_j = diag(I, -I) x_j and Y^H X = I; the weights do not depend on it.
__global__ void __launch_bounds__(256) canon_phase_kernel(int n, double2* __restrict__ X, double2* __restrict__ Y) {
  __shared__ double sv[8];
  __shared__ int si[8];
  __shared__ double2 s_p;
  __shared__ double s_h;
  __shared__ int s_r;
  const long m = 2L * n;
  double2* x = X + (long)blockIdx.x * m;
  double best = -1.0;
  int bi = 0;
  for (int i = threadIdx.x; i < n; i += 256) {  // increasing i: the first of equals stays
    const double2 v = x[i];
    const double a = v.x * v.x + v.y * v.y;
    if (a > best) {
      best = a;
      bi = i;
    }
  }
  for (int o = 16; o >= 1; o >>= 1) {
    const double ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ob > best || (ob == best && oi < bi)) {
      best = ob;
      bi = oi;
    }
  }
  if ((threadIdx.x & 31) == 0) {
    sv[threadIdx.x >> 5] = best;
    si[threadIdx.x >> 5] = bi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = sv[0];
    int r = si[0];
    for (int w = 1; w < 8; ++w)
      if (sv[w] > b || (sv[w] == b && si[w] < r)) {
        b = sv[w];
        r = si[w];
      }
    const double2 v = x[r];
    const double h = hypot(v.x, v.y);
    s_p = h > 0.0 ? make_double2(v.x / h, -v.y / h) : make_double2(1.0, 0.0);  // conj(v) / |v|
    s_h = h;
    s_r = r;
  }
  __syncthreads();
  const double2 p = s_p;
  const double h = s_h;
  const int r = s_r;
  for (int i = threadIdx.x; i < m; i += 256) {
    const double2 v = x[i];
    x[i] = (i == r && h > 0.0) ? make_double2(h, 0.0) : make_double2(v.x * p.x - v.y * p.y, v.x * p.y + v.y * p.x);
    if (Y) {
      double2* y = Y + (long)blockIdx.x * m;
      const double2 u = y[i];
      y[i] = (i == r && h > 0.0) ? make_double2(h, 0.0) : make_double2(u.x * p.x - u.y * p.y, u.x * p.y + u.y * p.x);
    }
  }
}

static int canon_phase(int n, double* X, double* Y, cudaStream_t s) {
  kcount(1);
  canon_phase_kernel<<<n, 256, 0, s>>>(n, reinterpret_cast<double2*>(X), reinterpret_cast<double2*>(Y));
  BSE_LAUNCH_CHECK();
  return BSE_OK;
}

// Runs the whole pipeline on device-resident inputs into the workspace outputs
// (ws->lam, ws->X, ws->Y). Stage events go to ev[0..8] when timing.
// MRRR is selected and the workspace's scratch holds its tree (a workspace made
// before the selection may not)
static bool mrrr_fits(const Workspace* ws, int m, int n) {
  if (!use_mrrr()) return false;
  const size_t used = (size_t)((const char*)ws->scratch - (const char*)ws->base);
  return ws->bytes >= used && ws->bytes - used >= tdeig_mrrr_worksize(m, n);
}

int run_pipeline(bse_ctx* c, Workspace* ws, int n, const double* dA, int lda, const double* dB, int ldb,
                 int precision, bool want_Y, bse_info* info, cudaStream_t s, bool real_blocks) {
  const int m = 2 * n;
  cudaEvent_t* ev = c->ev;
  const bool tm = c->timing;
  StatusScope ss(ws->status);
  BSE_CUDA(cudaMemsetAsync(ws->status, 0, sizeof(DevStatus), s));
  if (tm) cudaEventRecord(ev[0], s);
  const bool f32 = precision != BSE_FP64;
  BSE_TRY(form_M(n, dA, lda, dB, ldb, ws->M, m, f32 ? ws->Lf : nullptr, ws->ldw, s));
  if (tm) cudaEventRecord(ev[1], s);
  if (!f32) {
    double* W = (double*)ws->W;
    double* tau = (double*)ws->tau;
    if (real_blocks) {
      // real A, B: M = diag(A + B, A - B), two Cholesky factorizations (Algorithm 2 step 1)
      BSE_TRY(potrf<double>(n, ws->M, m, ws->scratch, ws->status, s));
      BSE_TRY(potrf<double>(n, ws->M + n + (long)n * m, m, ws->scratch, ws->status, s, n));
    } else {
      BSE_TRY(potrf<double>(m, ws->M, m, ws->scratch, ws->status, s));
    }
    if (tm) cudaEventRecord(ev[2], s);
    BSE_TRY(form_W<double>(n, ws->M, m, W, ws->ldw, s));
    if (tm) cudaEventRecord(ev[3], s);
    BSE_TRY(tridiagonalize<double>(m, W, ws->ldw, ws->e, tau, ws->scratch, s, ws->status));
    if (tm) cudaEventRecord(ev[4], s);
    if (mrrr_fits(ws, m, n)) {
      // cluster-safe vectors from the representation tree: no reorthogonalization
      BSE_TRY(tdeig_mrrr(m, nullptr, ws->e, 1, n, m, 1e-3, ws->lam, ws->Vs, n, 1, ws->scratch, ws->status, s));
    } else {
      // X is free until the back-transform: the vector kernel's second pivot array
      BSE_TRY(tdeig(m, ws->e, ws->lam, ws->Vs, (double*)ws->scratch, ws->status, s, ws->X));
      // the FP64 path has no refinement: its eigenvectors are reorthogonalized (remark 2)
      BSE_TRY(tdeig_reorth(m, ws->Vs, ws->scratch, s));
    }
    if (tm) cudaEventRecord(ev[5], s);
    BSE_TRY(backtransform<double>(m, ws->M, m, W, ws->ldw, tau, ws->Vs, ws->lam, ws->X, want_Y ? ws->Y : nullptr, m,
                                  ws->scratch, s));
    if (tm) cudaEventRecord(ev[6], s);
  } else {
    float* W = (float*)ws->W;
    float* tau = (float*)ws->tau;
    if (real_blocks) {
      BSE_TRY(potrf<float>(n, ws->Lf, ws->ldw, ws->scratch, ws->status, s));
      BSE_TRY(potrf<float>(n, ws->Lf + n + (long)n * ws->ldw, ws->ldw, ws->scratch, ws->status, s, n));
    } else {
      BSE_TRY(potrf<float>(m, ws->Lf, ws->ldw, ws->scratch, ws->status, s));
    }
    if (tm) cudaEventRecord(ev[2], s);
    BSE_TRY(form_W<float>(n, ws->Lf, ws->ldw, W, ws->ldw, s));
    if (tm) cudaEventRecord(ev[3], s);
    const bool band = ws->sbr != nullptr && use_band_reduction(m, precision);
    if (band)
      BSE_TRY(sbr_reduce(m, W, ws->ldw, ws->e, tau, ws->sbr, ws->status, s));
    else
      BSE_TRY(tridiagonalize<float>(m, W, ws->ldw, ws->e, tau, ws->scratch, s, ws->status));
    if (tm) cudaEventRecord(ev[4], s);
    if (mrrr_fits(ws, m, n))
      BSE_TRY(tdeig_mrrr(m, nullptr, ws->e, 1, n, m, 1e-3, ws->lam, ws->Vs, n, 1, ws->scratch, ws->status, s));
    else  // X is free until the back-transform: the vector kernel's second pivot array
      BSE_TRY(tdeig(m, ws->e, ws->lam, ws->Vs, (double*)ws->scratch, ws->status, s, ws->X));
    if (tm) cudaEventRecord(ev[5], s);
    const bool refine_now = precision == BSE_MIXED_REFINED;
    BSE_TRY(backtransform<float>(m, ws->Lf, ws->ldw, W, ws->ldw, tau, ws->Vs, ws->lam, ws->X,
                                 (want_Y && !refine_now) ? ws->Y : nullptr, m, ws->scratch, s,
                                 band ? kSbrBand : 1, band ? ws->sbr : nullptr));
    if (tm) cudaEventRecord(ev[6], s);
    if (refine_now) {
      int sweeps = 0;
      double resid = 0, dl = 0, dl0 = 0;
      BSE_TRY(refine(n, ws->M, ws->lam, ws->X, 3, 0.0, ws->scratch, ws->status, s, &sweeps, &resid, &dl, &dl0));
      if (info) {
        info->sweeps = sweeps;
        info->refine_resid = resid;
        info->refine_dlam = dl;
        info->unrefined_dlam = dl0;
      }
      if (want_Y) {
        // Y = diag(I, -I) X
        BSE_CUDA(cudaMemcpyAsync(ws->Y, ws->X, (size_t)16 * m * n, cudaMemcpyDeviceToDevice, s));
        BSE_TRY(negate_bottom(n, ws->Y, s));
      }
    }
  }
  // the real path makes its columns real by a phase of its own (real_vectors)
  if (!real_blocks) BSE_TRY(canon_phase(n, ws->X, want_Y ? ws->Y : nullptr, s));
  if (tm) cudaEventRecord(ev[7], s);
  return BSE_OK;
}

static int copy_out(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  if (!dst) return BSE_OK;
  BSE_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s));
  return BSE_OK;
}

}  // namespace bse

extern "C" int bse_solve(bse_ctx* c, int n, const double* A, int lda, const double* B, int ldb, int precision,
                         double* lambda, double* X, double* Y, bse_sol** keep, bse_info* info) {
  if (info) memset(info, 0, sizeof(*info));
  // n <= 32767 keeps every per-column grid dimension (2n) within gridDim.y
  if (!c || n < 1 || n > 32767 || !A || !B || lda < n || ldb < n) return BSE_ERR_ARG;
  if (precision != BSE_FP64 && precision != BSE_MIXED && precision != BSE_MIXED_REFINED) return BSE_ERR_ARG;
  if (keep) *keep = nullptr;
  BSE_CUDA(cudaSetDevice(c->device));
  cudaStream_t s = c->stream;
  Workspace* ws = nullptr;
  BSE_TRY(get_workspace(c, n, precision, &ws));
  const int m = 2 * n;
  if (c->timing) cudaEventRecord(c->ev[8], s);
  const double *dA, *dB;
  int la, lb;
  BSE_TRY(copy_in(A, lda, n, ws->A, s, &dA, &la));
  BSE_TRY(copy_in(B, ldb, n, ws->B, s, &dB, &lb));
  if (c->timing) cudaEventRecord(c->ev[9], s);
  int rc = run_pipeline(c, ws, n, dA, la, dB, lb, precision, Y != nullptr, info, s);
  if (rc != BSE_OK) {
    if (info) info->status = rc;
    return rc;
  }
  DevStatus hst;
  BSE_CUDA(cudaMemcpyAsync(&hst, ws->status, sizeof(hst), cudaMemcpyDeviceToHost, s));
  BSE_TRY(copy_out(lambda, ws->lam, 8 * (size_t)n, s));
  BSE_TRY(copy_out(X, ws->X, 16 * (size_t)m * n, s));
  BSE_TRY(copy_out(Y, ws->Y, 16 * (size_t)m * n, s));
  if (c->timing) cudaEventRecord(c->ev[10], s);
  BSE_CUDA(cudaStreamSynchronize(s));
  if (info) {
    info->precision = precision;
    info->status = hst.code;
    info->info = hst.info;
    if (c->timing) {
      float ms = 0;
      const int map[8] = {0, 1, 2, 3, 4, 5, 6, 7};
      for (int k = 0; k < 7; ++k) {
        cudaEventElapsedTime(&ms, c->ev[map[k]], c->ev[map[k + 1]]);
        info->stage_ms[k] = ms;
      }
      // stage 5 (back-transform) ends at ev[6]; stage 6 (refinement) ends at ev[7]
      cudaEventElapsedTime(&ms, c->ev[8], c->ev[9]);
      float ms2 = 0;
      cudaEventElapsedTime(&ms2, c->ev[7], c->ev[10]);
      info->stage_ms[8] = ms + ms2;
      cudaEventElapsedTime(&ms, c->ev[8], c->ev[10]);
      info->stage_ms[9] = ms;
    }
  }
  if (hst.code != 0) {
    record_message(hst.code == BSE_ERR_NOT_DEFINITE ? "Eq. cond fails: Cholesky of M met a non-positive pivot"
                                                    : "device-side failure");
    return hst.code;
  }
  if (keep) {
    bse_sol* sol = new bse_sol();
    sol->n = n;
    sol->device = c->device;
    // stream-ordered allocations from the device pool (which keeps freed memory
    // cached, see bse_create): no device-wide synchronisation per kept solution
    if (cudaMallocAsync((void**)&sol->lam, 8 * (size_t)n, s) != cudaSuccess ||
        cudaMallocAsync((void**)&sol->X, 16 * (size_t)m * n, s) != cudaSuccess) {
      cudaGetLastError();
      bse_sol_free(sol);
      record_message("bse_solve: cannot allocate the kept solution");
      return BSE_ERR_NOMEM;
    }
    BSE_CUDA(cudaMemcpyAsync(sol->lam, ws->lam, 8 * (size_t)n, cudaMemcpyDeviceToDevice, s));
    BSE_CUDA(cudaMemcpyAsync(sol->X, ws->X, 16 * (size_t)m * n, cudaMemcpyDeviceToDevice, s));
    BSE_CUDA(cudaStreamSynchronize(s));
    *keep = sol;
  }
  return BSE_OK;
}

// Algorithm 2 (Section 3.2): real A = A^T, B = B^T with A + B > 0, A - B > 0.
// Outputs lambda (n, ascending) and the real X1, X2 (n x n each, ld n) with
// H [X1; X2] = [X1; X2] Lambda and X1^T X1 - X2^T X2 = I (Theorem 5).
extern "C" int bse_solve_real(bse_ctx* c, int n, const double* A, int lda, const double* B, int ldb, int precision,
                              double* lambda, double* X1, double* X2, bse_info* info) {
  if (info) memset(info, 0, sizeof(*info));
  if (!c || n < 1 || n > 32767 || !A || !B || lda < n || ldb < n) return BSE_ERR_ARG;
  if (precision != BSE_FP64 && precision != BSE_MIXED && precision != BSE_MIXED_REFINED) return BSE_ERR_ARG;
  BSE_CUDA(cudaSetDevice(c->device));
  cudaStream_t s = c->stream;
  Workspace* ws = nullptr;
  BSE_TRY(get_workspace(c, n, precision, &ws));
  const int m = 2 * n;
  // the real inputs go through the X buffer (2n x n complex = 4 n^2 doubles,
  // unused until the back-transform) and become complex A, B in the workspace
  double* rA = ws->X;
  double* rB = ws->X + (size_t)n * n;
  const double* srcA = A;
  const double* srcB = B;
  long la = lda, lb = ldb;
  auto stage = [&](double* dst, const double* src, int ld) -> cudaError_t {
    if (ld == n) return cudaMemcpyAsync(dst, src, (size_t)n * n * 8, cudaMemcpyHostToDevice, s);
    return cudaMemcpy2DAsync(dst, (size_t)n * 8, src, (size_t)ld * 8, (size_t)n * 8, n, cudaMemcpyHostToDevice, s);
  };
  if (!is_device_ptr(A)) {
    BSE_CUDA(stage(rA, A, lda));
    srcA = rA;
    la = n;
  }
  if (!is_device_ptr(B)) {
    BSE_CUDA(stage(rB, B, ldb));
    srcB = rB;
    lb = n;
  }
  BSE_TRY(real_to_complex(n, srcA, la, ws->A, s));
  BSE_TRY(real_to_complex(n, srcB, lb, ws->B, s));
  int rc = run_pipeline(c, ws, n, ws->A, n, ws->B, n, precision, false, info, s, true);
  if (rc != BSE_OK) {
    if (info) info->status = rc;
    return rc;
  }
  // X1, X2 into the Y buffer (2 n^2 doubles of its 4 n^2), then out
  double* rX1 = ws->Y;
  double* rX2 = ws->Y + (size_t)n * n;
  BSE_TRY(real_vectors(n, ws->X, m, (X1 && is_device_ptr(X1)) ? X1 : rX1, (X2 && is_device_ptr(X2)) ? X2 : rX2, n,
                       s));
  DevStatus hst;
  BSE_CUDA(cudaMemcpyAsync(&hst, ws->status, sizeof(hst), cudaMemcpyDeviceToHost, s));
  BSE_TRY(copy_out(lambda, ws->lam, 8 * (size_t)n, s));
  if (X1 && !is_device_ptr(X1)) BSE_TRY(copy_out(X1, rX1, 8 * (size_t)n * n, s));
  if (X2 && !is_device_ptr(X2)) BSE_TRY(copy_out(X2, rX2, 8 * (size_t)n * n, s));
  BSE_CUDA(cudaStreamSynchronize(s));
  if (info) {
    info->precision = precision;
    info->status = hst.code;
    info->info = hst.info;
  }
  if (hst.code != 0) {
    record_message(hst.code == BSE_ERR_NOT_DEFINITE ? "A + B or A - B is not positive definite (Cholesky pivot)"
                                                    : "device-side failure");
    return hst.code;
  }
  return BSE_OK;
}

extern "C" int bse_sol_view(const bse_sol* sol, int* n, const double** lambda_dev, const double** X_dev) {
  if (!sol) return BSE_ERR_ARG;
  if (n) *n = sol->n;
  if (lambda_dev) *lambda_dev = sol->lam;
  if (X_dev) *X_dev = sol->X;
  return BSE_OK;
}

extern "C" int bse_sol_free(bse_sol* sol) {
  if (!sol) return BSE_OK;
  // every call that used the solution has synchronised its stream before
  // returning, so the blocks can go back to the pool in the default stream's order
  // (valid even after the context that made the solution is destroyed)
  if (sol->lam) cudaFreeAsync(sol->lam, 0);
  if (sol->X) cudaFreeAsync(sol->X, 0);
  delete sol;
  return BSE_OK;
}

extern "C" int bse_spectrum(bse_ctx* c, const bse_sol* sol, const double* d_r, const double* d_l, double* w) {
  if (!c || !sol || !d_r || !d_l || !w) return BSE_ERR_ARG;
  BSE_CUDA(cudaSetDevice(c->device));
  cudaStream_t s = c->stream;
  const int n = sol->n, m = 2 * n;
  double* buf = nullptr;
  const bool dr_dev = is_device_ptr(d_r), dl_dev = is_device_ptr(d_l), w_dev = is_device_ptr(w);
  if (!dr_dev || !dl_dev || !w_dev) BSE_CUDA(cudaMallocAsync((void**)&buf, 16 * (size_t)(2 * m + n), s));
  const double* dr = d_r;
  const double* dl = d_l;
  double* dw = w;
  if (!dr_dev) {
    BSE_CUDA(cudaMemcpyAsync(buf, d_r, 16 * (size_t)m, cudaMemcpyHostToDevice, s));
    dr = buf;
  }
  if (!dl_dev) {
    BSE_CUDA(cudaMemcpyAsync(buf + 2 * m, d_l, 16 * (size_t)m, cudaMemcpyHostToDevice, s));
    dl = buf + 2 * m;
  }
  if (!w_dev) dw = buf + 4 * m;
  int rc = weights(n, sol->X, m, dr, dl, dw, s);
  if (rc == BSE_OK && !w_dev) BSE_CUDA(cudaMemcpyAsync(w, dw, 16 * (size_t)n, cudaMemcpyDeviceToHost, s));
  if (buf) cudaFreeAsync(buf, s);
  BSE_CUDA(cudaStreamSynchronize(s));
  return rc;
}
