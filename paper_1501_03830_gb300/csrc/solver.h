// Host-side state behind the opaque bse_ctx / bse_sol handles.
#pragma once

#include <list>
#include <map>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace bse {

struct Workspace {
  int n = 0, precision = 0;
  size_t bytes = 0;
  unsigned long last_use = 0;
  void* base = nullptr;
  double *A = nullptr, *B = nullptr;  // staging for host inputs (complex128)
  double* M = nullptr;                // FP64 M (L and then Phi on the FP64 path)
  float* Lf = nullptr;                // FP32 copy of M -> L -> Phi (mixed paths)
  void* W = nullptr;                  // W, then the reflectors (FP64 or FP32)
  int ldw = 0;                        // W's leading dimension (2n padded to 32)
  double* e = nullptr;                // sub-diagonal of T
  void* tau = nullptr;
  double* lam = nullptr;
  double* Vs = nullptr;               // sign-folded V+ (row-major m x n)
  double *X = nullptr, *Y = nullptr;  // complex128 2n x n
  DevStatus* status = nullptr;
  void* sbr = nullptr;                // band reduction state kept from the reduction to the back-transform
  void* scratch = nullptr;            // stage scratch (max over stages)
  int init(int n, int precision);  // allocate workspace_bytes(n, precision) and carve it for n
  void carve(int n);               // lay the buffers out for n (workspace_bytes(n) <= bytes)
  void release();
};

size_t workspace_bytes(int n, int precision);
// the mixed paths reduce W in two stages (band, then tridiagonal) from this order m = 2n on
bool use_band_reduction(int m, int precision);
// the tridiagonal eigenvectors come from the MRRR representation tree (else twisted
// factorizations on the root matrix, reorthogonalized on the FP64 path)
bool use_mrrr();
bool is_device_ptr(const void* p);

struct ServeState;

}  // namespace bse

struct bse_ctx {
  int device = 0;
  size_t budget = 0;
  cudaStream_t own_stream = nullptr;
  cudaStream_t stream = nullptr;
  bool timing = false;
  cudaEvent_t ev[12];
  std::list<bse::Workspace> ws;  // a workspace serves every n whose layout fits its bytes
  std::vector<bse_ctx*> batch_slots;  // per-stream contexts of bse_solve_batched
  unsigned long use_clock = 0;
  bse::ServeState* serve = nullptr;
};

struct bse_sol {
  int n = 0;
  int device = 0;
  double* lam = nullptr;
  double* X = nullptr;
};

namespace bse {
int get_workspace(bse_ctx* c, int n, int precision, Workspace** out);
int run_pipeline(bse_ctx* c, Workspace* ws, int n, const double* dA, int lda, const double* dB, int ldb,
                 int precision, bool want_Y, bse_info* info, cudaStream_t s, bool real_blocks = false);
}  // namespace bse
