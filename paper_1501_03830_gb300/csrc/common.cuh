// Shared device/host helpers for the structure-preserving BSE solver (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include "../../include/bse.h"
#include "kprof.cuh"

namespace bse {

// Device-side status word written by kernels that can detect a failure
// (non-positive Cholesky pivot, bisection that does not converge, a bounded
// wait that gave up). Kernels never trap: they record and return.
struct DevStatus {
  int code;   // 0 = ok, else a BSE_ERR_* value
  int info;   // e.g. 1-based pivot column for BSE_ERR_NOT_DEFINITE
  int spare[2];
};

__device__ __forceinline__ void set_status(DevStatus* st, int code, int info) {
  if (atomicCAS(&st->code, 0, code) == 0) st->info = info;
}

// The status word of the solve running on this host thread, for kernels whose
// launchers take none (the tensor-core GEMM behind gemm<float>): a bounded wait
// that gives up records there. Set for the duration of a call by StatusScope.
DevStatus*& current_status();
struct StatusScope {
  DevStatus* prev;
  explicit StatusScope(DevStatus* st) : prev(current_status()) { current_status() = st; }
  ~StatusScope() { current_status() = prev; }
};

template <typename T>
struct Eps;
template <>
struct Eps<double> {
  static constexpr double value = 2.220446049250313e-16;
};
template <>
struct Eps<float> {
  static constexpr float value = 1.1920929e-07f;
};

__host__ __device__ inline int ceil_div(long a, long b) { return (int)((a + b - 1) / b); }

// Host error plumbing: the first CUDA error of a call is kept as text for
// bse_last_error().
void record_error(const char* what, cudaError_t err, const char* file, int line);
void record_message(const char* msg);

#define BSE_CUDA(call)                                              \
  do {                                                              \
    cudaError_t _e = (call);                                        \
    if (_e != cudaSuccess) {                                        \
      ::bse::record_error(#call, _e, __FILE__, __LINE__);          \
      return BSE_ERR_CUDA;                                          \
    }                                                               \
  } while (0)

#define BSE_LAUNCH_CHECK()                                          \
  do {                                                              \
    cudaError_t _e = cudaGetLastError();                            \
    if (_e != cudaSuccess) {                                        \
      ::bse::record_error("kernel launch", _e, __FILE__, __LINE__); \
      return BSE_ERR_CUDA;                                          \
    }                                                               \
  } while (0)

#define BSE_TRY(expr)              \
  do {                             \
    int _rc = (expr);              \
    if (_rc != BSE_OK) return _rc; \
  } while (0)

}  // namespace bse
