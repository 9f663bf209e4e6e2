// Launch accounting and optional per-kernel event timing.
//
// Every kernel launch of the library bumps a global counter (bse_launch_count).
// When kernel profiling is on (bse_kprof_enable), the launches of each kernel
// class are bracketed by CUDA events on their own stream and tagged with the
// algorithmic bytes and flops they are charged with; bse_kprof_read returns per
// class: launches, total device time and the charged bytes / flops, from which
// a caller gets achieved GB/s or FLOP/s. Profiling adds event records, so it
// is meant for an extra instrumented run, not for the timed one.
#pragma once

#include <cuda_runtime.h>

namespace bse {

enum KClass {
  K_FORM_M = 0,
  K_POTRF_DIAG,
  K_GEMM_F64,
  K_GEMM_F32,
  K_TRD_SYMV,
  K_TRD_COL,
  K_TDEIG_BISECT,
  K_TDEIG_VEC,
  K_WEIGHTS,
  K_ELEMENTWISE,
  K_GEMM_TC,
  K_GEMM_TF32,
  K_SBR_QR,     // band reduction: panel QR
  K_SBR_CHASE,  // band reduction: bulge chasing
  K_SBR_Q2,     // band reduction: back-transform of the chase
  K_TF32_SPLIT, // hi / lo TF32 planes of the FP32 products' operands
  K_NUM_CLASSES
};

void kcount(int launches = 1);
bool kprof_on();
// begin/end around one launch of class k on stream s (no-ops unless enabled)
int kprof_begin(int k, cudaStream_t s);
void kprof_end(int slot, cudaStream_t s, double bytes, double flops);

struct KprofScope {
  int slot;
  cudaStream_t s;
  double bytes, flops;
  KprofScope(int k, cudaStream_t st, double b, double f) : slot(-1), s(st), bytes(b), flops(f) {
    kcount(1);
    if (kprof_on()) slot = kprof_begin(k, st);
  }
  ~KprofScope() {
    if (slot >= 0) kprof_end(slot, s, bytes, flops);
  }
};

}  // namespace bse
