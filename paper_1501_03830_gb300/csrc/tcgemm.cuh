// Tensor-core (tcgen05) GEMM interface: see k_tcgemm.cu.
#pragma once

#include "common.cuh"

namespace bse {
namespace tc {

constexpr int kMaxUnits = 72;

// Kernel parameters (passed by value).
struct TcParams {
  int M, N, K;           // output M x N, reduction length K
  int a_rows, b_rows;    // rows per digit matrix in the stacked A / B tensors
  int units;             // digit pairs accumulated by every output tile
  int a_digit[kMaxUnits], b_digit[kMaxUnits];
  double unit_scale[kMaxUnits];
  int mode;              // 0: Cf = acc (FP32); 1: Cd += acc * rs[row] * cs[col] * unit_scale
  float* Cf;
  double* Cd;
  long ldc;
  const double* rs;
  const double* cs;
  int* status;           // first int of the caller's status word (nullable)
};

// Host-side description of one launch. A holds a_digits stacked matrices of
// a_rows x K (K contiguous, row pitch ldk), B likewise; both bf16.
struct TcProblem {
  int M, N, K, ldk;
  const void* A;
  const void* B;
  int a_rows, b_rows, a_digits, b_digits;
  int units;
  int a_digit[kMaxUnits], b_digit[kMaxUnits];
  double unit_scale[kMaxUnits];
  int mode;
  float* Cf;
  double* Cd;
  long ldc;
  const double* rs;
  const double* cs;
  int* status;
};

int tc_gemm(const TcProblem& pb, cudaStream_t s);

}  // namespace tc
}  // namespace bse
