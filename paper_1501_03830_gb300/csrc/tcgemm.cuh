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
  int chunk_kb;          // K blocks (of 64) per exact accumulation chunk in TMEM
  int a_digit[kMaxUnits], b_digit[kMaxUnits];
  unsigned char fold[kMaxUnits];  // unit u ends a group summed together: write it out
  int mode;              // 0: Cf = sum (FP32); 1: plane g of Si = integer sum of group g
  float* Cf;
  int* Si;               // mode 1: int32 planes, M x N column-major (ldc), plane apart
  long plane;
  long ldc;
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
  int chunk_kb;
  int a_digit[kMaxUnits], b_digit[kMaxUnits];
  unsigned char fold[kMaxUnits];
  int mode;
  float* Cf;
  int* Si;
  long plane;
  long ldc;
  int* status;
};

int tc_gemm(const TcProblem& pb, cudaStream_t s);

}  // namespace tc
}  // namespace bse
