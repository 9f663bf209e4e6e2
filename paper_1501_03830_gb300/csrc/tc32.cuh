// FP32 GEMM on the tcgen05 tensor cores with 3xTF32 splitting: see k_tc32.cu.
#pragma once

#include "gemm_simt.cuh"

namespace bse {
namespace tc32 {

// Layouts the kernel takes: no batch, no triangular operand masks, 16-byte
// aligned A and B with leading dimensions divisible by 4 (TMA pitch rule).
bool eligible(const GemmArgs& g);
// C = alpha op(A) op(B) + beta C (lower triangle only if g.c_uplo); split = 1
// for 3xTF32, 0 for one TF32 pass. `status` (nullable) gets BSE_ERR_TIMEOUT if
// a bounded wait gives up. BSE_ERR_ARG if !eligible(g).
int gemm(const GemmArgs& g, int split, int* status, cudaStream_t s);
// 1: FP32 GEMMs of the mixed path go to the tensor cores when eligible; 0: SIMT.
int mode();

}  // namespace tc32
}  // namespace bse
