// Internal (C++) entry points of the pipeline stages, shared by the solver,
// the batched solver and the request loop.
#pragma once

#include "common.cuh"

namespace bse {

int form_M(int n, const double* A, int lda, const double* B, int ldb, double* M, int ldm, float* Mf, int ldmf,
           cudaStream_t s);

template <typename T>
size_t potrf_worksize(int m);
template <typename T>
int potrf(int m, T* A, long lda, void* work, DevStatus* st, cudaStream_t s, int col_offset = 0);

template <typename T>
int form_W(int n, const T* L, long ldl, T* W, long ldw, cudaStream_t s);

template <typename T>
size_t trd_worksize(int m);
template <typename T>
int tridiagonalize(int m, T* W, long ldw, double* e, T* tau, void* work, cudaStream_t st, DevStatus* status);

// vec_scratch (nullable): m x n doubles for the two-thread vector kernel
int tdeig(int m, const double* e, double* lam, double* Vs, double* work, DevStatus* st, cudaStream_t s,
          double* vec_scratch = nullptr);
// the same eigenpairs (or any index range of a general symmetric tridiagonal) by the
// MRRR representation tree (k_mrrr.cu); Z row-major m x ldz
size_t tdeig_mrrr_worksize(int m, int nz);
int tdeig_mrrr(int m, const double* a, const double* b, int bse_form, int il, int iu, double gaptol, double* lam,
               double* Z, long ldz, int bse_signs, void* work, DevStatus* st, cudaStream_t s);
// remark 2: reorthogonalization of the tridiagonal eigenvectors Vs (row-major m x n)
size_t tdeig_reorth_worksize(int m);
int tdeig_reorth(int m, double* Vs, void* work, cudaStream_t s);

template <typename T>
size_t bt_worksize(int m);
// Phi = L U from the reflectors in W (reflector j starts at row j + off), then
// (with sbr_work, the band reduction's workspace) Phi <- Phi Q2, then X, Y.
template <typename T>
int backtransform(int m, T* L, long ldl, const T* W, long ldw, const T* tau, const double* Vs, const double* lam,
                  double* X, double* Y, long ldx, void* work, cudaStream_t s, int off = 1, void* sbr_work = nullptr);

// two-stage (band) reduction of the FP32 skew W (k_sbr.cu): e = T's sub-diagonal,
// stage-1 reflectors in W below the band (explicit unit entries at rows j + b)
// with scalars in tau; stage-2 reflectors kept in the workspace for sbr_apply_q2
constexpr int kSbrBand = 64;  // half-bandwidth of the first stage (the off of its reflectors)
size_t sbr_worksize(int m);
int sbr_reduce(int m, float* W, long ldw, double* e, float* tau, void* work, DevStatus* st, cudaStream_t s);
int sbr_apply_q2(int m, float* Phi, long ldp, void* work, cudaStream_t s);

int weights(int n, const double* X, long ldx, const double* dr, const double* dl, double* w, cudaStream_t s);

// real problems (k_real.cu)
int real_to_complex(int n, const double* R, long ldr, double* Z, cudaStream_t s);
int real_vectors(int n, const double* X, long ldx, double* X1, double* X2, long ldo, cudaStream_t s);

size_t ozaki_worksize(int M, int N, int K, int s);
// an operand of the digit-split product: K-vectors at ptr + v*ld (strided = false)
// or at ptr + v with stride ld between consecutive k (strided = true)
struct OzOperand {
  const void* ptr;
  long ld;
  bool strided;
  bool f32;
};
// s digits are split for A (and the workspace is laid out for s); s_use <= s of
// them (and of B's) are paired in this product (0 = all s).
int ozaki_gemm_ex(const OzOperand& A, const OzOperand& B, int M, int N, int K, double* C, long ldc, int s,
                  bool accumulate, void* work, bool split_A, int* status, cudaStream_t st, int s_use = 0);
int ozaki_gemm(int M, int N, int K, const double* A, long lda, const double* B, long ldb, double* C, long ldc, int s,
               void* work, bool split_A, int* status, cudaStream_t st, int s_use = 0);
// digits per operand for a K-long product carrying `bits` bits (50: FP64-accurate)
int ozaki_digits(int K, int bits = 50);

size_t refine_worksize(int n);
// FP64 structure-preserving refinement of (lam, X) in place (X: 2n x n complex128, ld 2n),
// against the FP64 M (2n x 2n). Returns BSE_OK and fills the diagnostics.
int refine(int n, const double* M, double* lam, double* X, int max_sweeps, double tol, void* work,
           DevStatus* st, cudaStream_t s, int* sweeps_done, double* resid, double* dlam_last, double* dlam_first);

}  // namespace bse
