/*
 * bse_stages.h -- stage-level C ABI of the BSE solver: one entry point per
 * step of Algorithm 1 / Algorithm 3, on DEVICE pointers, asynchronous on the
 * given stream (a cudaStream_t passed as void*; NULL = legacy default stream).
 * These are what bse_solve chains; they are exported for testing each stage
 * against the oracle and for timing each kernel on its own.
 *
 * Shared rules
 *   - All matrices are column-major with the given leading dimension, except
 *     the eigenvector matrix Vs of bse_stage_tdeig (row-major, see there).
 *   - `fp32 = 1` selects FP32 storage and arithmetic for a stage that has both
 *     (the mixed path); otherwise FP64.
 *   - `work` is caller-owned device scratch of at least the *_worksize bytes,
 *     256-byte aligned; its contents on entry do not matter.
 *   - `dev_status` points to 16 zero-initialised device bytes (4 ints); a stage
 *     that detects a failure stores {code, info} there (first failure wins) and
 *     never traps. The host reads it after the stream is synchronised.
 *   - Return value: BSE_OK, BSE_ERR_ARG on a bad argument (checked on the host
 *     before any launch), BSE_ERR_CUDA on a launch error.
 */
#ifndef BSE_GB300_STAGES_H
#define BSE_GB300_STAGES_H

#include <stddef.h>

#include "bse.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Algorithm 1 step 1 (Theorem 2, Eq. embedding):
 *   M = [Re(A+B) Im(A-B); -Im(A+B) Re(A-B)]   (2n x 2n real symmetric, FULL storage)
 * A, B: n x n complex128 (interleaved), ld in complex elements, lower triangles read.
 * M: FP64, ldm >= 2n. Mf (nullable): an FP32 copy, ldmf >= 2n. */
int bse_stage_form_M(int n, const double* A, int lda, const double* B, int ldb, double* M, int ldm, float* Mf,
                     int ldmf, void* stream);

/* Algorithm 1 step 2: M = L L^T in place (lower triangle; the strict upper
 * triangle is not touched). A non-positive pivot (Eq. cond violated) stores
 * {BSE_ERR_NOT_DEFINITE, 1-based column} in dev_status. A: m x m, FP64 or FP32. */
size_t bse_stage_potrf_worksize(int m, int fp32);
int bse_stage_potrf(int m, void* A, int lda, int fp32, void* work, int* dev_status, void* stream);

/* Algorithm 1 step 3: W = L^T J L with J = [0 I; -I 0] (Eq. J). L: 2n x 2n lower
 * (the upper triangle is ignored). Writes the STRICT LOWER triangle of W and its
 * diagonal (zero); W's upper-right n x n block is used as scratch. */
int bse_stage_form_W(int n, const void* L, int ldl, void* W, int ldw, int fp32, void* stream);

/* Algorithm 3 step 1 (remark 1): W = U T U^T by blocked skew-symmetric Householder
 * reduction, m = 2n. Reads W's strict lower triangle; on return e[k] = T[k+1,k]
 * (k = 0..m-2, FP64), tau[k] (FP64 or FP32 like W) and W[k+1:m, k] = v_k with
 * v_k[0] = 1 (H_k = I - tau_k v_k v_k^T, U = H_0 H_1 ... H_{m-2}).
 * Each 64-column panel is one cooperative launch whose grid barriers wait at most
 * ~2 s; a barrier that gives up stores BSE_ERR_TIMEOUT in dev_status (the kernel
 * returns, it never hangs). A failure already in dev_status skips the work. */
size_t bse_stage_tridiag_worksize(int m, int fp32);
int bse_stage_tridiag(int m, void* W, int ldw, double* e, void* tau, int fp32, void* work, int* dev_status,
                      void* stream);

/* Two-stage (successive band) form of Algorithm 3 step 1 for FP32 W (Section 3.3,
 * closing remark: band reduction in place of the memory-bound skew SYMV). m >= 3;
 * W: m x m FP32, strict lower triangle read, leading dimension ldw divisible by 32
 * and a 16-byte aligned base (else BSE_ERR_ARG); W's upper triangle is used.
 * Stage 1 (dense -> half-bandwidth 64, panel QR plus tensor-core two-sided
 * updates) leaves, for every column k, the reflector v_k with its unit entry
 * written at row k+64 in W[k+64:m, k] and its scalar in tau[k] (FP32, m entries;
 * zero where there is none); stage 2 (bulge chasing) leaves its reflectors in
 * `work` (size bse_stage_sbr_worksize(m), owned by the caller) for
 * bse_stage_sbr_apply_q2 / bse_stage_sbr_backtransform. On return e[k] = T[k+1, k]
 * (FP64, k = 0..m-2, e[m-1] = 0) with W = Q T Q^T, Q = Q1 Q2, Q e_1 = e_1, so |e|
 * equals |e| of bse_stage_tridiag in exact arithmetic (implicit-Q theorem). Both
 * stages' bounded waits store BSE_ERR_TIMEOUT in dev_status instead of hanging. */
size_t bse_stage_sbr_worksize(int m);
int bse_stage_sbr(int m, float* W, int ldw, double* e, float* tau, void* work, int* dev_status, void* stream);

/* Phi <- Phi Q2 (m x m FP32, column-major, leading dimension ldp >= m) with the
 * stage-2 reflectors that the last bse_stage_sbr left in `work`. */
int bse_stage_sbr_apply_q2(int m, float* Phi, int ldp, void* work, void* stream);

/* Algorithm 3 steps 3-6 after bse_stage_sbr: Phi = L Q1 Q2 in place of L (FP32,
 * lower triangle of L read), then X, Y as bse_stage_backtransform (fp32 = 1) makes
 * them. bt_work: bse_stage_backtransform_worksize(m, 1) bytes; sbr_work: the
 * workspace of the bse_stage_sbr call that reduced this W. */
int bse_stage_sbr_backtransform(int m, float* L, int ldl, const float* W, int ldw, const float* tau,
                                const double* Vs, const double* lam, double* X, double* Y, int ldx, void* bt_work,
                                void* sbr_work, void* stream);

/* Order m = 2n from which the mixed paths of bse_solve (and of the batched and
 * serving calls) use the two-stage reduction instead of the one-stage one
 * (default 0 = never: measured slower than the one-stage panel on GB300 at
 * n = 8192, see the design notes). Process-wide; set it before solving. */
int bse_set_band_reduction(int min_m);

/* Diagnostics of the tridiagonal reduction (no counterpart in the paper):
 * bse_debug_trace_tridiag makes every later bse_stage_tridiag / bse_solve record,
 * for columns j < `columns`, the device clock (ns) of each block at eight points
 * of the column's work (0 column start, 1 after the first grid barrier, 2 SYMV
 * start, 3 the block's SYMV share done, 4 after the second barrier,
 * 5 panel vectors staged, 6 p at the column's leading row known, 7 the block's
 * rows updated) into the device buffer (layout [column][8][G] with
 * G = bse_stage_tridiag_grid(m, fp32), unsigned 64-bit; panels launched with
 * fewer blocks leave the rest of a row untouched); NULL turns it off. The buffer
 * must hold columns * 8 * G entries. */
int bse_debug_trace_tridiag(void* dev_buffer, int columns);

/* Test hook for failure detection without a GPU fault: the number of polls after
 * which a grid-barrier wait of the tridiagonal panel kernel gives up (polls > 0),
 * or 0 to restore the default (2^25 polls, about 2 s). With a tiny value the
 * blocks of the next panel launch stop waiting for one another: each records
 * BSE_ERR_TIMEOUT in the device status word and returns, the stage returns
 * normally, and the status reaches the host through dev_status / bse_info. The
 * barrier words are reset at the start of every reduction, so the next solve on
 * the same context runs normally once the default is restored. Process-wide;
 * not for concurrent use. */
int bse_debug_barrier_spin(long polls);
/* Blocks in the cooperative grid of the panel kernel (the largest launched). */
int bse_stage_tridiag_grid(int m, int fp32);

/* Algorithm 3 step 2 (remark 2): positive eigenpairs of Tsym = -i D^H T D (zero
 * diagonal, off-diagonal -e[k]), D = diag(i^k), k = 0..m-1, m even. FP64.
 *   lam: n = m/2 eigenvalues, ascending.
 *   Vs (nullable): ROW-major m x n (element (k, j) at k*n + j): the eigenvectors
 *   with the D phase folded in, Vs[k][j] = s_k v_j[k], s_k = +1,+1,-1,-1 for
 *   k mod 4 = 0,1,2,3 (so D v_j = even rows + i * odd rows of Vs). */
size_t bse_stage_tdeig_worksize(int m);
int bse_stage_tdeig(int m, const double* e, double* lam, double* Vs, void* work, int* dev_status, void* stream);

/* Remark 2 of Algorithm 3 (reorthogonalization of the computed eigenvectors when
 * high accuracy is wanted): the eigenvectors Vs that bse_stage_tdeig returned (row-major m x n,
 * ascending eigenvalues) are made orthonormal again among index neighbours: a
 * symmetric correction v_j <- v_j - 1/2 sum_i v_i (v_i^T v_j) over
 * 0 < |i - j| <= 48, then unit norms, twice. Twisted-factorization vectors of
 * close eigenvalues are orthogonal only to eps ||T|| / gap; this takes the
 * nearby pairs to rounding level. work: bse_stage_tdeig_reorth_worksize(m)
 * bytes. The FP64 path of bse_solve runs it; the refined path does not need it. */
size_t bse_stage_tdeig_reorth_worksize(int m);
int bse_stage_tdeig_reorth(int m, double* Vs, void* work, void* stream);

/* Algorithm 3 step 2 by a representation tree (MRRR; Section 3.3's closing
 * remarks name it for the tridiagonal step, and it makes remark 2's
 * reorthogonalization unnecessary): eigenpairs il .. iu-1 (0-based, ascending) of
 * the m x m symmetric tridiagonal T with diagonal a (NULL: zero) and off-diagonal
 * b (m - 1 entries; with bse_form != 0, b is the sub-diagonal e of the skew T that
 * bse_stage_tridiag returns and T = Tsym = -i D^H T D, off-diagonal -e, zero
 * diagonal). FP64, device pointers.
 *   Root T - sigma I = L D L^T (sigma below the Gershgorin interval); eigenvalues by
 *   multisection on the representation; runs whose relative gaps are below gaptol
 *   (0: 1e-3) get child representations L D L^T - tau I (stationary qd transform)
 *   down a tree of at most 8 levels (64 more for clusters of more than 1/gaptol
 *   members, which are split ~1/gaptol eigenvalues at a time); vectors by twisted
 *   factorizations of their representation, three Rayleigh-quotient corrections of
 *   the eigenvalue, normalised.
 *   lam: iu - il values. Z: row-major m x ldz (ldz >= iu - il), column j = the
 *   eigenvector of value il + j; with bse_signs != 0 the D phase is folded in as in
 *   bse_stage_tdeig (rows scaled by +1,+1,-1,-1 for k mod 4), so bse_form = 1,
 *   il = m/2, iu = m, ldz = m/2, bse_signs = 1 gives bse_stage_tdeig's lam and Vs.
 *   work: bse_stage_tdeig_mrrr_worksize(m, il, iu) bytes (16 m (iu - il) + small:
 *   two levels of child representations). The call synchronises its stream once per
 *   tree level (it reads the count of new child representations). A bisection that
 *   does not converge records BSE_ERR_NOT_CONVERGED in dev_status. */
size_t bse_stage_tdeig_mrrr_worksize(int m, int il, int iu);
/* Tridiagonal eigenvectors of bse_solve (and the batched and serving calls): 0 =
 * twisted factorizations on the root matrix, reorthogonalized on the FP64 path
 * (remark 2; the default), 1 = the representation tree of bse_stage_tdeig_mrrr
 * (no reorthogonalization). Process-wide; set it before solving. */
int bse_set_tdeig_method(int method);
int bse_stage_tdeig_mrrr(int m, const double* a, const double* b, int bse_form, int il, int iu, double gaptol,
                         double* lam, double* Z, int ldz, int bse_signs, void* work, int* dev_status, void* stream);

/* Allocation-free variant of bse_stage_tdeig (the paper has no counterpart: this
 * is a packaging choice of this library). Same arguments and results, minus
 * `work`: the scratch is a fixed 512 KiB array compiled into the library, so the
 * call needs no device memory from the caller and allocates none itself (no
 * cudaMalloc, no allocating library routine). It is for callers that cannot
 * allocate device memory at the point of the call -- e.g. code that runs with a
 * fixed, pre-reserved memory budget, or that is not allowed to synchronise the
 * device the way cudaMalloc/cudaFree can.
 *   - Limit: m <= 65536 (n <= 32768); larger m returns BSE_ERR_ARG with a message
 *     in bse_last_error().
 *   - The first call on a device looks up the array's device address (one
 *     cudaGetSymbolAddress per device, with that device current); make that first
 *     call before any stream capture.
 *   - Every call on a device shares the one array and leaves its contents behind;
 *     nothing in it needs clearing between calls, but calls that overlap on the GPU
 *     (different streams, or host threads) race on it: serialise them. */
int bse_stage_tdeig_noalloc(int m, const double* e, double* lam, double* Vs, int* dev_status, void* stream);

/* Algorithm 3 steps 3-6 with the Lambda^{-1/2} of Algorithm 1 step 5:
 * Phi = L U (L overwritten by Phi), Y+ = Q Phi D V+, X = diag(I,-I) Y+ Lambda^{-1/2},
 * Y = diag(I,-I) X. L, W, tau: FP64 or FP32 (fp32); Vs, lam: FP64 as produced by
 * bse_stage_tdeig; X, Y (Y nullable): 2n x n complex128, ldx >= 2n. */
size_t bse_stage_backtransform_worksize(int m, int fp32);
int bse_stage_backtransform(int m, void* L, int ldl, const void* W, int ldw, const void* tau, const double* Vs,
                            const double* lam, double* X, double* Y, int ldx, int fp32, void* work, void* stream);

/* Eq. absp weights w_j = (d_r^H x_j)(y_j^H d_l)/(y_j^H x_j), y_j = diag(I,-I) x_j.
 * X: 2n x n complex128 (ldx >= 2n); d_r, d_l: 2n complex128; w: n complex128. */
int bse_stage_weights(int n, const double* X, int ldx, const double* d_r, const double* d_l, double* w,
                      void* stream);

/* FP64 structure-preserving refinement of (lam, X) in place (X: 2n x n complex128,
 * ld 2n) against the FP64 M of bse_stage_form_M, at most max_sweeps sweeps of a
 * Newton-type correction on the pencil M u = lambda (-iJ) u, u = Q^H x (Theorem 2,
 * Eq. GMG, Theorem 3). The negative half stays the exact conjugate, so the +/-
 * pairing and y = diag(I,-I) x are preserved. SYNCHRONISES the stream (it reads
 * the convergence measures on the host between sweeps).
 * diag3 (nullable, host): {max scaled residual, max rel. eigenvalue change of the
 * last sweep, max rel. change of the first sweep}. */
size_t bse_stage_refine_worksize(int n);
int bse_stage_refine(int n, const double* M, double* lam, double* X, int max_sweeps, void* work, int* dev_status,
                     void* stream, int* sweeps, double* diag3);

/* Gaussian-broadened spectral density and absorption spectrum (Eq. DOS, Eq. absp,
 * Section 5's Gaussian of standard deviation sigma > 0), device pointers:
 * lambda: n positive eigenvalues; w: n complex128 weights (nullable when eps is
 * NULL); omega: n_omega grid energies; dos: n_omega out; eps: n_omega complex128
 * out (nullable). Sums over every eigenvalue (terms below the FP64 range are
 * exact zeros and skipped). */
int bse_stage_broaden(int n, const double* lambda, const double* w, int n_omega, const double* omega, double sigma,
                      double* dos, double* eps, void* stream);

/* ---- tensor-core products (no counterpart in the paper: the FP64-accurate residual
 * of the refinement runs on the bf16 tensor cores) ---------------------------- */

/* C (M x N FP32, column-major, ldc) = A B^T on the tcgen05 tensor cores, with
 * A: M x K bf16 and B: N x K bf16, both K-contiguous with row pitch ldk
 * (ldk >= K, ldk % 8 == 0, bases 16-byte aligned). FP32 accumulation: the tensor
 * cores sum 256-deep chunks, the chunks are added in FP32 registers. A bounded
 * internal wait that gives up stores BSE_ERR_TIMEOUT in dev_status. */
int bse_tc_gemm_bf16(int M, int N, int K, const void* A, const void* B, int ldk, float* C, int ldc, int* dev_status,
                     void* stream);

/* C (M x N FP64, column-major, ldc) = A B to FP64-level accuracy on the bf16
 * tensor cores by error-free digit splitting (Ozaki scheme): row i of A is the
 * K-vector A + i*lda (for a symmetric matrix stored column-major, the matrix
 * itself), column j of B is B + j*ldb. s digits of beta bits per operand give
 * about beta*s - 1 bits relative to the largest entry of each row of A times that
 * of each column of B; beta is the largest width <= 8 for which the 256-deep chunk
 * sums stay exact (K >= 256: beta <= 8) and one anti-diagonal's integer sum over
 * K stays below 2^31 (K 2^(2 beta - 2) s < 2^31: beta = 8 for K = 16384 up to
 * s = 7, 7 beyond); 1 <= s <= 11, s (s+1)/2 tensor-core passes (digit pairs
 * p + q < s). The
 * tensor cores sum each pair exactly over 256-deep chunks and the chunks are
 * added as integers, so the result does not depend on the launch shape.
 * work: bse_ozaki_worksize bytes. */
size_t bse_ozaki_worksize(int M, int N, int K, int s);
/* Digit width beta (bits) the digit-split product uses for reduction length K
 * with one digit (K >= 1; BSE_ERR_ARG otherwise); more digits can lower it, see
 * bse_ozaki_gemm. */
int bse_ozaki_digit_bits(int K);
int bse_ozaki_gemm(int M, int N, int K, const double* A, int lda, const double* B, int ldb, double* C, int ldc, int s,
                   void* work, int* dev_status, void* stream);

/* C (M x N FP32, column-major, ldc) = alpha op(A) op(B) + beta C on the tcgen05
 * tensor cores (kind::tf32), op(X) = X or X^T (trans flags), all column-major.
 * split = 1: 3xTF32 -- each operand value x = hi + lo with hi = x rounded to TF32
 * and lo = x - hi, accumulating hi*hi + hi*lo + lo*hi in FP32 (FP32-level
 * accuracy); split = 0: one TF32 pass. uplo = 1 (2) writes only C(i,j) with i >= j
 * (i > j) and needs M == N; 0 writes all of C. A and B need 16-byte aligned bases
 * and leading dimensions divisible by 4 (TMA pitch rule), else BSE_ERR_ARG. A
 * bounded internal wait that gives up stores BSE_ERR_TIMEOUT in dev_status. This
 * is the kernel behind the FP32 products of the mixed path. */
int bse_tc32_gemm(int M, int N, int K, float alpha, const float* A, int lda, int transA, const float* B, int ldb,
                  int transB, float beta, float* C, int ldc, int uplo, int split, int* dev_status, void* stream);

/* Engine of the FP32 products inside the mixed path, wherever the operand
 * layout allows the tensor cores: 2 (default) = 3xTF32 on operands split once
 * into K-major TF32 hi / lo planes in global memory (an internal buffer per
 * device and stream, grown on demand) for products with M N >= 500 (M + N)
 * (M N halved for a triangular C), the splitting in shared memory inside the
 * GEMM kernel for the smaller ones; 3 = pre-split planes for every product;
 * 1 = splitting in shared memory for every product; 0 = the SIMT FP32 kernel
 * everywhere. Modes 0, 1 and 3 are for comparisons; modes 1, 2 and 3 give
 * bit-identical products. bse_tc32_gemm with split = 1 follows modes 2 and 3
 * and splits in shared memory otherwise. Process-wide; BSE_ERR_ARG outside
 * 0..3. */
int bse_set_fp32_gemm(int mode);

#ifdef __cplusplus
}
#endif
#endif /* BSE_GB300_STAGES_H */
