/*
 * bse.h -- C ABI of the GB300-native structure-preserving Bethe--Salpeter
 * eigensolver (Shao, da Jornada, Yang, Deslippe, Louie, "Structure Preserving
 * Parallel Algorithms for Solving the Bethe--Salpeter Eigenvalue Problem").
 *
 * Problem (Section 1, Eq. 1-2; Eq. cond):  given A = A^H and B = B^T in C^{n x n}
 * with Omega = [A B; conj(B) conj(A)] positive definite, compute every positive
 * eigenvalue lambda_j of H = [A B; -conj(B) -conj(A)], the right eigenvectors x_j
 * and left eigenvectors y_j = diag(I,-I) x_j normalised so that Y^H X = I
 * (Theorem 3), and the optical-absorption weights of Eq. absp.
 *
 * Conventions shared by every entry point
 *   - Complex matrices are interleaved complex128 (re, im pairs of double),
 *     COLUMN-MAJOR, with a leading dimension counted in complex elements.
 *   - Only the LOWER triangles of A and B are read (LAPACK 'L'); the upper
 *     triangles are implied by A = A^H and B = B^T and are never checked.
 *   - lambda is returned ascending; column j of X and Y belongs to lambda[j].
 *   - Eigenvectors are unique up to a unit factor; the complex solves fix it so
 *     that the largest-modulus entry of the top half of x_j (the first of equal
 *     ones) is real and positive, y_j carrying the same factor.
 *   - Pointers may be host or device memory; the library tells them apart
 *     (cudaPointerGetAttributes). The caller owns every buffer it passes.
 *     The library owns its workspace and every bse_sol it hands out.
 *   - Every call returns an int status: BSE_OK (0) or a negative BSE_ERR_*.
 *     No C++ exception crosses this boundary. bse_last_error() gives text.
 *   - A context is not thread safe except bse_submit/bse_poll, which may be
 *     called from any thread.
 */
#ifndef BSE_GB300_H
#define BSE_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define BSE_OK 0
#define BSE_ERR_ARG (-1)           /* invalid argument (size, pointer, flag)           */
#define BSE_ERR_NOT_DEFINITE (-2)  /* Eq. cond fails: Cholesky of M met a pivot <= 0;   */
                                   /* bse_info.info holds the 1-based pivot column      */
#define BSE_ERR_NOT_CONVERGED (-3) /* bisection / refinement did not converge           */
#define BSE_ERR_NOMEM (-4)         /* device allocation failed or HBM budget exceeded   */
#define BSE_ERR_BUSY (-5)          /* request queue full (bse_submit)                   */
#define BSE_ERR_TIMEOUT (-6)       /* a bounded wait gave up                            */
#define BSE_ERR_CUDA (-7)          /* CUDA runtime error (see bse_last_error)           */
#define BSE_ERR_NO_TICKET (-8)     /* bse_poll: unknown ticket                          */

/* ---- precision modes ---------------------------------------------------- */
#define BSE_FP64 0          /* every stage in FP64 arithmetic                         */
#define BSE_MIXED 1         /* FP32 bulk (M copy, L, W, tridiagonal reduction,        */
                            /* back-transform) with FP64 tridiagonal eigensolve;      */
                            /* no refinement: FP32-level accuracy, reported           */
#define BSE_MIXED_REFINED 2 /* BSE_MIXED followed by FP64 structure-preserving        */
                            /* eigenpair refinement to FP64-level accuracy            */

typedef struct bse_ctx bse_ctx; /* one GPU, one stream, a workspace cache      */
typedef struct bse_sol bse_sol; /* device-resident solution (lambda, X)        */

/* Per-call diagnostics (all fields written by bse_solve). */
typedef struct bse_info {
  int status;          /* same as the return value                                   */
  int info;            /* BSE_ERR_NOT_DEFINITE: 1-based pivot column of M            */
  int precision;       /* the mode that ran                                          */
  int sweeps;          /* refinement sweeps done (BSE_MIXED_REFINED)                 */
  double stage_ms[10]; /* device time per stage when timing is on (bse_set_timing):  */
                       /* 0 form M, 1 Cholesky, 2 form W, 3 tridiagonal reduction,   */
                       /* 4 tridiagonal eigensolve, 5 back-transform, 6 refinement,  */
                       /* 7 weights, 8 host<->device copies, 9 total                 */
  double refine_resid; /* max_j ||M z_j - lambda_j K z_j|| / (||M||_F ||z_j||) after   */
                       /* the last refinement sweep (0 if no refinement ran)          */
  double refine_dlam;  /* max_j |dlambda_j| / lambda_j of the last sweep              */
  double unrefined_dlam; /* max_j |dlambda_j| / lambda_j of the first sweep: the      */
                         /* FP32 path's own eigenvalue error estimate                 */
} bse_info;

/* Create a context on CUDA device `device`. hbm_budget caps the bytes of
 * workspace the context may hold (0 = 90% of the device's free memory).
 * The context creates its own non-blocking stream. */
int bse_create(bse_ctx** ctx, int device, size_t hbm_budget);

/* Release every workspace buffer and the stream. Outstanding bse_sol objects
 * stay valid (they own their memory). Safe on NULL. */
int bse_destroy(bse_ctx* ctx);

/* Make the context issue its work on `stream` (a cudaStream_t; NULL restores
 * the context's own stream). The library never synchronises other streams. */
int bse_set_stream(bse_ctx* ctx, void* stream);

/* Record per-stage device times into bse_info.stage_ms (adds event syncs). */
int bse_set_timing(bse_ctx* ctx, int on);

/* Solve one problem (Algorithm 1 with Algorithm 3 for its steps 4-5), 1 <= n <= 32767.
 *   n       problem size (H is 2n x 2n), n >= 1
 *   A, lda  n x n complex128, column-major, lower triangle read (host or device)
 *   B, ldb  same for B
 *   precision  BSE_FP64 | BSE_MIXED | BSE_MIXED_REFINED
 *   lambda  out: n doubles, ascending (host or device); may be NULL
 *   X       out: 2n x n complex128, ld = 2n: right eigenvectors x_j (may be NULL)
 *   Y       out: 2n x n complex128, ld = 2n: left eigenvectors y_j = diag(I,-I) x_j
 *           (may be NULL)
 *   keep    out (nullable): a device-resident solution for bse_spectrum;
 *           free it with bse_sol_free
 *   info    out (nullable): diagnostics
 * Blocks until the results are in the caller's buffers. Errors: BSE_ERR_ARG,
 * BSE_ERR_NOT_DEFINITE (info->info = pivot column), BSE_ERR_NOMEM, BSE_ERR_CUDA. */
int bse_solve(bse_ctx* ctx, int n, const double* A, int lda, const double* B, int ldb,
              int precision, double* lambda, double* X, double* Y, bse_sol** keep,
              bse_info* info);

/* Real Bethe-Salpeter problem (Section 3.2, Theorem 5, Algorithm 2): A, B real
 * symmetric n x n (FP64, col-major, lower triangles read, host or device) with
 * A + B > 0 and A - B > 0.
 *   lambda  out: n positive eigenvalues, ascending
 *   X1, X2  out (nullable): n x n real each, ld n, with
 *           H [X1; X2] = [X1; X2] diag(lambda), H = [A B; -B -A], and
 *           X1^T X1 - X2^T X2 = I (column signs: largest-modulus entry positive)
 * Step 1 factors A + B and A - B separately; the SVD of L2^T L1 (step 2) is
 * computed through the skew embedding W = [0 L1^T L2; -L2^T L1 0] by the same
 * tridiagonal machinery as bse_solve, and X1, X2 follow as in step 3. Blocks
 * until the outputs are written. Errors as bse_solve (BSE_ERR_NOT_DEFINITE:
 * info->info = pivot column, counted from A + B's first column, then A - B's at n). */
int bse_solve_real(bse_ctx* ctx, int n, const double* A, int lda, const double* B, int ldb, int precision,
                   double* lambda, double* X1, double* X2, bse_info* info);

/* Absorption weights of Eq. absp for a kept solution:
 *   w_j = (d_r^H x_j)(y_j^H d_l) / (y_j^H x_j),  j = 0..n-1
 *   d_r, d_l  2n complex128 each (host or device)
 *   w         out: n complex128 (host or device)
 * The weights are complex in general (x_j != y_j) and invariant to the phase of
 * the eigenvectors. Blocks until w is written. */
int bse_spectrum(bse_ctx* ctx, const bse_sol* sol, const double* d_r, const double* d_l,
                 double* w);

/* Spectral density (Eq. DOS) and optical absorption spectrum (Eq. absp) of a
 * kept solution on a grid of energies, with the delta function replaced by the
 * Gaussian exp(-t^2/(2 sigma^2)) / (sqrt(2 pi) sigma) (Section 5):
 *   dos[k] = 1/(2n) sum_j [g(omega_k - lambda_j) + g(omega_k + lambda_j)]
 *            (all 2n eigenvalues +-lambda_j of H, Theorem 1)
 *   eps[k] = sum_j w_j g(omega_k - lambda_j), w_j the Eq. absp weights
 *   omega     n_omega energies (host or device)
 *   sigma     > 0
 *   d_r, d_l  2n complex128 dipole vectors, or both NULL (then eps must be NULL)
 *   dos       out: n_omega doubles (host or device)
 *   eps       out (nullable): n_omega complex128 (host or device)
 * Blocks until the outputs are written. Errors: BSE_ERR_ARG, BSE_ERR_CUDA. */
int bse_absorption(bse_ctx* ctx, const bse_sol* sol, const double* d_r, const double* d_l, int n_omega,
                   const double* omega, double sigma, double* dos, double* eps);

/* Size n and device pointers of a kept solution (lambda: n doubles; X: 2n x n
 * complex128, ld 2n). The pointers stay owned by the solution. */
int bse_sol_view(const bse_sol* sol, int* n, const double** lambda_dev, const double** X_dev);

/* Free a kept solution. Safe on NULL. Its device memory goes back to the
 * device's memory pool (stream-ordered allocator), where later kept solutions
 * reuse it without a device-wide synchronisation. */
int bse_sol_free(bse_sol* sol);

/* ---- request queue with continuous batching ---------------------------- */
/* A request: the problem and where its results go (host memory). The buffers
 * must stay valid until bse_poll reports the ticket done. */
typedef struct bse_request {
  int n;
  const double* A; /* n x n complex128, col-major, ld = n, lower triangle read */
  const double* B;
  const double* d_r; /* nullable: 2n complex128 dipole vectors for weights   */
  const double* d_l;
  int precision;   /* BSE_FP64 | BSE_MIXED | BSE_MIXED_REFINED                */
  double* lambda;  /* out: n                                                   */
  double* X;       /* out (nullable): 2n x n complex128                        */
  double* w;       /* out (nullable): n complex128 weights (needs d_r, d_l)    */
} bse_request;

typedef struct bse_result {
  int status;        /* BSE_OK or a BSE_ERR_* of this request                  */
  int n;
  double t_submit;   /* seconds on the context's monotonic clock               */
  double t_start;    /* admission time                                          */
  double t_done;     /* completion time                                         */
  double refine_dlam;
} bse_result;

/* Start the request loop: `slots` worker threads, each with its own stream and
 * workspace. A queued request is admitted (first fit in arrival order) when a
 * slot is free and its workspace fits the HBM budget next to the running ones;
 * each admitted request runs the kernels of one bse_solve on its slot's stream,
 * so requests on different slots overlap on the device. */
int bse_serve_start(bse_ctx* ctx, int slots);

/* Queue a request; never blocks. BSE_ERR_BUSY if the queue is full. */
int bse_submit(bse_ctx* ctx, const bse_request* req, uint64_t* ticket);

/* Non-blocking completion check. *done = 1 and *res filled once finished;
 * the ticket is then forgotten. BSE_ERR_NO_TICKET for unknown tickets. */
int bse_poll(bse_ctx* ctx, uint64_t ticket, bse_result* res, int* done);

/* Drain the queue and stop the scheduler thread (waits at most timeout_s,
 * BSE_ERR_TIMEOUT after that). */
int bse_serve_stop(bse_ctx* ctx, double timeout_s);

/* ---- batched solves ----------------------------------------------------- */
/* Solve `count` independent problems of sizes ns[i] in one call. A[i], B[i]
 * are host or device pointers (ld = ns[i]); lambdas[i] (ns[i] doubles) and
 * Xs[i] (2ns[i] x ns[i] complex128, nullable) receive the results. The
 * problems are dealt largest first to several streams of the context's GPU
 * (16 by default; BSE_BATCH_SLOTS overrides, 1..32), each with its own workspace
 * cache, so their pipelines overlap on the device; every problem runs the
 * kernels of a single bse_solve and gets bit-for-bit its results. Per-problem
 * status goes to statuses[i] (nullable); the return value is the first
 * failure, or BSE_OK. Blocks until every result is in place. */
int bse_solve_batched(bse_ctx* ctx, int count, const int* ns, const double* const* A,
                      const double* const* B, int precision, double* const* lambdas,
                      double* const* Xs, int* statuses);

/* ---- launch accounting and kernel timing -------------------------------- */
/* Number of kernels this library has launched since it was loaded (all
 * contexts and threads). */
long long bse_launch_count(void);

/* Kernel profiling: while on, each launch of a kernel class is bracketed by
 * CUDA events on its stream and charged with the algorithmic bytes / flops of
 * that launch (e.g. the skew SYMV: the strict lower triangle of the trailing
 * matrix, once). Turning it on or off clears the totals. Adds event records to
 * every launch: use it for an instrumented run, not a timed one. */
int bse_kprof_enable(int on);

/* Totals for kernel class k since profiling was turned on (synchronises on the
 * recorded events): 0 form M, 1 Cholesky diagonal blocks, 2 FP64 GEMM, 3 FP32
 * GEMM, 4 skew SYMV, 5 other tridiagonal-column kernels, 6 bisection,
 * 7 tridiagonal eigenvectors, 8 weights, 9 elementwise, 10 digit-product
 * (FP64-accurate) tensor-core GEMM, 11 3xTF32 tensor-core GEMM, 12 band
 * reduction panel QR, 13 bulge chasing, 14 bulge-chasing back-transform,
 * 15 TF32 hi / lo splitting of FP32 GEMM operands. BSE_ERR_ARG for an unknown
 * class. */
int bse_kprof_read(int k, long long* launches, double* ms, double* bytes, double* flops);

/* Text of the last error recorded on this thread ("" if none). */
const char* bse_last_error(void);

/* Library version string. */
const char* bse_version(void);

#ifdef __cplusplus
}
#endif
#endif /* BSE_GB300_H */
