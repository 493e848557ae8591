/*
 * rxr.h -- C ABI of librxr: randomized XR-preconditioned CholeskyQR
 * (rLU- and rQR-CholeskyQR) of tall-and-skinny matrices on one GB300 GPU.
 *
 * Method: Fan, Guo & Lin, "A Novel Randomized XR-Based Preconditioned
 * CholeskyQR Algorithm".  For A (m x n, m >= n, full rank) the library computes
 * the thin QR factorisation A = QR of Section 1 (Q^T Q = I_n, R upper triangular)
 * by
 *   1. a Gaussian sketch Y = Omega A with s >= n rows (Section 2.3, "Gaussian
 *      Ensemble"; the paper's l is s here), Omega drawn in-kernel from
 *      Philox4x32-10 and never stored;
 *   2. R_s = the R factor of Y by LU with partial pivoting (Algorithm 4) or by
 *      Householder QR (Algorithm 5), rows scaled so that diag(R_s) > 0;
 *   3. X = A R_s^{-1} (row-wise substitution), fused with G = X^T X;
 *   4. CholeskyQR (Algorithm 1) on X, repeated `passes` times as in
 *      CholeskyQR2 (Algorithm 2): R_p = chol(G_p), X <- X R_p^{-1};
 *   5. Q = X and R = R_passes ... R_1 R_s.
 *
 * Conventions for every entry point:
 *  - Matrices are FP64, column-major (LAPACK style): entry (i, j) of a matrix
 *    with leading dimension ld is p[i + j*ld].  lda >= m, ldq >= m, ldr >= n.
 *  - Matrix pointers are DEVICE pointers owned by the caller unless the
 *    function name ends in _host.  The library never frees caller memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Work is enqueued on it; blocking calls synchronise it.
 *  - Return value: 0 on success; -i when argument i (1-based) is invalid
 *    (LAPACK `info` style, nothing is launched); a positive RXR_ERR_* code
 *    when the computation ran but failed.  No C++ exception crosses the ABI and
 *    there is no CPU fallback: without a usable GPU the calls return RXR_ERR_CUDA.
 *  - Results are bitwise reproducible for fixed inputs, seed and launch
 *    configuration (counter-based random numbers, fixed-order reductions).
 */
#ifndef RXR_H
#define RXR_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define RXR_API __attribute__((visibility("default")))
#else
#define RXR_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* XR factorisation of the sketch (Section 2.2).  RXR_NONE skips the sketch and
 * takes R_s = I, i.e. plain CholeskyQR repeated `passes` times (Algorithms 1
 * and 2), the paper's unpreconditioned comparator.  RXR_SKETCH_ROWS, OR-ed into
 * RXR_LU or RXR_QR, takes the sketch by row extraction (Section 2.3, the
 * paper's experimental choice; Theorem 3.2) instead of the Gaussian product:
 * s rows of A drawn independently with probability 1/m each (with
 * replacement), draw k from Philox4x32-10 at counter (k_lo, k_hi, 0, 3) and key
 * (seed_lo, seed_hi), u = out0 + 2^32 out1, row floor(u m / 2^64).  Coherent A
 * (large m max_i ||Q(i,:)||^2, e.g. A = [I; 0]) can leave that sketch
 * rank-deficient: RXR_ERR_SKETCH_SINGULAR.  RXR_SHIFTED is the shifted
 * CholeskyQR comparator of Section 2.1 (sCholeskyQR3 with passes = 3): no
 * sketch, R_1 = chol(A^T A + eps I) with eps = 1e-15 ||A||_2^2 (the shift of the
 * paper's experiments; ||A||_2^2 by 40 power iterations on A^T A), then
 * passes - 1 plain CholeskyQR steps.  RXR_NONE and RXR_SHIFTED ignore s and take
 * n <= 128; the batched form takes neither RXR_SHIFTED nor RXR_SKETCH_ROWS. */
typedef enum { RXR_LU = 0, RXR_QR = 1, RXR_NONE = 2, RXR_SHIFTED = 3 } rxr_variant;
#define RXR_SKETCH_ROWS 16

/* Arithmetic of the passes over A (the m-row contractions).
 *   RXR_FP64          : FP64 FMAs throughout.
 *   RXR_SPLIT_BF16    : every contraction over the m rows runs on the tcgen05
 *                       tensor cores: the sketch, both Grams, the trailing
 *                       updates of the substitutions (their 16-column diagonal
 *                       blocks are FP64 solves), and, for n <= 64 and m >= 2^17,
 *                       the middle pass's and the last pass's applies through
 *                       the explicit inverse (each chosen on the device; the
 *                       substitution otherwise).  Operands are exact balanced
 *                       8-bit digit slices of FP64 values (FP16 operands for
 *                       n <= 128, BF16 above) with FP32 accumulation kept exact
 *                       and combined in FP64, so these contractions are
 *                       FP64-grade (error about 2^-53 of the largest entries per
 *                       column), except the last apply's correction
 *                       X (R_P^{-1} - I) for n <= 128, formed in FP32 when
 *                       |R_P^{-1} - I| <= 2^-38 (error below 2^-55 |X|).
 *                       The sketch takes Omega on the 2^-12 grid (the same
 *                       Philox draws, rint(4096 z) / 4096).  The n x n
 *                       factorisations, inverses and all combining stay FP64.
 *   RXR_SPLIT_PRECOND : only the two contractions that shape the
 *                       preconditioner leave FP64: the sketch (as above) and
 *                       the first pass's Gram (BF16x3 for n <= 128, FP64-grade
 *                       digit slices above).  X = A R_s^{-1}, the later Grams
 *                       and every apply are FP64 FMAs; the repeated FP64 pass
 *                       wins the accuracy back (Appendix A's perturbation
 *                       argument).  Without a sketch (RXR_NONE, RXR_SHIFTED)
 *                       it is RXR_FP64.  Taken by rxr_cholqr, rxr_cholqr_async,
 *                       rxr_cholqr_host, rxr_rsvd and rxr_sketch (the split
 *                       sketch); the other entry points take the first two. */
typedef enum { RXR_FP64 = 0, RXR_SPLIT_BF16 = 1, RXR_SPLIT_PRECOND = 3 } rxr_precision;

/* Positive status codes. */
enum {
    RXR_OK = 0,
    RXR_ERR_SKETCH_SINGULAR = 1, /* |pivot| <= n u max|pivot| or non-finite in step 2:
                                    the sketch (or A) is rank deficient (Section 2.2) */
    RXR_ERR_CHOL_BREAKDOWN = 2,  /* non-positive / non-finite Cholesky pivot (Section 2.1);
                                    rxr_last_info() gives the pass and column */
    RXR_ERR_NONFINITE = 3,       /* A holds NaN or Inf */
    RXR_ERR_CUDA = 4,            /* a CUDA runtime call failed (no GPU, bad pointer, ...) */
    RXR_ERR_TIMEOUT = 5,         /* a bounded device-side wait gave up */
    RXR_ERR_NOMEM = 6,           /* the library could not allocate its workspace */
    RXR_ERR_UNSUPPORTED = 7,     /* valid arguments outside what this build supports */
    RXR_ERR_BAD_SPARSE = 8,      /* rxr_rsvd: a CSR row pointer or column index out of range */
    RXR_ERR_NO_CONVERGENCE = 9   /* rxr_rsvd: the k x k Jacobi SVD still rotated a pair by more
                                    than 2^-27 in its last allowed sweep (40, or the test hook's) */
};

/* Limits of this build. */
#define RXR_MAX_N 512
#define RXR_MAX_S 2048

typedef struct rxr_ctx *rxr_handle;

/* Create a handle bound to CUDA device `device`; it owns a workspace (grown on
 * demand with cudaMalloc unless rxr_set_workspace supplied one), a device
 * status word and pinned host staging.  Returns 0, -1 (h NULL), -2 (bad
 * device) or RXR_ERR_CUDA. */
RXR_API int rxr_create(rxr_handle *h, int device);

/* Release everything the handle owns.  Safe on NULL. */
RXR_API int rxr_destroy(rxr_handle h);

/* Bytes of device workspace that rxr_cholqr needs for these sizes (the sketch
 * and Gram partial sums, the s x n sketch, the n x n factors and the status
 * word).  The m x n intermediate X lives in the caller's Q. */
RXR_API int rxr_workspace_bytes(int64_t m, int64_t n, int64_t s, int prec, size_t *bytes);

/* Give the handle caller-owned device workspace (e.g. from PyTorch's caching
 * allocator); `bytes` must be at least rxr_workspace_bytes(...) of the calls
 * that follow, else they return RXR_ERR_NOMEM.  NULL returns to self-managed
 * workspace.  The memory must stay valid until replaced or the handle dies. */
RXR_API int rxr_set_workspace(rxr_handle h, void *d_workspace, size_t bytes);

/* Factorise A = QR (Algorithms 4/5 + repeated CholeskyQR pass, see top).
 *   A (1)           device, m x n, read only (unless Q == A: in-place allowed
 *                   when ldq == lda; A is then overwritten by Q).
 *   m, n, lda (2-4) m >= n >= 1, n <= RXR_MAX_N, lda >= m.
 *   variant (5)     RXR_LU, RXR_QR or RXR_NONE.
 *   s (6)           sketch rows, n <= s <= RXR_MAX_S (paper: l >= n; l = 2n in
 *                   Section 4).  Ignored for RXR_NONE.
 *   seed (7)        Philox key of Omega.
 *   passes (8)      CholeskyQR passes, 1..3 (Algorithms 4/5 print one; two =
 *                   CholeskyQR2 on X).
 *   Q, ldq (9-10)   device, m x n output (holds X between passes), ldq >= m.
 *   R, ldr (11-12)  device, n x n output (strictly lower part written as 0),
 *                   ldr >= n; R == NULL skips R ("R-less" QR, footnote to
 *                   Algorithm 2).
 *   prec (13)       rxr_precision.
 *   stream (14)     cudaStream_t.
 * Blocking: synchronises `stream` and returns the status.  On a positive code
 * Q and R hold partial results. */
RXR_API int rxr_cholqr(rxr_handle h, const double *A, int64_t m, int64_t n, int64_t lda, int variant, int64_t s,
               uint64_t seed, int passes, double *Q, int64_t ldq, double *R, int64_t ldr, int prec, void *stream);

/* Same as rxr_cholqr but asynchronous and stream-capturable: nothing waits on
 * the host.  The status is written on the device to d_status[0..3] = {code,
 * pass, column, 0} (caller-owned device memory, 16 bytes) when the stream
 * reaches the end of the sequence.  Argument errors are still returned
 * synchronously. */
RXR_API int rxr_cholqr_async(rxr_handle h, const double *A, int64_t m, int64_t n, int64_t lda, int variant, int64_t s,
                     uint64_t seed, int passes, double *Q, int64_t ldq, double *R, int64_t ldr, int prec,
                     void *stream, int *d_status);

/* End-to-end form with HOST buffers: copies A (pageable or pinned host
 * memory) to the device, factorises, and copies Q and R back; the device
 * buffers are owned by the handle.  Blocking.  Arguments as rxr_cholqr, with
 * hA, hQ, hR host pointers (hR may be NULL). */
RXR_API int rxr_cholqr_host(rxr_handle h, const double *hA, int64_t m, int64_t n, int64_t lda, int variant, int64_t s,
                    uint64_t seed, int passes, double *hQ, int64_t ldq, double *hR, int64_t ldr, int prec,
                    void *stream);

/* Batched form: `count` independent problems A_k (m_k x n_k) factorised as
 * one job (the many tall-skinny blocks of block Krylov, LOBPCG or randomized
 * SVD that Sections 1 and 5 mention).  Arrays are HOST arrays of length count;
 * the matrix pointers in them are device pointers.  variant, passes and prec
 * are common; s_k, seed_k per problem.  Per-problem status {code, pass,
 * column, 0} goes to d_status[4k .. 4k + 3] (device, caller owned).
 *   RXR_FP64 with RXR_LU, RXR_QR or RXR_NONE (n_k <= 128): one launch per stage
 *     for the whole batch; the sketch, the substitutions (+ Grams) and the
 *     reductions run persistent CTAs that pull (problem, row chunk) items from a
 *     device work queue, the row chunks sized by the tuned table of
 *     csrc/batched_tuning.h; the O(n^3) steps run one CTA per problem.
 *   Any other precision or variant: every problem's own launch sequence (the
 *     same kernels and results as rxr_cholqr), spread over eight streams that
 *     fork from and join back into `stream`.
 * Blocking; returns the first non-zero problem status (or 0). */
RXR_API int rxr_cholqr_batched(rxr_handle h, int count, const double *const *A, const int64_t *m, const int64_t *n,
                       const int64_t *lda, int variant, const int64_t *s, const uint64_t *seed, int passes,
                       double *const *Q, const int64_t *ldq, double *const *R, const int64_t *ldr, int prec,
                       void *stream, int *d_status);

/* Batched plan: the same batch prepared once -- arguments checked, every
 * problem's workspace allocated (device memory owned by the plan) and the job
 * tables copied to the device -- then run any number of times.
 * rxr_batch_run only enqueues device work on `stream` (memsets and kernel
 * launches, plus event fork/join across the plan's streams for the
 * per-problem form): no host synchronisation and no allocation, so it can be
 * captured into a CUDA graph; the statuses land in d_status when the stream
 * reaches the end of the run.  The matrices named at creation are read and
 * written by every run (update their contents in place between runs).  A plan
 * must not run on two streams at once.  rxr_batch_create: arguments as
 * rxr_cholqr_batched, plan (17) receives the plan; returns 0, a negative
 * argument error, RXR_ERR_UNSUPPORTED, RXR_ERR_NOMEM or RXR_ERR_CUDA.  The
 * handle must outlive the plan. */
typedef struct rxr_batch *rxr_batch_plan;
RXR_API int rxr_batch_create(rxr_handle h, int count, const double *const *A, const int64_t *m, const int64_t *n,
                             const int64_t *lda, int variant, const int64_t *s, const uint64_t *seed, int passes,
                             double *const *Q, const int64_t *ldq, double *const *R, const int64_t *ldr, int prec,
                             int *d_status, rxr_batch_plan *plan);
RXR_API int rxr_batch_run(rxr_batch_plan plan, void *stream);
RXR_API int rxr_batch_destroy(rxr_batch_plan plan);

/* Test hooks: they make error paths that correct inputs never reach run on
 * request, without faulting or hanging the GPU.  They are meant for tests.
 *   RXR_HOOK_STALL, value != 0: the following factorisations on this handle
 *     (rxr_cholqr and the calls built on it) make one bounded device-side wait
 *     run out.  The FP64 path's sketch kernel (its first CTA) and the
 *     split path's fused substitution (n <= 64, the first CTA's first row
 *     group) skip their first TMA copy and wait on an mbarrier that nothing
 *     arrives at.  No copy is in flight.  After about a second per wait the
 *     kernel records RXR_ERR_TIMEOUT, frees its tensor memory and returns.
 *     Every later kernel of the call returns at once, and the call returns
 *     RXR_ERR_TIMEOUT.  Only a TMA-eligible A (16-byte aligned, even lda)
 *     takes these waits.  value 0 restores normal operation; the handle stays
 *     usable.
 *   RXR_HOOK_JACOBI_SWEEPS, value in 0..40: caps the sweeps of rxr_rsvd's
 *     Jacobi SVD (0 = the default bound, 40); a cap it reaches before
 *     convergence makes rxr_rsvd return RXR_ERR_NO_CONVERGENCE.
 *   RXR_HOOK_BATCH_CTAS, value = (bucket << 8) | c: the batched form's row
 *     chunking for problems of n-bucket `bucket` (0..4: n <= 8, 16, 32, 64,
 *     128) becomes c CTAs per SM per stage (c = 0: the tuned table of
 *     csrc/batched_tuning.h); used by the tuning script.
 * Returns 0, -1 (h NULL), -2 (unknown hook) or -3 (value out of range). */
#define RXR_HOOK_STALL 1
#define RXR_HOOK_JACOBI_SWEEPS 2
#define RXR_HOOK_BATCH_CTAS 3
RXR_API int rxr_set_test_hook(rxr_handle h, int hook, int value);

/* Pass and column (0-based) of the last Cholesky breakdown seen by a blocking
 * call on this handle; both -1 if none. */
RXR_API int rxr_last_info(rxr_handle h, int *pass, int *column);

/* Static string for a status code. */
RXR_API const char *rxr_status_string(int code);

/* ---- Stage entry points: each runs one step of the path on the device.  They
 * expose the intermediates for testing and for callers that compose their own
 * pipeline (e.g. the least-squares preconditioner of Section 5.2, which only
 * needs R_s).  All are asynchronous on `stream` unless stated. ---- */

/* Standard normals of Omega (Section 2.3, Gaussian ensemble): for rows
 * i = row0..row0+rows-1 of A and sketch rows r < s, d_z[(i-row0)*s + r] = z,
 * Omega = z / sqrt(s).  The counter convention: Philox4x32-10 with key
 * (seed_lo, seed_hi) and counter (i_lo, i_hi, k, 0) gives z for r = 4k..4k+3
 * by Box-Muller on FP32 uniforms u = ((x >> 8) + 1) 2^-24.  d_z device,
 * rows * s floats. */
RXR_API int rxr_omega(uint64_t seed, int64_t s, int64_t row0, int64_t rows, float *d_z, void *stream);

/* Y = Omega A (s x n, column-major with leading dimension ldy >= s), step 1.
 * prec selects FP64 or the split BF16 tensor-core contraction. */
RXR_API int rxr_sketch(rxr_handle h, const double *A, int64_t m, int64_t n, int64_t lda, int64_t s, uint64_t seed,
               double *Y, int64_t ldy, int prec, void *stream);

/* Row-extraction sketch Y = P A (Section 2.3): row k of Y (s x n, ldy >= s)
 * is row idx_k of A, the draws of RXR_SKETCH_ROWS.  A is a read-only device
 * buffer (lda >= m).  Blocking; 0, RXR_ERR_NONFINITE (a drawn row holds NaN or
 * Inf) or a negative argument error. */
RXR_API int rxr_sketch_rows(rxr_handle h, const double *A, int64_t m, int64_t n, int64_t lda, int64_t s, uint64_t seed,
                            double *Y, int64_t ldy, void *stream);

/* R_s (n x n upper, diag > 0, zeros below) = R factor of Y (s x n) by LU with
 * partial pivoting (RXR_LU) or Householder QR (RXR_QR), step 2.  Y is read
 * only.  Blocking; returns 0 or RXR_ERR_SKETCH_SINGULAR. */
RXR_API int rxr_xr_factor(rxr_handle h, const double *Y, int64_t s, int64_t n, int64_t ldy, int variant, double *Rs,
                  int64_t ldrs, void *stream);

/* X = A R^{-1} and G = X^T X (full symmetric n x n, leading dimension
 * ldg >= n), step 3.  X may alias A (ldx == lda); X == NULL computes G only
 * (RXR_FP64).  RXR_FP64: row-wise FP64 substitution fused with the FP64 Gram.
 * RXR_SPLIT_BF16: right-looking blocked substitution (FP64 diagonal blocks,
 * trailing updates on the tensor cores at FP64 grade: normwise backward
 * stable) and the FP64-grade tensor-core Gram (exact digit slices). */
RXR_API int rxr_precond_gram(rxr_handle h, const double *A, int64_t m, int64_t n, int64_t lda, const double *R,
                     int64_t ldr, double *X, int64_t ldx, double *G, int64_t ldg, int prec, void *stream);

/* G = X^T X (full symmetric n x n, ldg >= n) of a tall-skinny X (Algorithm 1
 * step 1).  RXR_FP64: FP64 FMAs, n <= 128.  RXR_SPLIT_BF16: the tensor-core
 * Gram with exact 7-digit splitting (FP64-grade: error about 2^-53 of
 * |X|^T |X| column-normwise), n <= 512.  RXR_SPLIT_PRECOND: the first-pass Gram
 * of that mode, BF16x3 on the tensor cores (three 8-bit significand chunks,
 * FP32 accumulation drained to FP64 every 64 rows; error about 2^-19 of
 * |X|^T |X|), n <= 128.  Blocking. */
RXR_API int rxr_gram(rxr_handle h, const double *X, int64_t m, int64_t n, int64_t ldx, double *G, int64_t ldg, int prec,
                     void *stream);

/* X <- X R^{-1} in place (Algorithm 1 step 3, the Q of a CholeskyQR pass),
 * R upper triangular n x n (leading dimension ldr >= n, read only), X m x n
 * column-major (ldx >= m).  RXR_FP64: row-wise FP64 substitution.
 * RXR_SPLIT_BF16, n <= 128: T = R^{-1} by FP64 back substitution; when every
 * |T - I| <= 2^-38 (R within rounding of I, as after a repeated CholeskyQR
 * pass) X + X (T - I) with the correction in FP32 (error below 2^-55 |X| per
 * term), else X T on the tensor cores at FP64 grade (exact digit splitting,
 * n <= 64) or the fused substitution (64 < n <= 128).
 * RXR_SPLIT_BF16, n > 128: the blocked substitution of rxr_precond_gram.
 * R's diagonal must be nonzero and finite (not checked: X is then not
 * finite).  Blocking; 0 or a negative argument error (-i: argument i). */
RXR_API int rxr_apply_rinv(rxr_handle h, double *X, int64_t m, int64_t n, int64_t ldx, const double *R, int64_t ldr,
                           int prec, void *stream);

/* Least squares min ||A x - b||_2 by the solver of Section 5.2, preconditioned
 * by the sketch's R factor: B = A R_s^{-1} (the fused precondition step, its
 * Gram G = B^T B at FP64 grade on either path), c = B^T b, R_G = chol(G),
 * y = R_G^{-1} R_G^{-T} c, x = R_s^{-1} y.  A (m x n, lda >= m, m >= n) and b
 * (m x k, ldb >= m, 1 <= k <= 64) read-only device buffers; x (n x k,
 * ldx >= n) device output; variant RXR_LU or RXR_QR, optionally
 * | RXR_SKETCH_ROWS; s, seed and prec as for rxr_cholqr.  The handle holds B
 * (m x n) as scratch.  Blocking; 0, RXR_ERR_SKETCH_SINGULAR,
 * RXR_ERR_CHOL_BREAKDOWN, RXR_ERR_NONFINITE (A or b) or a negative argument
 * error (-i: argument i). */
RXR_API int rxr_lstsq(rxr_handle h, const double *A, int64_t m, int64_t n, int64_t lda, const double *b, int64_t k,
                      int64_t ldb, int variant, int64_t s, uint64_t seed, double *x, int64_t ldx, int prec,
                      void *stream);

/* Randomized SVD with power iteration (Algorithm 7, Section 5.1) of a sparse
 * m x n matrix A, every orthonormalisation done by this library's CholeskyQR
 * (the replacement for Householder QR that Section 5.1 makes):
 *   Y = orth(A X); `iters` times: Y = orth(A^T Y), Y = orth(A Y);
 *   then B = Y^T A through Z = A^T Y = Q_z R_z (one more orth), R_z = U_r S V_r^T
 *   by one-sided Jacobi, and U = Y V_r, V = Q_z U_r, so that
 *   Y Y^T A = U diag(S) V^T, A^T U = V diag(S), S descending.
 * Orthonormalisation j (j = 0 .. 2 iters + 1) is rxr_cholqr(., variant, s,
 * seed + j, passes, prec) of an m x k or n x k block.
 * A in compressed sparse row form, DEVICE arrays: a_ptr int64[m+1] (a_ptr[0]
 * = 0, nondecreasing, a_ptr[m] = nnz), a_idx int32[nnz] column indices in
 * [0, n), a_val double[nnz]; the same form of A^T in t_ptr int64[n+1],
 * t_idx int32[nnz] (row indices of A) and t_val double[nnz] (the caller
 * builds A^T: the iteration multiplies by both).  An index or row pointer out
 * of range is reported as RXR_ERR_BAD_SPARSE (the arrays themselves must have
 * the stated lengths).  X: the n x k starting block (ldx >= n), read-only;
 * 1 <= k <= min(m, n), k <= 128; 0 <= iters <= 1000; variant, s (>= k),
 * passes and prec as for rxr_cholqr.  Outputs (device): U (m x k, ldu >= m),
 * S (k), V (n x k, ldv >= n).  The handle keeps 2 (m + n) k + max(m, n) k
 * doubles of scratch.  A rank of A below k makes a factorisation fail.
 * Blocking; 0, the first failure of the factorisations (RXR_ERR_*; for a
 * breakdown rxr_last_info gives its pass and column), RXR_ERR_BAD_SPARSE,
 * RXR_ERR_NO_CONVERGENCE (S holds the unconverged column norms, U and V are
 * not written), or a negative argument error (-i: argument i). */
RXR_API int rxr_rsvd(rxr_handle h, int64_t m, int64_t n, const int64_t *a_ptr, const int32_t *a_idx,
                     const double *a_val, const int64_t *t_ptr, const int32_t *t_idx, const double *t_val,
                     int64_t nnz, const double *X, int64_t ldx, int64_t k, int iters, int variant, int64_t s,
                     uint64_t seed, int passes, int prec, double *U, int64_t ldu, double *S, double *V, int64_t ldv,
                     void *stream);

/* ---- Row-sharded factorisation (Section 2.4's parallel scheme, whose
 * communication Section 2.5 tabulates): A is split by contiguous row blocks
 * across processes or GPUs.  Each shard runs these calls and the stage calls
 * above on its own rows; between stages the caller gathers the s x n sketch
 * partials or n x n Gram partials of all shards (an allgather, in rank order)
 * and sums them with rxr_sum_parts, so that every shard holds the same Y, G and
 * R and runs the small factorisations itself (no broadcast).  Q's rows stay on
 * their shard.  paper_2111_11148_gb300/sharded.py composes them over
 * torch.distributed. ---- */

/* Partial sketch of a row shard: Y = Omega[:, row0 .. row0 + m) A_shard / sqrt(s),
 * Omega's columns indexed by the GLOBAL row (row0 + i), so the sum of all
 * shards' partials is the sketch of the whole matrix (Section 2.3's Gaussian
 * ensemble, drawn as rxr_omega describes).  A (m x n, lda >= m, m >= 1: a shard
 * may hold fewer rows than n) read-only device buffer; Y (s x n, ldy >= s)
 * device output; 0 <= row0 <= 2^62 - m; prec as for rxr_sketch.  Blocking; 0,
 * RXR_ERR_NONFINITE or a negative argument error (-i: argument i). */
RXR_API int rxr_sketch_part(rxr_handle h, const double *A, int64_t m, int64_t n, int64_t lda, int64_t s,
                            uint64_t seed, int64_t row0, double *Y, int64_t ldy, int prec, void *stream);

/* out[e] = sum over k = 0 .. count - 1 of parts[k * len + e] (device arrays;
 * parts holds count blocks of len doubles, e.g. the gathered partials of count
 * shards) in a fixed order: k = 0, 1, ... for fewer than 256 blocks; from 256
 * on, lane l of a warp adds blocks l, l + 32, ... and a fixed shuffle tree
 * combines the lanes.  Every shard that sums the same gathered blocks gets the
 * same bits.  out must not overlap parts.
 * Asynchronous on stream; 0 or a negative argument error. */
RXR_API int rxr_sum_parts(rxr_handle h, const double *parts, int count, int64_t len, double *out, void *stream);

/* C = A B for upper-triangular n x n A and B (their upper triangles are read;
 * C's strictly lower part is written as 0): the R = R_P ... R_1 R_s
 * accumulation of Algorithms 2, 4 and 5.  Device buffers, column-major;
 * C may alias neither A nor B.  Asynchronous on stream; 0 or a negative
 * argument error. */
RXR_API int rxr_trmm_upper(rxr_handle h, const double *A, int64_t lda, const double *B, int64_t ldb, int64_t n,
                           double *C, int64_t ldc, void *stream);

/* Upper Cholesky factor R (R^T R = G; reads the upper triangle of G).
 * Blocking; returns 0 or RXR_ERR_CHOL_BREAKDOWN (column in rxr_last_info). */
RXR_API int rxr_cholesky(rxr_handle h, const double *G, int64_t n, int64_t ldg, double *R, int64_t ldr, void *stream);

/* Accuracy measures of Section 4.2 with compensated (Dot2) dot products,
 * computed on the device; blocking, result in *out (host).
 *   rxr_orth_error : ||Q^T Q - I||_F
 *   rxr_resid_error: ||A - Q R||_F / ||A||_F (R upper triangular)          */
RXR_API int rxr_orth_error(rxr_handle h, const double *Q, int64_t m, int64_t n, int64_t ldq, double *out, void *stream);
RXR_API int rxr_resid_error(rxr_handle h, const double *A, int64_t m, int64_t n, int64_t lda, const double *Q,
                    int64_t ldq, const double *R, int64_t ldr, double *out, void *stream);

/* Measured FP64 FMA throughput of this GPU in TFLOP/s (a calibration kernel
 * of independent DFMA chains over all SMs), the denominator of the FP64
 * roofline.  Blocking. */
RXR_API int rxr_fp64_peak(double *tflops, void *stream);

/* Device time in milliseconds of one stage of the most recent blocking or
 * host factorisation on this handle, measured with CUDA events on the
 * launching stream.  Stage ids: 0 sketch (with its reduction), 1
 * preconditioning substitution X = A R_s^{-1} (FP64 path: with its Gram),
 * 2 substitution of a middle CholeskyQR pass (FP64 path: with the next
 * Gram), 3 last pass's Q formation, 4 first Gram on the tensor cores, 5 later
 * Gram on the tensor cores, 6 XR factorisation of the sketch.  A stage the
 * last call did not run reads 0.  Returns -1 for an unknown stage id. */
RXR_API int rxr_last_kernel_ms(rxr_handle h, int kernel, float *ms);

/* Enable or disable the per-kernel events of rxr_last_kernel_ms (off by default). */
RXR_API int rxr_set_kernel_timing(rxr_handle h, int enable);

/* ---- Allocation-free sketch.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory, and so cannot
 * create a handle or hand one a workspace: processes whose device memory is
 * reserved in full by another allocator (a framework's caching pool that owns
 * the whole GPU), and loops that forbid allocation after start-up because
 * cudaMalloc may synchronise the device or take an unbounded time.
 *
 * Y = Omega A exactly as rxr_sketch with RXR_FP64 (same kernels, same Omega),
 * but its scratch (the per-chunk partial sums and the status word) lives in a
 * fixed array of RXR_NOALLOC_SCRATCH_BYTES inside the library, which every GPU
 * that loads the library holds until the process exits.  The number of row
 * chunks is capped so that the partial sums fit (at s = 2048, n = 128 at most
 * 7 chunks), so the result may differ from rxr_sketch's in rounding (not in
 * the tolerance).
 *   A, m, n, lda (1-4)  device, column-major, m >= n >= 1, n <= 128, lda >= m.
 *   s (5), seed (6)     sketch rows (1..RXR_MAX_S) and the Philox key.
 *   Y, ldy (7-8)        device output, s x n, ldy >= s.
 *   stream (9)          cudaStream_t; the call is blocking (it copies the
 *                       status word to the host and synchronises the stream).
 * Returns 0, -i for an invalid argument i (s above RXR_MAX_S: -5),
 * RXR_ERR_UNSUPPORTED for n > 128 or m > 2^31, RXR_ERR_NONFINITE, or
 * RXR_ERR_CUDA.  Every admissible s x n fits the array (checked when the
 * library is compiled).
 * The call allocates nothing: no cudaMalloc, cudaFree or allocating library
 * routine.  Its first call on a device (the current device) looks up the
 * array's device address and sets the kernel's shared-memory limit; make that
 * first call before any stream capture.  Every call uses the same array and
 * the array keeps the last call's contents (the status word is cleared at the
 * start of each call; the partial sums are overwritten in full), so calls
 * whose work overlaps on the GPU (other threads, other streams) race:
 * serialise them. */
#define RXR_NOALLOC_SCRATCH_BYTES (16u << 20)
RXR_API int rxr_sketch_noalloc(const double *A, int64_t m, int64_t n, int64_t lda, int64_t s, uint64_t seed,
                               double *Y, int64_t ldy, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* RXR_H */
