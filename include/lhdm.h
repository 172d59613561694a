/*
 * lhdm.h -- C ABI of the GB300 (sm_103a) FP64 solver for dense nonnegative
 * least squares by Lawson-Hanson with Deviation Maximization (LHDM).
 *
 *   minimise ||A x - b||_2  subject to  x >= 0                  (problem (1))
 *
 * Method: Algorithm 3 of "The Lawson-Hanson Algorithm with Deviation
 * Maximization: Finite Convergence and Sparse Recovery" (Dessole, Dell'Orto,
 * Marcuzzi), with Algorithm 2 (DM) choosing up to k_max columns per outer
 * step, Householder updating (Algorithm 4) of the partial QR factorisation
 * Q^T A Pi = [R B; 0 C] (section 2.1) applied to the whole matrix, and
 * Givens downdating (Algorithm 5) in the inner loop.  k_max = 1 is the
 * one-column Lawson-Hanson method (Algorithm 1).  Every step runs in CUDA
 * kernels on the device; there is no CPU fallback.
 *
 * Conventions shared by every entry point
 *  - All matrices are column-major FP64.  A is m x n with leading dimension
 *    lda >= max(1, m).  Vectors are contiguous FP64 (int32 for index lists).
 *  - "device" pointers must point to device memory the caller owns and keeps
 *    alive until the stream work of the call has completed; "host" pointers
 *    are ordinary host memory.
 *  - stream is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Every call only enqueues work on that stream, except where a
 *    host-side result is documented: those calls synchronise the stream.
 *  - Return value: LHDM_OK (0) or one of the LHDM_ERR_* codes below.  No call
 *    aborts, throws or traps; CUDA errors are reported as LHDM_ERR_CUDA.
 *  - Numerical status of a solve (iteration cap, non-finite input, ...) is
 *    reported in lhdm_info.status; the call itself still returns LHDM_OK when
 *    the work was enqueued and completed.
 *  - Not thread-safe per context: calls on one lhdm_ctx must be serialised
 *    by the caller.  Distinct contexts are independent.
 */
#ifndef LHDM_H
#define LHDM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status / error codes. */
#define LHDM_OK 0
#define LHDM_ERR_INVALID_ARG 1 /* bad size, pointer or parameter             */
#define LHDM_ERR_MAX_ITER 2    /* outer-iteration cap reached (info.status)  */
#define LHDM_ERR_NONFINITE 4   /* NaN/Inf in A or b (info.status)            */
#define LHDM_ERR_CUDA 5        /* a CUDA runtime call failed                 */
#define LHDM_ERR_TIMEOUT 6     /* a device-side wait exceeded its bound      */
#define LHDM_ERR_ALLOC 7       /* device or host allocation failed           */
#define LHDM_ERR_NO_STATE 8    /* backward called without a matching solve   */
#define LHDM_ERR_TOO_LARGE 9   /* beyond the fixed workspace of the
                                  allocation-free entry point              */

/* Largest supported block size k_max (columns chosen per outer step). */
#define LHDM_KMAX_LIMIT 64

/* Problem modes (lhdm_params.mode). */
#define LHDM_MODE_NNLS 0        /* min ||A x - b||, x >= 0 (problem (1))        */
#define LHDM_MODE_SIGNED 1      /* positivity trick, problem (positivity_trick)
                                   of section 3.2: NNLS on [A  -A] without
                                   forming -A; x = (x+, x-) has 2n entries     */
#define LHDM_MODE_SIGNED_FLIP 2 /* the same, with the sign flip of section 4.2
                                   in place of the inner loop's downdates      */

/*
 * Algorithm parameters (Algorithm 2 and Algorithm 3).
 *  tau1, tau2 in (0, 1]: candidate thresholds on the dual vector w and on
 *      the trailing column norms u (Algorithm 2, candidate set I).
 *  delta in (0, 1]: bound on the absolute cosine between chosen projected
 *      columns (Algorithm 2; Algorithm 3 names it tau_c in its signature).
 *  k_max in [1, LHDM_KMAX_LIMIT]: at most k_max columns enter per outer step;
 *      k_max = 1 is Lawson-Hanson (Algorithm 1).
 *  tol_w: the outer loop stops when max over Z of w <= tol_w (the test
 *      "max w > 0" of Algorithms 1 and 3 with a floating-point tolerance);
 *      tol_w < 0 selects 10 * 2^-52 * max(m,n) * max_j ||a_j|| * ||b||.
 *  max_outer: cap on outer iterations; <= 0 selects 3n.
 *  mode: LHDM_MODE_NNLS, LHDM_MODE_SIGNED or LHDM_MODE_SIGNED_FLIP.  In the
 *      signed modes the problem is NNLS on the m x 2n matrix [A  -A]: A is
 *      still passed as m x n, x and passive have 2n entries (x_j for column
 *      j, x_{n+j} for column -a_j), and n stands for 2n in the defaults of
 *      tol_w and max_outer.  The adjoint (lhdm_backward) is not available
 *      for the signed modes.
 *  reserved: set to 0.
 * Defaults (lhdm_default_params): tau1 = 0.6, tau2 = 0.15, delta = 0.9,
 * k_max = 32, the values of section 5; mode = LHDM_MODE_NNLS.
 */
typedef struct {
  double tau1;
  double tau2;
  double delta;
  double tol_w;
  int32_t k_max;
  int32_t max_outer;
  int32_t mode;
  int32_t reserved;
} lhdm_params;

/* Per-solve report. */
typedef struct {
  int32_t status;       /* LHDM_OK, LHDM_ERR_MAX_ITER, LHDM_ERR_NONFINITE,
                           LHDM_ERR_TIMEOUT                                  */
  int32_t n_outer;      /* outer iterations                                  */
  int32_t n_inner;      /* inner-loop iterations (step-length/removal steps) */
  int32_t n_drop;       /* columns dropped by the feasibility loop           */
  int32_t n_passive;    /* |P| at exit                                       */
  int32_t rank_limited; /* 1 if columns with w > tol_w were left out because
                           their trailing norm was <= 100 eps ||a_j||        */
  int32_t n_flip;       /* sign flips (LHDM_MODE_SIGNED_FLIP)                */
  int32_t mode;         /* the mode solved                                   */
  double resid_norm;    /* ||b - A x||                                       */
  double max_wZ;        /* max over Z of w = A^T (b - A x) at exit           */
  double tol_w;         /* tolerance actually used                           */
} lhdm_info;

typedef struct lhdm_ctx lhdm_ctx;
typedef struct lhdm_batch lhdm_batch;

/* Fills *p with the defaults listed above.  p: host. */
int lhdm_default_params(lhdm_params* p);

/* Short English description of a status code (static storage). */
const char* lhdm_status_string(int status);

/*
 * Creates a solve context on the current CUDA device for single problems up
 * to max_m x max_n (lhdm_solve) and for batches of up to max_batch problems,
 * each at most max_m x max_n (lhdm_solve_batched; max_batch = 0: no batched
 * solves).  Allocates the single-solve workspace here (FP64, about
 * 8 * (max_m * max_n + min(max_m,max_n)^2) bytes plus O(max_m + max_n));
 * later single solves allocate nothing.  The batch workspace is sized by the
 * first lhdm_solve_batched call with a given set of instances (see there).
 * *ctx receives the handle (host).
 * Errors: INVALID_ARG (sizes < 1, max_batch < 0 or ctx NULL), ALLOC, CUDA.
 */
int lhdm_create(lhdm_ctx** ctx, int32_t max_m, int32_t max_n, int32_t max_batch);

/* Releases the context and its device memory (synchronises the device). */
int lhdm_destroy(lhdm_ctx* ctx);

/*
 * lhdm_solve: one NNLS problem, all steps on the device in one persistent
 * cooperative launch over every SM (Algorithm 3; Algorithm 1 if k_max = 1).
 *  m, n        problem size, 0 <= m <= max_m, 0 <= n <= max_n of the context.
 *  A           device, m x n, column-major, leading dimension lda.
 *  b           device, length m.
 *  prm         host; NULL selects the defaults.
 *  x           device, length n (2n in the signed modes): the solution
 *              (x_Z = 0).
 *  passive     device, length n (2n in the signed modes): the passive set P
 *              sorted ascending, then -1.
 *  info        host or NULL.  When non-NULL the call synchronises the stream
 *              and fills it; when NULL the call is asynchronous and
 *              lhdm_get_info() retrieves the report later.
 * The context keeps R, the ordered P, x_P and the residual for
 * lhdm_backward until the next solve on the same context.
 * Errors: INVALID_ARG (sizes, lda < max(1,m), NULL pointers, parameters out
 * of range), CUDA.  A, b are not modified.
 */
int lhdm_solve(lhdm_ctx* ctx, int32_t m, int32_t n, const double* A, int32_t lda,
               const double* b, const lhdm_params* prm, double* x, int32_t* passive,
               lhdm_info* info, void* stream);

/*
 * lhdm_solve_host: the same solve with HOST buffers (the end-to-end path):
 * copies A (m x n, lda) and b to the device on the stream, solves, copies x
 * and passive back and synchronises.  A, b, x, passive, info: host.  Pinned
 * host memory gives asynchronous copies; pageable memory works too.
 * Errors as lhdm_solve.
 */
int lhdm_solve_host(lhdm_ctx* ctx, int32_t m, int32_t n, const double* A, int32_t lda,
                    const double* b, const lhdm_params* prm, double* x, int32_t* passive,
                    lhdm_info* info, void* stream);

/*
 * lhdm_solve_noalloc: the single solve of lhdm_solve for callers that must
 * not allocate device memory -- code running where cudaMalloc is not
 * allowed or not wanted (a real-time or embedded loop with a fixed memory
 * budget, a plug-in inside a host framework that owns the device heap, a
 * recovery path entered after an allocation failed).  It takes no context:
 * all workspace is one statically sized device array compiled into the
 * library, so this call allocates nothing (no cudaMalloc, no cudaFree, no
 * allocating library routine).
 *
 * The paper has no counterpart: it is a deployment variant of the same
 * kernel, with the same arithmetic and results as lhdm_solve.
 *
 * Limits: m <= 256 and n <= 512 (larger sizes return LHDM_ERR_TOO_LARGE
 * without launching anything), on a GPU with at most 160 SMs.  The array
 * (5 MiB) occupies device memory on every GPU that loads the library until
 * the process exits.
 *
 * Arguments as lhdm_solve, except:
 *  info   DEVICE pointer to one lhdm_info the call writes (required).
 * The call is asynchronous on `stream`.  The first call on each device
 * looks up the array's device address and sets kernel attributes, so make
 * that first call before capturing a stream.  Every call shares the one
 * array and overwrites it (the kernel re-initialises all the state it
 * reads; the barrier words are cleared with cudaMemsetAsync): calls whose
 * work overlaps on the GPU -- concurrent streams, or several host threads
 * -- race and corrupt each other, so serialise them (one stream is enough).
 * No adjoint state is kept for lhdm_backward.
 * Errors: INVALID_ARG, TOO_LARGE, CUDA.
 */
int lhdm_solve_noalloc(int32_t m, int32_t n, const double* A, int32_t lda, const double* b,
                       const lhdm_params* prm, double* x, int32_t* passive, lhdm_info* info,
                       void* stream);

/* Copies the report of the last solve on ctx to *info (host); synchronises. */
int lhdm_get_info(lhdm_ctx* ctx, lhdm_info* info, void* stream);

/*
 * lhdm_backward: adjoint of the solution map on the final passive set P of
 * a solve on ctx (x_P is the least-squares solution on P, subproblem (6) of
 * section 2.1; P is locally constant where the solution is strictly
 * complementary).  With g = dL/dx it solves R^T R u = g_P with the final R
 * factor and writes
 *     dL/db   = A_P u                          (length m)
 *     dL/dA_P = r u^T - (A_P u) x_P^T,  dL/dA_Z = 0   (m x n, ld ld_dA)
 * where r = b - A x.
 *  idx   < 0: the last lhdm_solve on ctx (one cooperative launch over every
 *        SM, asynchronous on stream);
 *        >= 0: instance idx of the last lhdm_solve_batched on ctx (one CTA;
 *        the call synchronises the stream).
 *  A     device; the matrix passed to that solve (lda as then).
 *  dLdx  device, length n.  dLdb (length m), dLdA (m x n, ld_dA >= m):
 *        device; either may be NULL.
 * Errors: NO_STATE (no completed solve of that kind), INVALID_ARG (idx out
 * of range, pointers, ld_dA), CUDA.
 */
int lhdm_backward(lhdm_ctx* ctx, int32_t idx, const double* A, int32_t lda, const double* dLdx,
                  double* dLdb, double* dLdA, int32_t ld_dA, void* stream);

/*
 * lhdm_solve_batched: `batch` independent problems of uneven sizes (paper
 * problem (1) per instance, Algorithm 3 on each) in ONE persistent launch;
 * each CTA takes instances from a device work queue, largest first.
 *  batch          0 <= batch <= max_batch of the context.
 *  m, n, lda      host arrays [batch]; m[i] <= max_m, n[i] <= max_n.
 *  A, b, x, passive  host arrays [batch] of DEVICE pointers, shapes as in
 *                 lhdm_solve (A[i] column-major m[i] x n[i], ld lda[i]).
 *  prm            host, NULL = defaults; prm->k_max <= 0 takes k_max per
 *                 instance from the autotuner's table (lhdm_batch_autotune).
 *  info           DEVICE array of batch lhdm_info, one per instance.
 * The first call with a given argument set (sizes, pointers, parameters)
 * plans the batch: it allocates the batch workspace, uploads the instance
 * table and synchronises the stream, so it cannot be captured in a CUDA
 * graph.  Every later call with the same arguments reuses that plan and only
 * enqueues one small reset and one kernel launch (no allocation, no host
 * synchronisation): that call can be captured.  Different arguments replace
 * the plan.  The per-instance state for lhdm_backward(idx >= 0) and
 * lhdm_backward_batched lives in the plan until the next replacement.
 * Errors: INVALID_ARG, ALLOC, CUDA.
 */
int lhdm_solve_batched(lhdm_ctx* ctx, int32_t batch, const int32_t* m, const int32_t* n,
                       const double* const* A, const int32_t* lda, const double* const* b,
                       const lhdm_params* prm, double* const* x, int32_t* const* passive,
                       lhdm_info* info, void* stream);

/*
 * Adjoint of every instance of the last lhdm_solve_batched on ctx, one
 * launch (formulas of lhdm_backward): host arrays [batch] of device pointers
 * dLdx, dLdb, dLdA (entries may be NULL; a NULL dLdx[i] skips instance i)
 * and host ld_dA[batch] (NULL: ld = m[i]).  Synchronises the stream.
 * Errors: NO_STATE, INVALID_ARG, CUDA.
 */
int lhdm_backward_batched(lhdm_ctx* ctx, const double* const* dLdx, double* const* dLdb,
                          double* const* dLdA, const int32_t* ld_dA, void* stream);

/*
 * lhdm_solve_l1: l1-NNLS (section 3.3, eq. (l1_NNLS)), the squared-l1
 * regularised least squares  min ||x||_1^2 + lambda^2 ||A x - b||^2  recast
 * as NNLS on the (m+1) x 2n system
 *     [1^T  1^T; lambda A  -lambda A] (x+; x-) = (0; lambda b),  x+, x- >= 0.
 * The stacked system is written into a buffer of the context by one kernel
 * (one read of A, two column writes) and solved by lhdm_solve.
 *  m, n, A, lda, b  the data of the regularised problem (A device, m x n,
 *                 column-major; b device, length m); the context must allow
 *                 m + 1 rows and 2n columns (max_m >= m+1, max_n >= 2n).
 *  lambda         > 0, the weight of the residual.
 *  prm            host, NULL = defaults; prm->mode must be LHDM_MODE_NNLS.
 *  x, passive     device, 2n entries: (x+, x-) and the passive set of the
 *                 stacked system (indices j < n for x+_j, n + j for x-_j).
 *  info           host or NULL, as lhdm_solve.
 * The first call on a context allocates the stacked buffers (about
 * 8 * max_m * max_n bytes); later calls allocate nothing.  No adjoint state
 * is kept.  Errors: INVALID_ARG, ALLOC, CUDA.
 */
int lhdm_solve_l1(lhdm_ctx* ctx, int32_t m, int32_t n, const double* A, int32_t lda, const double* b,
                  double lambda, const lhdm_params* prm, double* x, int32_t* passive, lhdm_info* info,
                  void* stream);

/*
 * Bound, in nanoseconds, on every wait of one CTA for another in the solves
 * and adjoints launched on ctx after this call (the grid barrier, the flags
 * of the pipelined triangular solve and of the rotation log); ns <= 0
 * restores the default of 4 s.  When a wait runs out the waiting CTA sets an
 * error flag, every CTA leaves the kernel without further waits, and the
 * solve reports status LHDM_ERR_TIMEOUT; the context stays usable (the next
 * call clears the barrier words).  Host only.  Errors: INVALID_ARG.
 */
int lhdm_set_wait_limit(lhdm_ctx* ctx, int64_t ns);

/*
 * Test aid for the accuracy guard of the tensor-core commit (the FP64
 * products of the block reflector update formed from exact 7-bit digit
 * products on bf16 tensor cores, with a fallback to FP64 where the digits
 * could be less accurate than an FP64 evaluation): mode 1 sends every batch
 * of the later solves on ctx to the FP64 path as the guard would, mode 0
 * restores the guard's own decisions.  Results must not change beyond
 * rounding; the count of batches sent is word [10] of the "ctl" state of
 * lhdm_debug_state.  Errors: INVALID_ARG.
 */
int lhdm_debug_commit_guard(lhdm_ctx* ctx, int32_t mode);

/*
 * Failure-detection test aid: the next lhdm_solve on ctx runs with a grid
 * barrier that expects one arrival more than the grid has, so no CTA ever
 * releases it, every CTA's bounded wait runs out (lhdm_set_wait_limit) and
 * the solve reports LHDM_ERR_TIMEOUT.  Nothing faults or hangs: the kernel
 * returns after the wait limit.  Later solves are unaffected.
 * Errors: INVALID_ARG.
 */
int lhdm_debug_stall_next_solve(lhdm_ctx* ctx);

/*
 * Verification aid for the reciprocal and square root the solver's scalar
 * chains use in place of the compiler's correctly rounded ones (Newton-
 * Raphson from a single-precision seed; Goldschmidt with a Newton
 * correction).  For each of the n device doubles x[i], out (device, 4 n
 * doubles) receives out[4i] = the solver's 1/x, out[4i+1] = 1.0/x,
 * out[4i+2] = the solver's sqrt(|x|), out[4i+3] = sqrt(|x|), computed on the
 * device on `stream`; the call does not synchronise.
 * Errors: INVALID_ARG (n < 0, or a null pointer with n > 0), CUDA.
 */
int lhdm_debug_fast_math(const double* x, double* out, int32_t n, void* stream);

/* Decision trace of the last solve (verification aid): up to max_rows rows
 * of 6 int32 per outer step, host buffer out[6 * max_rows]:
 *   |J| from Algorithm 2, |J| kept after the feasibility loop, inner-loop
 *   steps, |P| after the step, columns removed by the inner loop, and the
 *   first column of J (the Lawson-Hanson argmax).
 * Returns the number of rows written (negative status on error);
 * synchronises the stream. */
int lhdm_trace(lhdm_ctx* ctx, int32_t* out, int32_t max_rows, void* stream);

/* Verification aid: copies `count` elements of a named piece of the
 * context's device state after the last solve to host memory `host`
 * (synchronises).  Names: "w", "u", "anorm" (length n), "bt", "r"
 * (length m), "yP", "xP", "order", "rslot" (positions), "pos" (columns),
 * "W" (ld = max_m rounded up to even), "R" (slot-major, ld = the context's
 * min(max_m, max_n) rounded up to even), "ctl" (16 int32 control words;
 * [10] = commit batches that the accuracy guard of the tensor-core commit
 * sent to FP64).  FP64 except the int32 arrays.  Errors: INVALID_ARG for an unknown name or count too large. */
int lhdm_debug_state(lhdm_ctx* ctx, const char* name, void* host, int64_t count, void* stream);

/* Profile of the last solve on ctx.  ms[0..12) = device time in ms of each
 * solver phase: setup, DM, panel, triangular solve (outer step), commit,
 * inner-loop control and bookkeeping, residual, dual vector, feasibility
 * loop, Givens chain on R, rotations of the Z columns, triangular solves of
 * the inner loop; ms[12..24) = the algorithmic FP64 flops of the same
 * phases (an FMA counts 2); ms[24] = bf16 tensor-core MMA instructions
 * (m16n8k16, 4096 flops each) the commit issued.  Writes min(n, 25) values
 * and returns how many (negative status on error).  Synchronises the
 * stream. */
int lhdm_phase_times(lhdm_ctx* ctx, double* ms, int32_t n, void* stream);

/*
 * Batched solves: many independent problems of uneven sizes in ONE
 * persistent launch (each CTA takes instances from a device work queue,
 * largest first, and runs Algorithm 3 on its own).
 *
 * lhdm_batch_create plans a batch: host arrays m[batch], n[batch],
 * lda[batch] and host arrays of DEVICE pointers A[batch], b[batch],
 * x[batch], passive[batch] (shapes as in lhdm_solve); info: device array of
 * batch lhdm_info.  prm: host, NULL = defaults; prm->k_max <= 0 takes
 * k_max per instance from the autotuner's table (lhdm_batch_autotune), or
 * from a built-in rule for sizes it has not tuned.  Allocates all device
 * workspace and uploads the descriptor table on the stream (synchronises).
 * Errors: INVALID_ARG, ALLOC, CUDA.
 */
int lhdm_batch_create(lhdm_batch** plan, int32_t batch, const int32_t* m, const int32_t* n,
                      const int32_t* lda, const double* const* A, const double* const* b,
                      double* const* x, int32_t* const* passive, lhdm_info* info,
                      const lhdm_params* prm, void* stream);

/* Runs the planned batch: exactly one kernel launch plus one small reset,
 * no allocation and no host synchronisation, so it can be captured in a
 * CUDA graph.  Results land in the x / passive / info arrays of the plan. */
int lhdm_batch_run(lhdm_batch* plan, void* stream);

/*
 * Adjoint of every instance of the last lhdm_batch_run, one launch:
 * host arrays of device pointers dLdx[batch], dLdb[batch], dLdA[batch]
 * (entries may be NULL) and host ld_dA[batch].  Same formulas as
 * lhdm_backward.  Errors: NO_STATE, INVALID_ARG, CUDA.
 */
int lhdm_batch_backward(lhdm_batch* plan, const double* const* dLdx, double* const* dLdb,
                        double* const* dLdA, const int32_t* ld_dA, void* stream);

/* k_max the tuner chose for instance i (host int); -1 if out of range. */
int lhdm_batch_kmax(const lhdm_batch* plan, int32_t i);

/* Releases a plan (synchronises the device). */
int lhdm_batch_destroy(lhdm_batch* plan);

/*
 * Autotuner of the batched solve (the paper fixes k_max by hand; choosing it
 * per instance size is this library's addition).  Instances are bucketed by
 * column count n: bucket b holds 128 * 2^(b-1) < n <= 128 * 2^b (bucket 0:
 * n <= 128; the last bucket is open).  For every bucket present in the
 * given instances (same argument conventions as lhdm_batch_create, without
 * outputs), one batch of that bucket's instances is planned, run once to
 * warm up and timed once with CUDA events for each k_max in {4, 8, 16, 32};
 * the fastest k_max is stored in a process-wide table that
 * lhdm_batch_create consults when prm->k_max <= 0 (buckets never tuned use
 * the built-in rule).  prm: other parameters of the trial solves (NULL =
 * defaults; its k_max is ignored).  table: host array of
 * LHDM_TUNE_BUCKETS ints receiving the table (0 = untuned), or NULL.
 * Allocates and frees temporary device buffers and synchronises the stream;
 * not for use inside graph capture.
 * Errors: INVALID_ARG, ALLOC, CUDA.
 */
#define LHDM_TUNE_BUCKETS 6
int lhdm_batch_autotune(int32_t batch, const int32_t* m, const int32_t* n, const int32_t* lda,
                        const double* const* A, const double* const* b, const lhdm_params* prm,
                        int32_t* table, void* stream);

/* Reads (table != NULL) the tuner's table of LHDM_TUNE_BUCKETS k_max values
 * (0 = untuned).  Host memory.  Errors: INVALID_ARG. */
int lhdm_tuning_get(int32_t* table);

/* Replaces the tuner's table (host, LHDM_TUNE_BUCKETS entries, each 0 or
 * 1..LHDM_KMAX_LIMIT), e.g. to restore a table saved from an earlier run.
 * Errors: INVALID_ARG. */
int lhdm_tuning_set(const int32_t* table);

#ifdef __cplusplus
}
#endif

#endif /* LHDM_H */
