/*
 * rorbk.h -- C ABI of the GB300 ROR-BK solver.
 *
 * ROR-BK (Regularized Orthogonality and Residual based Block-Kaczmarz) solves a
 * consistent linear system A x = b, A in R^{m x n}, square, over- or
 * under-determined (Kar & Venkatapathi, arXiv 2510.02156, Section 1 Eq. (1)
 * and Section 2).  Algorithm 1 of the paper is the method:
 *
 *   setup   (Algorithm 1's set-up; Section 2; Section 3.1)
 *     - split the rows into k contiguous blocks of >= floor(m/k) rows;
 *     - centroids Abar_t = sum of block t's rows;
 *       C(i,j) = |<Abar_i,Abar_j>| / (|Abar_i| |Abar_j|);
 *     - Pbar_t = exp(-2 sum_j C(t,j) / n),  P = Pbar / sum(Pbar);
 *     - for each block, W_t = (A_t A_t^T + mu I)^{-1}, formed once and stored
 *       (Section 3.1), here through a Cholesky factor L_t: W_t = L_t^-T L_t^-1;
 *       a block with at least n rows stores V_t = (A_t^T A_t + mu I)^{-1}
 *       instead (Lemma 1, Section 3.1).
 *   iteration j (Algorithm 1, the loop body)
 *     - 3 times: draw tau ~ P; x += A_tau^T W_tau (b_tau - A_tau x)
 *       (or x += V_tau A_tau^T (b_tau - A_tau x));
 *     - r = b - A x; stop if ||r|| / ||b|| <= tol;
 *     - I = the floor(m/k) rows with the largest r_i^2;
 *       x += A_I^T (A_I A_I^T + mu I)^{-1} r_I   (Gram + Cholesky per call;
 *       the n x n form when K >= n).
 *
 * Beside the method: a mixed-precision form (FP64 refinement around FP32
 * ROR-BK), an incremental residual, residual-weighted draws, Algorithm 2's
 * initial solution, Algorithm 3 (FAB-GMRES with ROR-BK inner solves), batched
 * solves, the adjoint solve of a differentiable solve, single steps for
 * testing, and a residual entry point that allocates no memory.
 *
 * All arithmetic runs in CUDA kernels compiled for sm_103a; nothing falls back
 * to the CPU.  Every call returns an rorbk_status; on failure
 * rorbk_last_error(h) holds a message.  A handle is not thread-safe: use one
 * host thread per handle.
 *
 * Readings of points the paper leaves open (block remainder placement, the
 * random stream, tie-breaking, zero centroids, zero right-hand side) are
 * listed beside each entry point below.
 */
#ifndef RORBK_H
#define RORBK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rorbk_ctx *rorbk_handle;

typedef enum {
    RORBK_OK = 0,                 /* converged (solve) or success            */
    RORBK_NOT_CONVERGED = 1,      /* non-fatal: maxit reached; x holds the last iterate */
    RORBK_ERR_INVALID_ARG = -1,   /* bad pointer, size, partition or CSR structure */
    RORBK_ERR_CUDA = -2,          /* a CUDA runtime call failed               */
    RORBK_ERR_OOM = -3,           /* device allocation failed                 */
    RORBK_ERR_NOT_SPD = -4,       /* a block Gram lost positive definiteness (only reachable with lambda = 0) */
    RORBK_ERR_NUMERIC = -5,       /* NaN/Inf in A, b or the residual          */
    RORBK_ERR_BOUNDS = -6,        /* an index escaped its range on the device */
    RORBK_ERR_UNSUPPORTED = -7,   /* a mode the library does not provide      */
    RORBK_ERR_DEVICE_TIMEOUT = -8 /* a bounded device-side wait gave up; the
                                     kernel returned instead of hanging      */
} rorbk_status;

enum { RORBK_FORMAT_CSR = 0, RORBK_FORMAT_DENSE = 1 };
enum { RORBK_F64 = 0, RORBK_F32 = 1 };

/* Arithmetic of the iteration.
 *   FP64  : the plain method, every step in FP64 (values stored as FP32 are
 *           widened exactly).
 *   MIXED : FP64 iterative refinement around FP32 ROR-BK: r = b - A x in
 *           FP64, an FP32 ROR-BK solve of A d = r to a relative residual of
 *           inner_tol (or inner_maxit iterations), x += d in FP64, repeated
 *           until ||b - A x|| / ||b|| <= tol.  The block operators W_t and the
 *           dynamic block's Cholesky are formed in FP64 and applied in FP32.
 *           Blocks with at least as many rows as A has columns (s >= n)
 *           use the n x n form of Lemma 1 (Section 3.1) in both
 *           arithmetics: V_t = (A_t^T A_t + mu I)^{-1} and, when K >= n, the
 *           dynamic block's (A_I^T A_I + mu I)^{-1} A_I^T r_I.  The s x s
 *           form would carry 1/mu on the null space of A_t A_t^T, which FP32
 *           rounding cannot hold. */
enum { RORBK_PREC_FP64 = 0, RORBK_PREC_MIXED = 1 };

/* Matrix description for rorbk_setup.
 *   CSR  : row_ptr[m+1] (int32, row_ptr[0] = 0, non-decreasing, nnz < 2^31),
 *          col_idx[nnz] (int32, strictly ascending inside each row, in [0,n)),
 *          values[nnz] (dtype).
 *   DENSE: values is row-major m x n with leading dimension ld >= n
 *          (row_ptr, col_idx and nnz are ignored; m * n < 2^31).  The handle
 *          keeps it as CSR with all m * n entries stored, so every step runs
 *          the same arithmetic as for a sparse A, except the dynamic block:
 *          all of its rows share all columns, and its Gram, Cholesky and
 *          A_I^T y run as dense kernels.
 * Pointers are host memory unless on_device != 0 (then CUDA device memory of
 * the current device).  rorbk_setup copies A into memory the handle owns; the
 * caller may free its arrays when setup returns. */
typedef struct {
    int32_t format;
    int32_t dtype;
    int64_t m, n, nnz;
    const int32_t *row_ptr;
    const int32_t *col_idx;
    const void *values;
    int64_t ld;
    int32_t on_device;
    int32_t reserved_;
} rorbk_matrix;

/* Row partition.  num_blocks = k >= 1.  offsets == NULL selects the uniform
 * contiguous split of Algorithm 1's partition: block t holds rows
 * [t*floor(m/k) + min(t, m mod k), (t+1)*floor(m/k) + min(t+1, m mod k)),
 * so the first (m mod k) blocks carry one extra row (the paper only asks for
 * at least floor(m/k) rows per block).  A caller-supplied offsets[k+1]
 * (host, strictly increasing, 0 .. m) gives any other contiguous split.
 * Blocks may hold at most 1024 rows. */
typedef struct {
    int32_t num_blocks;
    int32_t reserved_;
    const int64_t *offsets;
} rorbk_partition;

/* Optional per-iteration record (device pointers; each may be NULL).
 *   tau [capacity * n_static] int64 : sampled blocks
 *   rrn [capacity]            double: ||b - A x|| / ||b|| after the statics
 *   I   [capacity * K]        int32 : dynamic index set, ascending (K = floor(m/k))
 *   x   [capacity * n]        double: x at the end of the iteration (after the
 *                                     dynamic update; on the converging
 *                                     iteration, after the static updates)
 *   dyn [capacity * 4]        int32 : dynamic block structure per iteration:
 *                                     nonzeros of A_I, nonzeros in columns
 *                                     shared inside I, coupled rows |S|,
 *                                     Gram contributions
 * Iterations beyond capacity are not recorded.  FP64 mode only. */
typedef struct {
    int64_t capacity;
    int64_t *tau;
    double *rrn;
    int32_t *I;
    double *x;
    int32_t *dyn;
} rorbk_trace;

/* Options (NULL = defaults). */
typedef struct {
    uint64_t seed;          /* Philox key word 0                       (0)    */
    uint64_t system_id;     /* Philox key word 1                       (0)    */
    int32_t n_static;       /* sampled updates per iteration, l       (3)    */
    int32_t precision;      /* RORBK_PREC_*                            (FP64) */
    int64_t start_iter;     /* counter of the first iteration (resume) (0)    */
    double inner_tol;       /* MIXED: inner relative residual target   (1e-4) */
    int64_t inner_maxit;    /* MIXED: inner iteration cap per refinement (2000000) */
    int32_t host_loop;      /* 0: the whole loop runs on the device inside one
                               CUDA graph (a conditional WHILE node);
                               1: the host enqueues batches of `poll`
                               iterations and reads the stop flag between
                               batches (profilers that cannot see kernels in
                               conditional graphs)             (0)    */
    int32_t poll;           /* iterations per batch when host_loop = 1 (64)   */
    rorbk_trace *trace;     /* FP64 only                               (NULL) */
    void *stream;           /* cudaStream_t for all work               (0 = legacy default) */
    int32_t dist_mode;      /* RORBK_DIST_*: how the static blocks are drawn (PAPER) */
    int32_t residual_mode;  /* RORBK_RESIDUAL_*: how r = b - A x is formed   (EXACT) */
    int32_t refresh;        /* INCREMENTAL: an exact residual every `refresh`
                               iterations (0: 50)                          (0)    */
    int32_t fault_inject;   /* RORBK_FAULT_*: host-chosen failure injection for
                               tests of the failure paths              (NONE) */
} rorbk_options;

/* Failure injection (rorbk_options.fault_inject); nothing faults, traps or
 * hangs the GPU.
 *   NONE       : normal operation.
 *   WAIT_LIMIT : the first bounded wait of each sampled update whose block was
 *                staged by asynchronous copies waits, with a limit of one
 *                poll, on a barrier that nothing completes, so the wait gives
 *                up the way a copy that never lands would make it: the kernel
 *                records RORBK_ERR_DEVICE_TIMEOUT, waits (bounded) for the
 *                copies it did issue, and returns; the solve ends with that
 *                status and the handle stays usable. */
enum { RORBK_FAULT_NONE = 0, RORBK_FAULT_WAIT_LIMIT = 1 };

/* How the full residual of each iteration is formed (rorbk_options.residual_mode).
 *   EXACT       : r = b - A x over all of A (Algorithm 1).
 *   INCREMENTAL : a cheaper evaluation of the same residual, which Section
 *                 3.1's cost discussion leaves open (there the O(mn) residual
 *                 dominates an iteration): every x += dx of
 *                 the iteration is logged as (column, increment) pairs and
 *                 r -= A dx is applied through a CSC copy of A (built at the
 *                 first such solve, 16 bytes per nonzero) with atomic adds, so
 *                 r carries rounding drift and the order of the adds varies
 *                 from run to run.  An exact residual is formed in the first
 *                 iteration, every `refresh` iterations, when the log
 *                 overflows, and whenever the incremental residual reaches the
 *                 tolerance: the solve stops only on an exact residual.
 *                 Sparse (CSR) systems, FP64 or MIXED; not with
 *                 residual-weighted draws; single solves (not batched);
 *                 RORBK_ERR_UNSUPPORTED otherwise.  `refresh` < 0 is
 *                 RORBK_ERR_INVALID_ARG. */
enum { RORBK_RESIDUAL_EXACT = 0, RORBK_RESIDUAL_INCREMENTAL = 1 };

/* Distribution of the static blocks (rorbk_options.dist_mode).
 *   PAPER             : tau ~ P, P_t proportional to Pbar_t (Algorithm 1's proposal;
 *                       static over the solve).
 *   RESIDUAL_WEIGHTED : not in the paper.  Iteration j draws block t with
 *                       weight Pbar_t * rho_t, rho_t = sum of r_i^2 over the
 *                       block's rows (one fused chain, rows ascending) of the
 *                       residual r of iteration j-1 (r = b - A x0 for j = 0).
 *                       The running sum of the weights is formed in chunks of
 *                       64 blocks (each chunk from zero, the chunk totals in
 *                       order, each entry offset by the totals before its
 *                       chunk); if every weight is zero the draws use P.
 *                       FP64 precision, single solves (not batched). */
enum { RORBK_DIST_PAPER = 0, RORBK_DIST_RESIDUAL_WEIGHTED = 1 };

typedef struct {
    int64_t iters;          /* ROR-BK iterations executed (MIXED: inner iterations summed) */
    double rrn;             /* the last ||b - A x|| / ||b|| Algorithm 1 tested:
                               after the static updates of the last iteration.
                               Converged: the returned x's.  After maxit the
                               returned x also holds that iteration's dynamic
                               update, which the paper never re-tests (FP64) */
    int32_t converged;      /* 1 if rrn <= tol                                   */
    int32_t status;         /* same as the call's return value                   */
    int64_t refinements;    /* MIXED: outer refinement steps                     */
    double time_ms;         /* device time of the iteration loop (CUDA events)   */
} rorbk_result;

typedef struct {
    int64_t m, n, nnz;
    int32_t num_blocks;     /* k                                                 */
    int32_t dyn_rows;       /* K = floor(m/k), rows of the dynamic block         */
    int32_t max_block_rows; /* largest static block                              */
    int32_t format;
    double lambda;          /* mu                                                */
    int64_t device_bytes;   /* device memory the handle owns                     */
} rorbk_info;

/* Fills *opt with the defaults listed above. */
void rorbk_default_options(rorbk_options *opt);

/* Setup (Algorithm 1's set-up and Section 3.1): validates and copies A,
 * builds the partition, the centroids, C's row sums, P and its running sum
 * (cdf, summed sequentially in FP64), and the static operators W_t.
 *   lambda : mu, added to the diagonal of every block Gram; lambda < 0 selects
 *            the paper's default mu = 1e-6 * floor(m/k) (Section 2, after
 *            Theorem 1; Section 3.1).  lambda = 0 is allowed and may fail with
 *            RORBK_ERR_NOT_SPD on rank-deficient blocks.
 *   opt    : only opt->precision (which operator copies to keep) and
 *            opt->stream are read; NULL = defaults.
 *   *out   : the new handle, or NULL on failure.
 * Zero centroids: C(t,t) = 1 and C(t,j) = 0 (j != t) when either centroid is 0. */
rorbk_status rorbk_setup(const rorbk_matrix *A, const rorbk_partition *part,
                         double lambda, const rorbk_options *opt,
                         rorbk_handle *out);

/* rorbk_update_values: new values for h's A, same pattern (row_ptr, col_idx,
 * partition and lambda as set up).  Everything of the set-up that depends on
 * the values (the SELL copy, row norms, block transposes, centroids, C, P
 * and its running sum, the static operators W_t, their FP32 copies, and the
 * column-major copy of the incremental residual if it was built) is formed
 * again on the device by the set-up's own kernels, so the handle equals a
 * fresh rorbk_setup with these values bit for bit.  No host copy of A is made
 * and nothing new is allocated beyond per-call scratch.
 *   values    : nnz entries in the order A was given in (CSR order; a dense A:
 *               m x n row-major with leading dimension n), of the handle's
 *               value type dtype (RORBK_F64 or RORBK_F32).
 *   on_device : 1 if values is device memory, 0 for host memory.
 * Handles that share h's set-up (rorbk_clone, rorbk_multi_create) see the new
 * values too (a clone's own incremental-residual copy is formed again at its
 * next incremental solve); no solve of any of them may be in flight.  A batch or graph
 * built earlier stays valid (no buffer moves).  Errors: RORBK_ERR_INVALID_ARG
 * (NULL values, dtype other than the handle's); RORBK_ERR_NUMERIC (a NaN or Inf
 * among the values: the handle is left unchanged); RORBK_ERR_UNSUPPORTED for a
 * handle made by rorbk_setup_adjoint (set up a new one); RORBK_ERR_NOT_SPD
 * (lambda = 0 and dependent rows: the handle must then be given valid values
 * again or freed). */
rorbk_status rorbk_update_values(rorbk_handle h, const void *values, int32_t dtype, int32_t on_device);

/* Solve (Algorithm 1's iteration) from x0 until ||b - A x|| / ||b|| <= tol or
 * maxit iterations.
 *   b  : device, m doubles.   x0 : device, n doubles, or NULL for x0 = 0.
 *   x  : device, n doubles (may alias x0); receives the last iterate.
 *   The random stream: iteration j's l-th draw uses Philox4x64-10 with key
 *   (seed, system_id) and counter (start_iter + j, l, 0, 0); u = (word0 >> 11)
 *   * 2^-53 and tau = min{t : u * cdf[k-1] < cdf[t]}.
 *   Convergence is tested after the static updates, before the dynamic one;
 *   ||b|| = 0 returns x = 0 with iters = 0.  Top-K ties go to the lower row.
 * Returns RORBK_OK, RORBK_NOT_CONVERGED or an error.  res may be NULL.  The
 * call returns after the device work finished (it synchronises the stream). */
rorbk_status rorbk_solve(rorbk_handle h, const double *b, const double *x0,
                         double *x, double tol, int64_t maxit,
                         const rorbk_options *opt, rorbk_result *res);

/* rorbk_solve with host buffers: b_host (m), x0_host (n or NULL), x_host (n).
 * The host<->device copies are part of the call. */
rorbk_status rorbk_solve_host(rorbk_handle h, const double *b_host,
                              const double *x0_host, double *x_host, double tol,
                              int64_t maxit, const rorbk_options *opt,
                              rorbk_result *res);

void rorbk_free(rorbk_handle h);                    /* NULL-safe */
const char *rorbk_last_error(rorbk_handle h);       /* never NULL */
rorbk_status rorbk_get_info(rorbk_handle h, rorbk_info *info);

/* ---- single steps of the iteration (parity tests, tracing, custom loops) --
 * All pointers are device memory of the handle's device; each call finishes
 * its device work before returning. */

/* Setup products to host: cdf[k] (running sum of Pbar) and C's row sums[k];
 * either may be NULL. */
rorbk_status rorbk_get_proposal(rorbk_handle h, double *cdf_host,
                                double *c_rowsum_host);

/* Static operator W_t = (A_t A_t^T + mu I)^{-1} of block t as a dense s_t x s_t
 * row-major host array (s_t = rows of block t).  A block with s_t >= n stores
 * V_t = (A_t^T A_t + mu I)^{-1} instead (Lemma 1 and Section 3.1: the update
 * is then x += V_t A_t^T (b_t - A_t x)); for such a block the call writes V_t
 * as an n x n row-major array. */
rorbk_status rorbk_get_static_operator(rorbk_handle h, int64_t t, double *W_host);

/* The device sampler: tau for (iteration counter it, draw l). */
rorbk_status rorbk_sample(rorbk_handle h, uint64_t seed, uint64_t system_id,
                          int64_t it, int64_t l, int64_t *tau_host);

/* One static update with block tau: x += A_tau^T W_tau (b_tau - A_tau x), or
 * x += V_tau A_tau^T (b_tau - A_tau x) for a block with s_tau >= n. */
rorbk_status rorbk_static_update(rorbk_handle h, int64_t tau, const double *b,
                                 double *x);

/* r = b - A x (device r, m doubles) and ||r||^2 to *rr_host.  With
 * rr_host == NULL the call only enqueues the kernel on the handle's stream and
 * returns without waiting (for back-to-back timing). */
rorbk_status rorbk_residual(rorbk_handle h, const double *b, const double *x,
                            double *r, double *rr_host);

/* The FP32 form of the residual used by the mixed-precision inner solve:
 * r = b - A x with b, x, r FP32 device vectors and A's FP32 values (handle set
 * up with precision = RORBK_PREC_MIXED, else RORBK_ERR_UNSUPPORTED); each row
 * is an FP32 fused multiply-add chain in stored order.  rr_host as for
 * rorbk_residual (NULL: enqueue only). */
rorbk_status rorbk_residual32(rorbk_handle h, const float *b, const float *x, float *r,
                              double *rr_host);

/* I[K] (device int32): the K = floor(m/k) rows with the largest |r_i|, ties to
 * the lower index, ascending. */
rorbk_status rorbk_topk(rorbk_handle h, const double *r, int32_t *I);

/* Dynamic update for the ascending row set I[K] (device) with the residual r
 * (device, m doubles, read at I): x += A_I^T (A_I A_I^T + mu I)^{-1} r_I, or,
 * when K >= n, x += (A_I^T A_I + mu I)^{-1} A_I^T r_I (Lemma 1).  The kernel
 * checks I before any row is read: an entry outside [0, m) or a set that is
 * not strictly ascending leaves x unchanged and returns RORBK_ERR_BOUNDS. */
rorbk_status rorbk_dynamic_update(rorbk_handle h, const int32_t *I,
                                  const double *r, double *x);

/* The residual-weighted running sum (RORBK_DIST_RESIDUAL_WEIGHTED) that the
 * draws after the residual r (device, m doubles) use: w_t = Pbar_t * rho_t,
 * rho_t = sum of r_i^2 over block t's rows (one fused chain, rows ascending),
 * and its running sum formed as the solve forms it (chunks of 64 blocks, each
 * from zero, then the chunk totals in order); cdf_host receives k doubles.
 * The result differs from the sequential running sum by rounding only (at
 * most a few units in the last place of cdf[k-1] per 64 blocks).  Not in the
 * paper, whose proposal is static. */
rorbk_status rorbk_weighted_cdf(rorbk_handle h, const double *r, double *cdf_host);

/* The dynamic block's Gram G = A_I A_I^T + mu I for the ascending row set I[K]
 * (device int32) of a DENSE handle, written packed lower (row-major: entry
 * (a, b), b <= a, at a (a + 1) / 2 + b) to G (device, K (K + 1) / 2 doubles).
 *   precision = RORBK_PREC_FP64 : the FP64 kernel of Algorithm 1's dynamic
 *     block update, each entry one fused chain over ascending columns.
 *   precision = RORBK_PREC_MIXED : the kernel of the mixed-precision inner
 *     solve: TF32 products of A's FP32 copy accumulated in FP32 on the tensor
 *     cores (tcgen05) per 128-column chunk, the chunks added in FP64; entry
 *     error within about 2^-10 sum_j |a_aj a_bj| (TF32 keeps 10 mantissa bits).
 *     Needs a handle set up with precision = RORBK_PREC_MIXED.
 * Sparse handles, an unknown precision or a mixed request on an FP64 handle:
 * RORBK_ERR_UNSUPPORTED / RORBK_ERR_INVALID_ARG.  Enqueued on the handle's
 * stream and waited for. */
rorbk_status rorbk_dense_gram(rorbk_handle h, const int32_t *I, double *G, int32_t precision);

/* ---- the initial solution of Algorithm 2 (Appendix) -----------------------
 * x0 = (<b, b~> / ||b~||^2) y, y = the sum of the rows of static block
 * `block` (each column summed over the block's rows in ascending order),
 * b~ = A y.  x0 lies in range(A^T) and ||b - A x0|| <= ||b|| (the Remark after
 * Algorithm 2); pass it as x0 to rorbk_solve.  b (m) and x0 (n) are device
 * FP64 vectors; the call uses the handle's workspace and returns when x0 is
 * written.  Errors: RORBK_ERR_INVALID_ARG for a NULL pointer, a block outside
 * [0, k), or A y = 0. */
rorbk_status rorbk_initial_solution(rorbk_handle h, int64_t block, const double *b, double *x0);

/* ---- Algorithm 3 (Appendix): flexible AB-GMRES with ROR-BK inside -------
 * Solves A x = b by GMRES on A B with B = ROR-BK as a right preconditioner:
 * x = x0 (NULL: 0), v_1 = (b - A x) / ||b - A x||; outer step j runs ROR-BK on
 * A z = v_j from z = 0 (rorbk_solve on this handle with tolerance eta and at
 * most lmax iterations; the Philox counter continues from opt->start_iter
 * across the inner solves), w = A z_j, modified Gram-Schmidt against
 * v_1..v_j (h_ij = <w, v_i>), v_{j+1} = w / ||w||, and Givens rotations on the
 * Hessenberg matrix.  It stops when the GMRES residual estimate reaches
 * tol * ||b||, at breakdown or after maxit (<= 4096) outer steps, then forms
 * x += Z y.  b (m), x0 and x (n) are device FP64 vectors; opt as for
 * rorbk_solve (FP64 or MIXED inner solves; no host loop, trace or weighted
 * draws).  res->iters = outer steps, res->refinements = inner ROR-BK
 * iterations in total, res->rrn = ||b - A x|| / ||b|| of the returned x.
 * The Krylov basis ((maxit + 1) m + maxit n doubles) is allocated for the
 * call.  Returns RORBK_OK or RORBK_NOT_CONVERGED; errors as rorbk_solve. */
rorbk_status rorbk_fabgmres(rorbk_handle h, const double *b, const double *x0, double *x,
                            double tol, int64_t maxit, double eta, int64_t lmax,
                            const rorbk_options *opt, rorbk_result *res);

/* ---- many solves in one launch --------------------------------------
 * (Beside the paper: its method solves one system; these run many ROR-BK
 * solves at once, each exactly the solve rorbk_solve would run.)
 *
 * rorbk_clone: a new handle *out that shares every set-up product of src (A
 *   and its copies, the partition, the proposal, the static operators: all
 *   read-only during solves) and owns a fresh per-solve workspace (vectors,
 *   loop state, dynamic-block scratch).  It solves the same system: use one
 *   clone per right-hand side.  The shared memory is freed when the last of
 *   src and its clones is freed (rorbk_free), in any order.  Errors:
 *   RORBK_ERR_INVALID_ARG (NULL), RORBK_ERR_OOM, RORBK_ERR_CUDA.
 * rorbk_batch_create: captures the whole solve loop of each of count
 *   distinct handles (systems of any sizes, clones, blocks of right-hand
 *   sides from rorbk_multi_create, or a mix; one device) as
 *   independent components of one CUDA graph, for precision FP64 or MIXED
 *   (MIXED needs handles set up for it).  The handles must outlive the batch
 *   and must not be solved on their own while a batch solve runs.  Errors:
 *   RORBK_ERR_INVALID_ARG (NULL or repeated handle, mixed devices, unknown
 *   precision), RORBK_ERR_CUDA; the message is at rorbk_last_error(NULL).
 * rorbk_batch_solve: one graph launch that runs every handle's solve to its
 *   own stop (tolerance, maxit or error): solve i takes device vectors b[i]
 *   (its m), x0[i] (its n; x0 == NULL or x0[i] == NULL: zero) and writes
 *   x[i] (its n); for a block of nr right-hand sides these are its m x nr and
 *   n x nr row-major arrays.  opt is shared (precision must be the batch's; host_loop and
 *   trace are not available); system_ids[i] (NULL: all opt->system_id) is
 *   solve i's Philox key word 1, so clones given the same id share the
 *   sampled block stream.  res[count] (may be NULL) receives each solve's
 *   result; time_ms is the whole launch.  Returns the first error of any
 *   solve, else RORBK_NOT_CONVERGED if any solve stopped at maxit, else
 *   RORBK_OK.
 * rorbk_batch_free: NULL-safe; does not free the handles. */
typedef struct rorbk_batch_ctx *rorbk_batch;
rorbk_status rorbk_clone(rorbk_handle src, rorbk_handle *out);
rorbk_status rorbk_batch_create(const rorbk_handle *hs, int32_t count, int32_t precision,
                                rorbk_batch *out);
rorbk_status rorbk_batch_solve(rorbk_batch batch, const double *const *b, const double *const *x0,
                               double *const *x, double tol, int64_t maxit,
                               const rorbk_options *opt, const uint64_t *system_ids,
                               rorbk_result *res);
void rorbk_batch_free(rorbk_batch batch);

/* ---- a block of right-hand sides ----------------------------------------
 * (Beside the paper, which solves one right-hand side.)  A x_j = b_j for
 * j = 0 .. nr-1, each column solved exactly as rorbk_solve would solve it
 * alone: its own Philox stream (key (seed, system_id), counter start_iter + j'
 * for its iteration j'), its own top-K sets, dynamic updates and stopping test
 * (a column that reaches the tolerance stops while the others continue), so
 * its iterates are those of the one-column solve.  What the block shares is
 * the data movement: the residual R = B - A X of all columns is one pass over
 * A, each gather of x bringing one contiguous row of X; the sampled updates of
 * all columns run side by side (one block of threads per column) and the
 * top-K and dynamic-update kernels run with one grid row per column.
 *
 * rorbk_multi_create: a handle *out for nr = 2, 4, 8, 16 or 32 right-hand sides
 *   of src's system.  It shares src's set-up (as rorbk_clone does) and owns
 *   nr per-column workspaces.  Sparse (CSR) systems whose static blocks and
 *   dynamic block have fewer rows than A has columns (else
 *   RORBK_ERR_UNSUPPORTED); src must be a one-column handle.  Free with
 *   rorbk_free; rorbk_solve on it is RORBK_ERR_INVALID_ARG.
 * rorbk_solve_multi: B (device, m x nr row-major: B[i * nr + j] = b_j[i]),
 *   X0 (n x nr row-major or NULL for 0) and X (n x nr row-major, may alias
 *   X0) as rorbk_solve's b, x0 and x for every column; tol, maxit and opt as
 *   rorbk_solve (FP64 or MIXED precision, the paper's draws, the exact
 *   residual; host_loop allowed; opt->trace, if not NULL, points to an array
 *   of nr records, one per column, FP64 only).  res (may be NULL) receives
 *   nr results, column j's in res[j].  Returns the first error of any column,
 *   else RORBK_NOT_CONVERGED if some column stopped at maxit, else RORBK_OK.
 * rorbk_solve_multi_host: the same with host buffers (copies inside the call).
 * rorbk_multi_results: the nr per-column results of the handle's last solve
 *   (also after rorbk_batch_solve, whose res entry for such a handle holds
 *   the largest iteration count and RRN and converged = all columns). */
rorbk_status rorbk_multi_create(rorbk_handle src, int32_t nr, rorbk_handle *out);
rorbk_status rorbk_solve_multi(rorbk_handle h, const double *B, const double *X0, double *X,
                               double tol, int64_t maxit, const rorbk_options *opt,
                               rorbk_result *res);
rorbk_status rorbk_solve_multi_host(rorbk_handle h, const double *B_host, const double *X0_host,
                                    double *X_host, double tol, int64_t maxit,
                                    const rorbk_options *opt, rorbk_result *res);
rorbk_status rorbk_multi_results(rorbk_handle h, rorbk_result *res);

/* The block's residual as a single step: R = B - A X for all nr columns in one
 * pass over A.  precision = RORBK_PREC_FP64: B (m x nr), X (n x nr), R (m x nr)
 * are FP64, each entry one fused chain over the row's stored entries in order
 * (as rorbk_residual); RORBK_PREC_MIXED: FP32 arrays and FP32 chains (as
 * rorbk_residual32; the handle must be set up for mixed precision).  All
 * row-major, device memory.  R == NULL keeps the residual in the handle only
 * (for timing).  rr_host (nr doubles) receives ||r_j||^2; with rr_host == NULL
 * the call only enqueues on the handle's stream. */
rorbk_status rorbk_residual_multi(rorbk_handle h, int32_t precision, const void *B, const void *X,
                                  void *R, double *rr_host);

/* ---- launch shapes ------------------------------------------------------
 * (Beside the paper.)  Grids that leave every result unchanged: the top-K
 * passes (their counts are exact whatever the grid), the dynamic update's
 * gather and scatter (each entry's arithmetic is fixed), and, for a block of
 * right-hand sides, the block residual (whose grid changes only the order in
 * which per-block sums of squares are added, so a stopping test can move
 * only when the relative residual lies within rounding of the tolerance).
 * All counts are per column of a block; 0 selects the library's default.
 *   us_default, us_tuned: microseconds per iteration measured by
 *   rorbk_autotune with the defaults and with the chosen shapes. */
typedef struct {
    int32_t topk_blocks;         /* first/second top-K pass             */
    int32_t collect_blocks;      /* top-K candidates pass               */
    int32_t dyn_mark_blocks;     /* dynamic update: gather and marks    */
    int32_t dyn_scatter_blocks;  /* dynamic update: x += A_I^T y        */
    int32_t residual_blocks;     /* block residual (blocks of columns)  */
    int32_t graph_unroll;        /* iterations per execution of the graph
                                    loop's body (1..16): the body holds that
                                    many iterations, and those after the
                                    loop's end return at once             */
    double us_default, us_tuned;
} rorbk_tuning;

/* rorbk_autotune: chooses the shapes above for this handle by timing iters
 * host-driven iterations per candidate (coordinate descent over each shape in
 * turn, candidates 1/4 .. 4 x the default), then the graph's unroll (1, 2, 4
 * or 8; iters graph-launched iterations per candidate), every candidate from
 * the same state: the iterate after iters iterations from x0 = 0 on the right-hand
 * side b (device; m doubles, or m x nr row-major for a block), with the same
 * draws.  precision: the iteration to tune (RORBK_PREC_FP64, or
 * RORBK_PREC_MIXED for the FP32 inner iterations).  cache_file (may be NULL):
 * a text file of earlier choices, one line per (m, nnz, k, nr, precision,
 * SMs); a matching line is applied without timing, a new choice is appended.
 * The shapes are applied to h (and kept by later clones); *out (may be NULL)
 * receives them.  Allocates a scratch copy of x for the call.  Errors: as
 * rorbk_solve; RORBK_ERR_INVALID_ARG for b == NULL or iters < 1.
 * rorbk_set_tuning: applies given shapes (NULL: the defaults). */
rorbk_status rorbk_autotune(rorbk_handle h, const double *b, int32_t precision, int64_t iters,
                            const char *cache_file, rorbk_tuning *out);
rorbk_status rorbk_set_tuning(rorbk_handle h, const rorbk_tuning *t);
/* A change of shapes drops the handle's instantiated graphs (the next solve
 * captures them again); a batch built earlier keeps the shapes it was built
 * with. */

/* ---- the differentiable solve ------------------------------------------
 * (No counterpart in the paper, which never differentiates its solution.)
 * For square non-singular A and a loss L(x) with x = A^{-1} b:
 *   dL/db = g with A^T g = dL/dx (the adjoint system), dL/dA = -g x^T,
 * restricted to A's stored pattern: dL/da_ij = -g_i x_j.
 *
 * rorbk_setup_adjoint: a new handle *out for the adjoint system, built from
 *   h's own copy of A.  ROR-BK, like every Kaczmarz-type method, is invariant
 *   to row scaling but not to column scaling, and A's row scaling is a column
 *   scaling of A^T; so the handle holds At~ = A^T C^{-1} with
 *   C = diag(||A_i||_2) (1 for a zero row): the transpose of A with its rows
 *   normalised, in FP64 values, each row of At~ listing its columns
 *   ascending.  It is then set up exactly as rorbk_setup would (Algorithm 1
 *   set-up on At~).  part partitions the n rows of At~; lambda and opt as
 *   for rorbk_setup (opt == NULL: defaults on h's stream).  Free *out with
 *   rorbk_free.  Errors: as rorbk_setup; RORBK_ERR_INVALID_ARG for a NULL h,
 *   part or out.
 * rorbk_adjoint_solve: solves A^T g = y on such a handle: ROR-BK on
 *   At~ h = y (as rorbk_solve, from h0 = 0), then g = C^{-1} h.  Because
 *   At~ h = A^T g, res->rrn is ||y - A^T g|| / ||y||.  y (length n of A)
 *   and g (length m of A) are device FP64 vectors; returns when g is
 *   written.  Errors: as rorbk_solve; RORBK_ERR_INVALID_ARG if adj was not
 *   made by rorbk_setup_adjoint.
 * rorbk_value_grad: dvals[p] = -(g_i * x_j) for every stored entry p = (i, j)
 *   of h's A, in the CSR order A was given in (nnz doubles).  g (m) and x (n)
 *   are device FP64 vectors; enqueued on h's stream, not waited for.  Errors:
 *   RORBK_ERR_INVALID_ARG for NULL pointers. */
rorbk_status rorbk_setup_adjoint(rorbk_handle h, const rorbk_partition *part, double lambda,
                                 const rorbk_options *opt, rorbk_handle *out);
rorbk_status rorbk_adjoint_solve(rorbk_handle adj, const double *y, double *g, double tol,
                                 int64_t maxit, const rorbk_options *opt, rorbk_result *res);
rorbk_status rorbk_value_grad(rorbk_handle h, const double *g, const double *x, double *dvals);

/* ---- a residual that allocates nothing --------------------------------
 * (No counterpart in the paper: a service for callers that cannot allocate.)
 * Some callers cannot call cudaMalloc where they need a residual: code that
 * runs inside an allocator or a memory-pool callback, processes whose device
 * memory a framework has fully reserved at start-up, and real-time loops
 * that forbid allocation after initialisation.  This entry point computes
 * r = b - A x and ||r||^2 for a CSR matrix in the caller's device memory
 * without any handle and without allocating: its per-block partial sums and
 * its completion counter live in a fixed file-scope device array.
 *   m, n, nnz, row_ptr, col_idx, values, dtype : the CSR matrix (device
 *       pointers; conventions as rorbk_matrix), m <= 16777216 (= 256 rows per
 *       thread block x 65536 partial sums), n and nnz below 2^31;
 *   b (m), x (n), r (m) : device FP64 vectors; rr_out : one device double
 *       that receives ||r||^2;
 *   stream : cudaStream_t (NULL = legacy default).  The call only enqueues.
 * Each row is a fused multiply-add chain over its stored entries in order
 * (the arithmetic of rorbk_residual), the sum of squares a fixed tree.
 * The scratch (about 512 KiB) is held by every GPU that loads the library
 * until the process exits.  All calls on a device share it and it keeps the
 * last call's contents: each call clears the completion counter on its stream
 * before its kernel starts (a 4-byte cudaMemsetAsync, not an allocation), so
 * calls ordered on one stream are independent, even after a call whose kernel
 * never finished; calls that overlap on the GPU race and give wrong results.
 * The first call on a device looks up the scratch's device address (once per
 * device, with that device current) and keeps it for the process: make that
 * first call before any stream capture begins, and do not use the entry point
 * after cudaDeviceReset (the kept address belongs to the reset context).
 * Errors: RORBK_ERR_INVALID_ARG (message in rorbk_last_error(NULL)),
 * RORBK_ERR_CUDA. */
rorbk_status rorbk_csr_residual_noalloc(int64_t m, int64_t n, int64_t nnz,
                                        const int32_t *row_ptr, const int32_t *col_idx,
                                        const void *values, int32_t dtype, const double *b,
                                        const double *x, double *r, double *rr_out,
                                        void *stream);

#ifdef __cplusplus
}
#endif
#endif /* RORBK_H */
