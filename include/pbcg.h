/*
 * pbcg.h -- C ABI of the GB300 (sm_103a) solver library libpbcg.so.
 *
 * Solves A x = b for a sparse, unsymmetric A in FP64 CSR with classical
 * BiCGStab (Algorithm 1 of arXiv 2404.13216, after van der Vorst) or pipelined
 * BiCGStab (Algorithm 2, after Cools and Vanroose), given x_0, a relative
 * tolerance and an iteration cap -- the problem statement of Section 2.  Dot
 * products are either plain FP64 or exact: the real sum rounded once to the
 * nearest double, the accuracy the paper obtains from the ExBLAS long
 * accumulator (Section 2) in place of residual replacement.
 *
 * Arithmetic contract (both dot modes): each SpMV row is an fma chain over the
 * row's stored entries in stored order starting from +0; every vector update
 * is the fixed fma form listed with the solver entry points below; scalars use
 * IEEE division and square root.  In exact mode the residual history,
 * iteration count and x are therefore a deterministic function of the inputs,
 * independent of launch shape, batching and partitioning.
 *
 * Conventions
 *   - Every call returns an int: 0 or a positive solver status on completion,
 *     a negative PBCG_ERR_* code on error (the context's last-error string then
 *     says why).  No call aborts the process.
 *   - Vector arguments (b, x, row_ptr, ...) may be host or device pointers; the
 *     library finds out which with cudaPointerGetAttributes.  Device pointers
 *     must be on the context's device.  The caller keeps ownership of every
 *     buffer it passes; the library copies what it keeps.
 *   - A context owns one CUDA stream (its own, or the caller's) and is not
 *     thread-safe: use one context per host thread.
 *   - Index types: int32 row pointers and column indices (nnz < 2^31).
 */
#ifndef PBCG_H
#define PBCG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pbcg_ctx pbcg_ctx;   /* opaque, library-owned */
typedef struct pbcg_mat pbcg_mat;   /* opaque, library-owned device copy of a CSR matrix */

/* solver statuses (>= 0) and error codes (< 0) */
enum {
    PBCG_OK = 0,            /* converged: true relative residual <= tol */
    PBCG_MAXIT = 1,         /* maxit iterations done without convergence */
    PBCG_BREAKDOWN = 2,     /* zero or non-finite denominator in alpha, beta or omega */
    PBCG_NONFINITE = 3,     /* NaN/Inf reached a dot product (input or overflow) */
    PBCG_ERR_INVALID = -1,  /* bad argument; nothing was launched */
    PBCG_ERR_OOM = -2,      /* device allocation failed */
    PBCG_ERR_CUDA = -3,     /* a CUDA call failed */
    PBCG_ERR_TIMEOUT = -4,  /* a bounded device wait expired */
    PBCG_ERR_COMM = -5      /* a communicator callback of a partitioned solve failed */
};

enum { PBCG_ALG_BICGSTAB = 0, PBCG_ALG_PIPELINED = 1, PBCG_ALG_PIPELINED_RR = 2 };
enum { PBCG_DOT_PLAIN = 0, PBCG_DOT_EXACT = 1 };

typedef struct {
    int32_t iters;            /* completed loop bodies */
    int32_t status;           /* PBCG_OK .. PBCG_NONFINITE */
    double relres_recursive;  /* sqrt((r,r)) / sqrt((b,b)) of the last iterate, solve's dot mode */
    double relres_true;       /* ||b - A x||_2 / ||b||_2 with the fixed SpMV and exact dots */
    double seconds;           /* wall time of the call on the host */
    int32_t launches;         /* kernel launches the call issued (graph-body kernels counted per body execution:
                                 a body holds 16 iterations, whose passes after a stop return at once) */
    int32_t reserved;
} pbcg_result;

/*
 * Create a context on CUDA device `device`.  cuda_stream: a cudaStream_t to
 * launch on, or NULL for a stream the context creates and owns.
 * Errors: INVALID (out == NULL or bad device), CUDA, OOM.
 */
int pbcg_create(pbcg_ctx **out, int device, void *cuda_stream);

/* Destroy a context and everything it allocated.  destroy(NULL) is a no-op. */
void pbcg_destroy(pbcg_ctx *ctx);

/* The last error message of this context ("" if none).  The string lives until the next call. */
const char *pbcg_last_error(pbcg_ctx *ctx);

/*
 * Copy a CSR matrix to the device.  row_ptr[n+1], col_idx[nnz], vals[nnz];
 * host or device pointers (ptrs_on_device is a hint only, the library checks).
 * Validation (INVALID on failure): 1 <= n <= 2^30 - 1, nnz >= 0, row_ptr[0] == 0,
 * row_ptr non-decreasing, row_ptr[n] == nnz < 2^31, 0 <= col_idx < n.
 * Duplicate columns are allowed and summed in stored order.
 * The matrix belongs to ctx and is freed by pbcg_mat_free or pbcg_destroy.
 */
int pbcg_csr_upload(pbcg_ctx *ctx, int32_t n, int64_t nnz, const int32_t *row_ptr, const int32_t *col_idx,
                    const double *vals, int ptrs_on_device, pbcg_mat **out);

/* Free a matrix created by pbcg_csr_upload (NULL is a no-op). */
int pbcg_mat_free(pbcg_ctx *ctx, pbcg_mat *mat);

/*
 * Solve A x = b from x (in: x_0, out: the last iterate, written for every
 * status).  b and x hold n doubles each.  alg: PBCG_ALG_* (PIPELINED_RR is
 * Algorithm 2 with residual replacement, see pbcg_set_option); dot_mode:
 * PBCG_DOT_*.  tol > 0; 0 <= maxit <= 2^31 - 2 (the history holds maxit + 1
 * entries); INVALID otherwise.
 *
 * Algorithm 2 (p-BiCGStab), with omega the scalar (q,y)/(y,y) and w the
 * vector A r (the paper uses the letter w for both):
 *   r_0 = b - A x_0, w_0 = A r_0 (the paper prints "A - r_0"), t_0 = A w_0,
 *   alpha_0 = (r_0,r_0)/(r_0,w_0); p_0 = r_0, s_0 = w_0, z_0 = t_0; then per i
 *     p = fma(beta, fma(-omega, s, p), r)   s = fma(beta, fma(-omega, z, s), w)
 *     z = fma(beta, fma(-omega, v, z), t)   q = fma(-alpha, s, r)
 *     y = fma(-alpha, z, w)                 v = A z      omega = (q,y)/(y,y)
 *     x = fma(omega, q, fma(alpha, p, x))   r = fma(-omega, y, q)
 *     w = fma(-omega, fma(-alpha, v, t), y) t = A w
 *     beta  = (alpha/omega) * ((r_0,r_new)/(r_0,r_old))
 *     alpha = (r_0,r_new) / (((r_0,w) + beta*(r_0,s)) - (beta*omega)*(r_0,z))
 * Algorithm 1 (BiCGStab): s = A p, alpha = (r_0,r)/(r_0,s), q = fma(-alpha,s,r),
 *   y = A q, omega = (q,y)/(y,y), x and r as above, beta as above,
 *   p = fma(beta, fma(-omega, s, p), r).
 *
 * Stopping (the paper gives none): res_k = sqrt((r_k,r_k))/sqrt((b,b)) in the
 * solve's dot mode is tested at k = 0 and after every iteration; when
 * res_k <= target the true residual ||b - A x||/||b|| (exact dots) is formed
 * and the solve stops if it is <= tol, else target = tol*(tol/true) and the
 * iteration continues unchanged.  (y,y) = 0 gives omega = 0 and, unless that
 * step converged, BREAKDOWN.  The residual history (res_0 .. res_iters) is
 * kept for pbcg_residual_history.
 *
 * Reproducibility: exact-mode results are bit-identical whatever the grid,
 * schedule or batch.  Plain-mode dots sum per-CTA partials; on a matrix whose
 * 256-row tiles exceed the shared-memory stage (more than 7 stored entries
 * per row on average, e.g. power-law rows) the passes hand tiles out
 * dynamically, so plain results there may differ in the last bits from run
 * to run.
 *
 * Returns the status (also in out->status) or a negative error.
 */
int pbcg_solve(pbcg_ctx *ctx, const pbcg_mat *A, const double *b, double *x, double tol, int32_t maxit,
               int alg, int dot_mode, pbcg_result *out);

/*
 * Solve nsys independent systems stored as one block-diagonal matrix:
 * system k owns rows (and columns) [sys_row_ptr[k], sys_row_ptr[k+1]) of A.
 * b, x: A's n entries; tol: nsys tolerances; out: nsys results.
 * Every system runs the same arithmetic as a pbcg_solve of its own block,
 * bit for bit in exact mode, and stops on its own.
 * Validation adds: sys_row_ptr[0] == 0, strictly increasing,
 * sys_row_ptr[nsys] == n, and no entry of a block outside its own columns.
 * Returns 0 when every system converged, else the largest status, or an error.
 */
int pbcg_solve_batched(pbcg_ctx *ctx, const pbcg_mat *A, int32_t nsys, const int32_t *sys_row_ptr,
                       const double *b, double *x, const double *tol, int32_t maxit, int alg, int dot_mode,
                       pbcg_result *out);

/*
 * Copy the residual history res_0 .. res_iters of the last solve (sys = 0) or
 * of system `sys` of the last batched solve into out[0 .. cap-1]; *len gets
 * the full length (iters + 1).  INVALID if no such history exists.
 */
int pbcg_residual_history(pbcg_ctx *ctx, int32_t sys, double *out, int32_t cap, int32_t *len);

/*
 * Pools: continuous batching of independent solves (serving).
 *
 * The method is that of pbcg_solve (Section 2, Algorithm 1 or 2 with the
 * stopping rule above); a pool only changes when each system starts and
 * stops.  Requests are admitted while others run, every live system advances
 * in the same launches, and a finished one leaves without stopping the rest.
 * Each system's arithmetic is the same as its own pbcg_solve: bit for bit in
 * exact mode.
 *
 * Memory: one block-diagonal SELL-32 layout of fixed capacity allocated by
 * pbcg_pool_create.  A system takes ceil(n / 256) whole 256-row tiles of the
 * 13 pool vectors and sum over its 32-row slices of 32 * (longest row of the
 * slice) matrix entries; both come from first-fit range allocators.
 *
 * Streams: steps run on the context's stream; uploads and result copies on a
 * stream the pool creates.  pbcg_pool_step only enqueues work; pbcg_pool_poll
 * reads control-block snapshots taken after each step and blocks only when
 * asked to.  One host thread at a time may call a pool's functions.
 */
typedef struct pbcg_pool pbcg_pool;  /* opaque, library-owned */

typedef struct {
    int64_t max_rows;          /* rows of all resident systems together (each rounded up to 256) */
    int64_t max_entries;       /* SELL-32 entries of all resident systems together */
    int32_t max_slots;         /* systems resident at a time */
    int32_t maxit;             /* largest maxit a request may ask for, 0 .. 2^31 - 2 (history length maxit + 1) */
    int32_t alg;               /* PBCG_ALG_*, for every system of the pool */
    int32_t dot_mode;          /* PBCG_DOT_*, for every system of the pool */
    int64_t max_request_rows;  /* largest n of one request */
    int64_t max_request_nnz;   /* largest nnz of one request (sizes the upload staging) */
    int32_t precond;           /* PBCG_PRECOND_NONE or PBCG_PRECOND_JACOBI, for every system of the pool */
    int32_t reserved;          /* 0 */
} pbcg_pool_config;

/*
 * Create a pool on ctx's device.  Device memory: about 8 * (13 * max_rows +
 * 1.5 * max_entries + max_slots * (maxit + 1)) + 12 * max_request_nnz bytes.
 * Errors: INVALID (NULL, non-positive or too large sizes, unknown alg,
 * dot_mode or precond, reserved not 0), OOM, CUDA.  A pool must be destroyed
 * before its context.  With precond = PBCG_PRECOND_JACOBI it holds 8 *
 * max_rows more bytes (the diagonals).
 */
int pbcg_pool_create(pbcg_ctx *ctx, const pbcg_pool_config *cfg, pbcg_pool **out);

/* Wait for the pool's work and free it.  destroy(NULL) is a no-op. */
void pbcg_pool_destroy(pbcg_pool *pool);

/*
 * Admit one system A x = b (CSR as for pbcg_csr_upload; row_ptr, col_idx,
 * vals, b, x0 host or device pointers; x0 NULL means zero) with its own tol
 * and maxit (<= the pool's maxit).  Its setup passes and iterations run in
 * the following pbcg_pool_step calls.  The caller's arrays are consumed when
 * the call returns.  Host work: O(n) on the row pointers; the column indices
 * are checked on the device, and a request with an index outside [0, n)
 * finishes at once with PBCG_ERR_INVALID as its result.  In a pool created
 * with precond = PBCG_PRECOND_JACOBI the request runs on A M^-1 y = b, M =
 * diag(A), with the fixed forms of pbcg_solve (d_i summed in stored order,
 * entries v / d_col, y0 = x0 * d, x = y / d in pbcg_pool_result); a row
 * whose diagonal is absent, zero or non-finite also ends it with
 * PBCG_ERR_INVALID.
 * Returns 0 and the slot in *slot, 1 when the pool has no room for it now
 * (no free slot, tile range or entry range; *slot = -1), or an error
 * (INVALID: NULL pointer, n or nnz beyond the pool's request limits, bad
 * row_ptr, tol <= 0, maxit out of range).
 */
int pbcg_pool_admit(pbcg_pool *pool, int32_t n, int64_t nnz, const int32_t *row_ptr, const int32_t *col_idx,
                    const double *vals, const double *b, const double *x0, double tol, int32_t maxit,
                    int32_t *slot);

/*
 * Enqueue one step: at most `iters` iterations of every live system (fewer
 * when none is left running), as one graph launch, followed by a snapshot of
 * the control blocks.  Does not wait for the GPU unless four steps are
 * already in flight.  Errors: INVALID (iters < 1), CUDA.
 */
int pbcg_pool_step(pbcg_pool *pool, int32_t iters);

/*
 * Report systems that finished, each once: the newest completed snapshot is
 * scanned and up to cap finished slots are written to slots[]; *count gets
 * how many were found (it can exceed cap; the rest are reported by the next
 * call).  wait != 0 first waits for the newest step.  *pending (may be NULL)
 * gets the number of steps not yet complete.
 * Errors: INVALID (count NULL, cap < 0, or cap > 0 with slots NULL), CUDA.
 */
int pbcg_pool_poll(pbcg_pool *pool, int wait, int32_t *slots, int32_t cap, int32_t *count, int32_t *pending);

/*
 * Retire a reported slot: copy its n solution entries to x (host or device,
 * may be NULL) and its result to out (may be NULL; status PBCG_OK ..
 * PBCG_NONFINITE, or PBCG_ERR_INVALID / PBCG_ERR_TIMEOUT for a request that
 * failed), then free its slot, tiles and entries for later admissions.
 * Waits only for the copy of x.  Returns the status, or the request's error,
 * or INVALID when the slot was not reported by pbcg_pool_poll.
 */
int pbcg_pool_result(pbcg_pool *pool, int32_t slot, double *x, pbcg_result *out);

/*
 * Residual history res_0 .. res_iters of a reported, not yet retired slot,
 * as for pbcg_residual_history (out host memory; empty for a request that
 * ended INVALID).  Errors: INVALID (the slot was not reported or is
 * retired), CUDA.
 */
int pbcg_pool_history(pbcg_pool *pool, int32_t slot, double *out, int32_t cap, int32_t *len);

/*
 * Free room: free slots, the largest free row range (a multiple of 256) and
 * the largest free entry range.  Any output may be NULL.  Errors: INVALID
 * (pool NULL).
 */
int pbcg_pool_room(const pbcg_pool *pool, int32_t *free_slots, int64_t *free_rows, int64_t *free_entries);

/*
 * Context options.
 *   PBCG_OPT_RR_PERIOD: k >= 1, the period of residual replacement used by
 *     PBCG_ALG_PIPELINED_RR (default 50).  Section 2 names residual replacement
 *     (resetting r, w, s and z to their true values every k iterations) as the
 *     stabiliser that exact dot products are proposed to replace, and the
 *     experiments compare against it (p-BiCGStabRR).  The paper gives no
 *     schedule beyond "every k iterations"; this library replaces at the start
 *     of every iteration i > 0 with i mod k == 0: r = b - A x, w = A r, p by
 *     its recurrence from the new r, s = A p, z = A s (t = A w follows in the
 *     same iteration); the scalars are kept.
 *   PBCG_OPT_PRECOND: PBCG_PRECOND_NONE (default) or PBCG_PRECOND_JACOBI.
 *     Section 2 notes that real implementations add a preconditioner M (its
 *     experiments use none).  With PBCG_PRECOND_JACOBI, pbcg_solve runs
 *     Algorithm 1 or 2 on the right-preconditioned system A M^{-1} y = b with
 *     M = diag(A), then returns x = M^{-1} y; a diagonal M is applied as
 *     scaled matrix entries, so no iteration does extra work.  Fixed forms:
 *     d_i = sum, in stored order, of row i's entries in column i (zero,
 *     non-finite or absent: INVALID); entries v / d_col (one IEEE division);
 *     y0 = x0 * d; x = y / d.  Residual histories and relres_* are those of
 *     the scaled system.  pbcg_solve_batched applies it to every system (a
 *     block-diagonal M); a pool applies it when its pbcg_pool_config asks
 *     for it (the option does not reach pools).
 *   PBCG_OPT_SMALL_CLUSTER: 1 (default) or 0.  With 1, pbcg_solve runs the
 *     iterations of Algorithm 1 or 2 (not PBCG_ALG_PIPELINED_RR) on a system
 *     of at most 16384 rows whose rows fit in shared memory as one launch
 *     over one thread-block cluster of up to 16 CTAs per stop test, the
 *     reduction points of every iteration becoming cluster barriers; with 0
 *     it uses the launch graph of passes whatever the size.  Exact-mode
 *     results are bit-identical either way; plain-mode dots sum their
 *     partials over fewer CTAs.  pbcg_profile_solve always runs the passes.
 *   PBCG_OPT_BATCH_GRAPH: 1 (default) or 0.  With 0, pbcg_solve_batched
 *     launches every kernel of its iteration loop from the host and reads
 *     the control kernel's "any system live" flag after each iteration,
 *     instead of one CUDA-graph launch with a conditional WHILE node; results
 *     are identical.  For profilers, which do not profile single kernels of a
 *     graph with conditional nodes.
 * Returns 0, or INVALID for an unknown option or value.
 */
enum { PBCG_OPT_RR_PERIOD = 1, PBCG_OPT_PRECOND = 3, PBCG_OPT_SMALL_CLUSTER = 4, PBCG_OPT_BATCH_GRAPH = 5 };
enum { PBCG_PRECOND_NONE = 0, PBCG_PRECOND_JACOBI = 1 };
int pbcg_set_option(pbcg_ctx *ctx, int option, int64_t value);

/*
 * Standalone kernels of the solver, for checks and measurement.
 * pbcg_dot: *out = (a, b) over n entries in dot_mode (exact: correctly
 *   rounded; NaN if an operand is NaN or Inf).  a, b host or device.
 * pbcg_spmv: y = A x with the fixed fma row order.  x, y host or device.
 * Errors: INVALID (NULL output or operand, n < 0, unknown dot_mode, a
 * matrix not of this context), OOM (host operands of pbcg_dot are staged in
 * device buffers freed before it returns), CUDA.  Both wait for the result.
 */
int pbcg_dot(pbcg_ctx *ctx, int64_t n, const double *a, const double *b, int dot_mode, double *out);
int pbcg_spmv(pbcg_ctx *ctx, const pbcg_mat *A, const double *x, double *y);

/*
 * Failure-detection check of the bounded device wait the staged passes use
 * on their shared-memory barriers: one CTA waits, with the passes' wait
 * function limited to `probes` attempts (1 .. 2^22; the passes use 2^18,
 * about one second on GB300), on
 * a barrier phase that nothing completes.  *expired receives 1 when the wait
 * gave up and reported it (the expected outcome; a pass then ends its solve
 * with PBCG_ERR_TIMEOUT), 0 if the phase completed; *seconds the time the
 * wait took, measured on the device.  The context stays usable.  Returns 0,
 * INVALID for a bad argument, or CUDA.
 */
int pbcg_check_wait(pbcg_ctx *ctx, int32_t probes, int32_t *expired, double *seconds);

/*
 * Time the solver's kernels: run the solve of pbcg_solve with a host-driven
 * launch loop (no CUDA graph) and CUDA events around every launch, on the
 * context's stream.  names receives up to cap kernel names (a
 * '\0'-terminated string each, at most 31 characters), ms their total
 * durations, launches their launch counts; *count gets the number of kernels.
 * Any of names, ms, launches and count may be NULL (that output is skipped).
 * The solve's results, return value and errors are those of pbcg_solve.
 */
int pbcg_profile_solve(pbcg_ctx *ctx, const pbcg_mat *A, const double *b, double *x, double tol,
                       int32_t maxit, int alg, int dot_mode, pbcg_result *out, char (*names)[32],
                       double *ms, int32_t *launches, int32_t cap, int32_t *count);

/*
 * Launch variants and the autotuner.
 *
 * How the passes are launched changes neither the paper's arithmetic nor,
 * in exact mode, a single bit of the results: every SpMV row keeps its fma
 * chain in stored order (a row is never split across lanes) and every exact
 * dot is rounded once from the same integer sum.  What may change is speed,
 * and in plain mode the order in which the partial sums are added.  The
 * choices:
 *   staged       1: tiles whose SELL entries fit the shared-memory stage are
 *                copied there by bulk copies (default); 0: entries stream
 *                from global memory;
 *   order        tile order of a pass: 0 default (round-robin when staged,
 *                claimed otherwise), 1 round-robin, 2 claimed from a
 *                grid-wide counter in index order, 3 round-robin except the
 *                last two tiles of each CTA's share, which are claimed (the
 *                SMs that run ahead take over the tail);
 *   ctas_per_sm  resident CTAs per SM of the passes of pbcg_solve (0: as
 *                many as fit; else at most that many);
 *   batched_ctas_per_sm  the same for pbcg_solve_batched's passes (fewer
 *                CTAs: longer chunks of the tile list per CTA).
 * A variant belongs to a matrix and is used by every later solve of it
 * (pbcg_solve, pbcg_profile_solve, pbcg_solve_batched); pools and
 * partitioned solves keep the default.
 */
typedef struct {
    int32_t staged;
    int32_t order;
    int32_t ctas_per_sm;
    int32_t batched_ctas_per_sm;
    double us_per_iter;          /* pbcg_tune: measured time per iteration; ignored by pbcg_set_variant */
} pbcg_variant;

/* Set (v != NULL) or reset to the default (v == NULL) A's launch variant.
 * Errors: INVALID (unknown matrix, a field out of range). */
int pbcg_set_variant(pbcg_ctx *ctx, pbcg_mat *A, const pbcg_variant *v);

/* A's current launch variant (us_per_iter: the last tuned figure, or 0). */
int pbcg_get_variant(pbcg_ctx *ctx, const pbcg_mat *A, pbcg_variant *out);

/*
 * Autotune A's launch variant for algorithm alg and dot_mode: every
 * candidate variant runs trial solves (b = A * ones, x0 = 0, no stop) of
 * `iters` and 3 * iters iterations after an untimed one; its time per
 * iteration is the difference of the two (CUDA events on the context's
 * stream) over 2 * iters, so setup, the first iterations and the
 * true-residual check drop out.  The fastest becomes A's variant; the
 * default is always a candidate, so the choice is never slower than it as
 * measured.  1 <= iters <= 30000.  nsys = 0 tunes pbcg_solve's passes; nsys >= 1 with
 * sys_row_ptr[nsys+1] tunes pbcg_solve_batched's passes for that block
 * structure.  A system small enough for the one-cluster loop keeps the
 * default (its launch is fixed).
 * cache_path (may be NULL): a file of JSON lines, one per tuned key
 * {"key": "...", "staged": s, "order": o, "ctas_per_sm": c,
 *  "batched_ctas_per_sm": b, "us_per_iter": t}; the key is made of n, nnz,
 * a hash of the row-length histogram (and of sys_row_ptr), alg, dot_mode and
 * the SM count.  A key found there is applied without timing; a new one is
 * appended.  chosen (may be NULL) receives the variant applied; tried (cap
 * entries, may be NULL) the candidates with their times, *ntried (may be
 * NULL) how many ran (0 when the cache answered).
 * Errors: INVALID (bad arguments, iters outside 1 .. 30000), OOM, CUDA, or
 * a trial's error.
 */
int pbcg_tune(pbcg_ctx *ctx, pbcg_mat *A, int alg, int dot_mode, int32_t nsys, const int32_t *sys_row_ptr,
              int32_t iters, const char *cache_path, pbcg_variant *chosen, pbcg_variant *tried, int32_t cap,
              int32_t *ntried);

/*
 * Memory-safety checks (compute-sanitizer is not available on the target
 * machines, so the library checks itself).
 *
 * pbcg_mat_check (every build): validate A's device layout with a read-only
 * kernel -- slice offsets non-decreasing in whole 32-entry columns, every row
 * no longer than its slice, every stored column inside the gathered vector,
 * every tile record matching the slice offsets with its gather blocks inside
 * the vector, every staged local index naming its entry's column.  *word
 * receives 0, or the first failure as kind << 56 | position (kinds: 1
 * column, 2 local index, 3 row length, 4 slice offsets, 5 gather block, 6
 * tile record).
 *
 * The checked build (libpbcg_checked.so, compiled with PBCG_CHECKS=1) also
 * checks, inside every kernel, each index it takes from the layout, a tile
 * record or a tile list before using it (a column, a staged local index, a
 * row length, a slice's span in its stage, a gather block, a tile, a tile's
 * system, a cluster CTA's entry count); a failure is recorded in a device
 * word and the access skipped, never trapped.  pbcg_check_word reads that
 * word (*enabled = 1 in the checked build, 0 otherwise, when *word is always
 * 0; same kinds as above, plus 7 system and 8 cluster) and clears it when
 * reset != 0.  pbcg_debug_set_col (checked build only; INVALID otherwise)
 * overwrites stored column `entry` of A's device layout, so that a test can
 * see the checks fire.
 * Errors: INVALID (unknown matrix, NULL output), CUDA.
 */
int pbcg_mat_check(pbcg_ctx *ctx, const pbcg_mat *A, uint64_t *word);
int pbcg_check_word(pbcg_ctx *ctx, int reset, int32_t *enabled, uint64_t *word);
int pbcg_debug_set_col(pbcg_ctx *ctx, pbcg_mat *A, int64_t entry, int32_t col);

/*
 * pbcg_dot_noalloc: the dot product of pbcg_dot for callers that cannot
 * allocate device memory (code inside another allocator's arena, a fixed or
 * capped memory budget, or a loop that must not enter the allocator, since
 * cudaMalloc and cudaFree can synchronise the device).  It needs no context
 * and calls no cudaMalloc, cudaFree or other allocating routine.  The paper
 * has no counterpart: it is a packaging of the exact dot for such callers.
 *
 * a, b: n doubles each, device pointers on the current device; out: one
 * double in device memory, written with the result ((a,b) in dot_mode; exact
 * mode: correctly rounded, NaN if an operand is NaN or Inf).  cuda_stream: the
 * stream to launch on (NULL: the legacy default stream).  The call is
 * asynchronous; the result is ready when the stream reaches it.
 *
 * Scratch: the grid-wide merge state lives in one file-scope device array of
 * 70,144 bytes that every GPU loading this library holds until the process
 * exits.  Every call on a device shares it and clears it first; calls that
 * overlap on the GPU (other streams, other host threads) race on it and give
 * wrong results, so serialise them.  Every call looks up the array's device
 * address (cudaGetSymbolAddress, which allocates nothing) with the current
 * device; the first call on a device also reads the occupancy of its
 * kernels.  Make that first call before any stream capture.
 *
 * Limits: 0 <= n <= 2^31 - 1 (INVALID beyond); at most 2048 CTAs per call.
 * Errors: INVALID (bad size, NULL pointer, unknown dot_mode, or a, b or out
 * not device memory of the current device, as cudaPointerGetAttributes
 * reports it; nothing is launched then), CUDA.
 */
int pbcg_dot_noalloc(int64_t n, const double *a, const double *b, int dot_mode, double *out, void *cuda_stream);

/*
 * Row-partitioned solves (Section 2: the method runs on distributed memory,
 * each process owning a block of rows, with the dot products as global
 * reductions; Tables 2 and 3: with ExBLAS dots the iteration counts do not
 * change with the number of processes).
 *
 * Each of nranks ranks (one GPU, or one context, each) owns the contiguous
 * global rows [row_starts[rank], row_starts[rank+1]) of A, b and x.  Before a
 * pass whose SpMV gathers a vector, the entries of it that the rank's columns
 * need from other ranks (the halo) are exchanged; at every reduction point
 * each rank forms its share of the dots (exact mode: the integer digits of
 * its long accumulator; plain mode: its partial sums), the shares are added
 * over the ranks by one collective, and every rank rounds the same total
 * once.  Exact-mode results -- residual history, iteration count, status and
 * every rank's block of x -- are therefore bit-identical to pbcg_solve of the
 * whole system whatever nranks and row_starts are.  Plain mode adds the
 * ranks' partial sums in rank order: deterministic for a given partition,
 * not across partitions.
 *
 * The library does not talk to other ranks itself: the caller supplies the
 * two collectives, on host memory, over any transport (MPI, NCCL, gloo, ...).
 * Every rank must make the same sequence of calls; each callback returns 0,
 * or nonzero to fail the calling entry point with PBCG_ERR_COMM.
 *   allreduce_sum_i64: buf[0 .. count-1] := the sum over all ranks of every
 *     rank's buf (two's complement int64 addition, in place);
 *   alltoallv: rank r sends the send_bytes[k] bytes at send + send_displs[k]
 *     to rank k and receives recv_bytes[k] bytes from rank k at
 *     recv + recv_displs[k] (byte counts and offsets; zero counts allowed).
 * A rank that fails leaves the others waiting in their next collective until
 * the transport's own timeout ends it; arguments are checked on every rank
 * and agreed with one allreduce before any other exchange, so bad arguments
 * fail on all ranks together.
 */
typedef struct {
    void *user;
    int (*allreduce_sum_i64)(void *user, int64_t *buf, int64_t count);
    int (*alltoallv)(void *user, const void *send, const int64_t *send_bytes, const int64_t *send_displs,
                     void *recv, const int64_t *recv_bytes, const int64_t *recv_displs);
} pbcg_comm;

typedef struct pbcg_part pbcg_part;   /* opaque, library-owned: one rank's block */

/*
 * The halo of one rank's row block, on the host only (no CUDA call): the
 * global columns outside [row_starts[rank], row_starts[rank+1]) that the
 * block's rows reference, sorted ascending (so grouped by owning rank), and
 * for every rank k the number of them that rank k owns.  row_ptr[nloc+1],
 * col_idx[nnz] hold the block in CSR with global column indices.
 * halo_cols (capacity cap, may be NULL), recv_counts[nranks] (may be NULL)
 * and local_col[nnz] (may be NULL) receive the halo, the counts and each
 * entry's column in the rank's local numbering (own columns c - row0, halo
 * column h at nloc + h); *nhalo gets the halo's length (which may exceed cap).
 * Validation (INVALID): 1 <= nranks, 0 <= rank < nranks, row_starts[0] == 0,
 * row_starts non-decreasing, the rank's block non-empty, row_ptr[0] == 0,
 * non-decreasing, row_ptr[nloc] == nnz, 0 <= col_idx < row_starts[nranks].
 */
int pbcg_part_plan(int32_t nranks, int32_t rank, const int32_t *row_starts, int64_t nnz, const int32_t *row_ptr,
                   const int32_t *col_idx, int32_t *nhalo, int32_t *halo_cols, int32_t cap, int32_t *recv_counts,
                   int32_t *local_col);

/*
 * Create this rank's block on ctx's device (collective: every rank calls it
 * with the same nranks and row_starts).  row_ptr, col_idx (global column
 * indices) and vals describe the block's rows as for pbcg_part_plan; host or
 * device pointers; the library copies them.  One alltoallv tells every rank
 * which of its entries the others gather.  The block must be destroyed before
 * ctx.  Errors: INVALID (validation as for pbcg_part_plan, on any rank, or a
 * halo request outside the receiving rank's rows), OOM, CUDA, COMM.
 */
int pbcg_part_create(pbcg_ctx *ctx, const pbcg_comm *comm, int32_t nranks, int32_t rank, const int32_t *row_starts,
                     int64_t nnz, const int32_t *row_ptr, const int32_t *col_idx, const double *vals,
                     pbcg_part **out);

/*
 * Solve A x = b over all ranks (collective).  b and x hold this rank's block
 * (row_starts[rank+1] - row_starts[rank] doubles, host or device; x: x_0 in,
 * the block of the last iterate out).  tol, maxit, dot_mode and the stopping
 * rule as for pbcg_solve; alg: PBCG_ALG_BICGSTAB or PBCG_ALG_PIPELINED (no
 * residual replacement or preconditioner).  Launches are driven from the
 * host, one pass at a time.  The residual history goes to the block's
 * context (pbcg_residual_history with sys = 0).  Returns the status (the
 * same on every rank) or an error.
 */
int pbcg_part_solve(pbcg_part *part, const double *b, double *x, double tol, int32_t maxit, int alg, int dot_mode,
                    pbcg_result *out);

/* Free a block (not collective).  destroy(NULL) is a no-op. */
void pbcg_part_destroy(pbcg_part *part);

#ifdef __cplusplus
}
#endif

#endif /* PBCG_H */
