/*
 * rbicg.h -- C ABI of the GB300 recycling-BiCG library (librbicg.so).
 *
 * Method: Ahuja, de Sturler, Gugercin, Chang, "Recycling BiCG with an application to model
 * reduction" (arXiv:1010.0762).  The library solves a sequence of slowly changing dual
 * sparse systems (Section 1, eq. (initialSys))
 *
 *        A^(j) x^(j) = b^(j),        A^(j)^H xt^(j) = bt^(j),        j = 1, 2, ...
 *
 * with RBiCG (Algorithm 2), carrying a recycle space U, Ut from one pair to the next and
 * refreshing it every s iterations from harmonic Ritz vectors (Section 4).
 *
 * Conventions shared by every entry point:
 *  - All vector / matrix pointers are DEVICE pointers unless a name ends in _host.  The
 *    caller owns them; the library never frees or retains them past the call, except the
 *    matrix handed to rbicg_update_recycle / rbicg_solve_pair, which must stay valid and
 *    unchanged until the next call that passes a matrix (the library reads it during each
 *    solve).
 *  - Real values are IEEE double (or float where a name says f32); complex values are two
 *    doubles (re, im) interleaved.
 *  - CSR matrices use int32 row_ptr[n+1] and col_idx[nnz] with row_ptr[0] = 0, row_ptr[n] =
 *    nnz, and strictly increasing column indices within each row (checked on the device;
 *    RBICG_ERR_ARG otherwise).
 *  - Inner product (a, b) = a^H b (the paper's "standard inner product", Section 1).
 *  - A handle is bound to one CUDA stream given at creation; all work is queued on it.
 *    A handle is not thread-safe.  Calls block until their result is on the host.
 *  - Return value: RBICG_OK (0); a positive status when the solve ended without meeting
 *    the tolerance (x then holds the last iterate); a negative status for an error, in
 *    which case outputs are unspecified and rbicg_last_error() describes it.  No call
 *    traps, aborts or exits; device-side waits are bounded.
 *  - Environment switches (read when first needed; none changes any result):
 *    RBICG_NO_GRAPHS: launch each cycle's iteration kernels one by one instead of as a CUDA
 *    graph (profilers then see and select the individual kernels); RBICG_NO_PDL: launch the
 *    iteration kernels without programmatic stream serialization; RBICG_NO_STAGE: the
 *    dual-SpMV kernel forms each gathered r_j + beta p_j on the fly instead of staging p with
 *    its bandwidth halo in shared memory; RBICG_DEBUG: print one line per solve on stderr.
 */
#ifndef RBICG_H
#define RBICG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RBICG_OK = 0,
  RBICG_NOT_CONVERGED = 1,   /* max_itn reached (Algorithm 2 step 5 bound) */
  RBICG_BREAKDOWN_RHO = 2,   /* |(rt_i, r_i)| <= 1e-14 ||rt_i|| ||r_i|| (Section 2, serious breakdown) */
  RBICG_BREAKDOWN_PQ = 3,    /* |(pt_i, q_i)| <= 1e-14 ||pt_i|| ||q_i|| (Section 2, second kind) */
  RBICG_RECYCLE_EMPTY = 4,   /* solve converged, but the system start's Section 4.3 truncation
                                left p = 0 columns of the recycle space carried in */
  RBICG_ERR_ARG = -1,        /* invalid argument (sizes, null pointers, malformed CSR) */
  RBICG_ERR_OOM = -2,        /* device allocation failed */
  RBICG_ERR_CUDA = -3,       /* a CUDA call failed */
  RBICG_ERR_TIMEOUT = -4,    /* a bounded device-side wait gave up */
  RBICG_ERR_NONFINITE = -5,  /* a non-finite scalar appeared in the iteration */
  RBICG_ERR_EIG = -6         /* the small dense eigen / SVD solve did not converge */
} rbicg_status;

typedef enum {
  RBICG_R64 = 0,   /* real double vectors and operator */
  RBICG_C128 = 1   /* complex double vectors (operator real or complex, see rbicg_csr) */
} rbicg_dtype;

typedef enum {
  RBICG_FP64 = 0,          /* every step in the vector dtype (FP64) */
  RBICG_FP32_REFINED = 1   /* FP64 iterative refinement around FP32 inner RBiCG solves.  If an
                              inner solve fails twice in a row (no residual reduction, even
                              without a recycle space; an inner residual above 1e6 ||b||; or
                              no new residual minimum for max(1000, 25 s) iterations),
                              the handle continues the refinement of this and later pairs with
                              FP64 RBiCG correction solves (A d = r from d = 0, to the relative
                              tolerance that brings r to tol, at least 1e-13), which reach tol
                              in the FP64 true residual where one FP64 solve of the whole system
                              can stop short of it (rbicg_result.fallback = 2), until
                              rbicg_reset */
} rbicg_precision;

/* Solver parameters.  Defaults (rbicg_default_params): k = 10, s = 40, max_itn = 20000,
 * tol = 1e-8, svd_tol = 1e-6, inner_tol = 1e-5, refine_max = 12, precision = FP64,
 * seed = 0, setup_fp32 = 1, recycle = 1, inner_svd_tol = 1e-3, guard = 1.5, restarts = 0,
 * grid_blocks = 0, refresh = 1, setup_blocks = 0, graphs = 1. */
typedef struct {
  int k;                   /* recycle dimension: columns kept in U, Ut (Section 3, 4.1); 1..32 */
  int s;                   /* cycle length (Section 4.1); 2..64, k + s <= 80 */
  int max_itn;             /* iteration bound of Algorithm 2 step 5 (per inner solve) */
  double tol;              /* relative residual: ||r|| <= tol ||b|| and ||rt|| <= tol ||bt|| */
  double svd_tol;          /* truncation of Section 4.3 after unit-norm column scaling */
  double inner_tol;        /* FP32_REFINED: relative tolerance of each inner solve */
  int refine_max;          /* FP32_REFINED: bound on outer refinement steps */
  rbicg_precision precision;
  uint64_t seed;           /* Philox4x32-10 key for the random restart of Algorithm 2 step 3 */
  int setup_fp32;          /* 1: per-cycle O(n) Gram / basis products in FP32 arithmetic on
                              the stored data (FP64 accumulation across row blocks); 0: FP64 */
  int recycle;             /* 0: plain BiCG (no recycle space computed or used) */
  double inner_svd_tol;    /* FP32_REFINED: Section 4.3 truncation used by the FP32 inner solver.
                              The oblique projector C D_c^{-1} Ct^H has norm about 1/sigma_min,
                              and FP32 rounding in q = z - C zeta grows by that factor, so the
                              FP32 solver keeps only sigma >= max(svd_tol, inner_svd_tol) */
  double guard;            /* stagnation guard (not in the paper): a pair solved with a recycle
                              space that has not converged after guard x (iterations of the last
                              pair this handle solved from its start without one, every leg
                              counted) iterations applies step 7 to
                              its current iterate and continues from it as plain BiCG (Algorithm 2
                              with an empty recycle space); rbicg_result.fallback reports it.
                              0 disables the guard. */
  int restarts;            /* restarts after a BiCG breakdown (not in the paper; default 0: the
                              breakdown is reported): a pair whose recurrence breaks down (rho or
                              (pt, q) below 1e-14 of the norms) applies step 7 and continues from
                              its iterate as plain BiCG, at most this many times */
  int grid_blocks;         /* blocks of 256 threads per iteration-phase launch (0: the default,
                              min(ceil(n / 256), 2 x SMs) with recycling, whose cycle refresh runs
                              concurrently and needs room on the SMs, 3 x SMs without);
                              rbicg_autotune picks one by timed
                              trials.  Reductions follow the block partition, so results are
                              reproducible for a given value. */
  int refresh;             /* 1 (default): refresh the recycle space every s iterations and hand the
                              last one to the next pair (Section 4); 0: solve with the current
                              recycle space and carry it to the next pair unchanged (Section 6.2:
                              the recycle space may be recomputed only for some systems of a
                              sequence, e.g. every fifth IRKA step).  Changeable between pairs
                              with rbicg_set_refresh. */
  int setup_blocks;        /* blocks of the refresh's Gram products (0: the default, 8 x SMs);
                              rbicg_autotune_params picks one by timed trials */
  int graphs;              /* 1 (default): each cycle's iteration launches run as one CUDA graph;
                              0: launched one by one */
} rbicg_params;

/* A sparse operator.  Operator = A when has_shift == 0, (shift I - A) otherwise. */
typedef struct {
  int64_t n, nnz;
  const int32_t *row_ptr;  /* device, n+1 */
  const int32_t *col_idx;  /* device, nnz */
  const void *val;         /* device, nnz doubles (val_complex = 0) or complex doubles (1) */
  int val_complex;
  int has_shift;
  double shift_re, shift_im;
} rbicg_csr;

typedef struct {
  int iters;               /* iterations of the (last inner) solve; summed over inner solves */
  int cycles;              /* completed cycles (recycle-space refreshes) */
  int recycle_dim;         /* columns of the recycle space used for this pair (p of Section 4.3) */
  int refine_steps;        /* FP32_REFINED outer steps (0 for FP64) */
  double relres, relres_dual;             /* recurrence residuals, relative */
  double true_relres, true_relres_dual;   /* ||b - A x|| / ||b||, ||bt - A^H xt|| / ||bt|| in FP64 */
  int status;              /* rbicg_status of the solve */
  int fallback;            /* 1: the stagnation guard dropped the recycle space during the solve;
                              2: an FP32_REFINED handle solved the pair in FP64 */
} rbicg_result;

typedef struct rbicg_ctx *rbicg_handle;

/* Fill *p with the defaults listed above. */
void rbicg_default_params(rbicg_params *p);

/* Create a solver for systems of order n.  stream: a cudaStream_t (NULL = legacy default
 * stream).  Allocates the device workspace for n, params->k and params->s (Section 4.1:
 * recycle bases U, Ut, C, Ct, the per-cycle U_j, C_j and the residual ring).  Returns
 * RBICG_ERR_ARG for invalid sizes, RBICG_ERR_OOM if the workspace does not fit. */
rbicg_status rbicg_create(const rbicg_params *params, int64_t n, rbicg_dtype dtype,
                          void *stream, rbicg_handle *out);

/* Set the operator of the next pair and prepare the recycle space for it (Section 4.3, last
 * paragraph): C = A U, Ct = A^H Ut, SVD Ct^H C = M Sigma N^H after unit-norm column
 * scaling, keep sigma >= svd_tol (p columns), U <- U N_p, Ut <- Ut M_p, C <- C N_p,
 * Ct <- Ct M_p, D_c = Sigma_p.  Also builds the library's copy of A^H (same pattern with
 * conjugated transposed values when A is structurally symmetric, a transposed CSR
 * otherwise).  With no recycle space yet (first pair) only the operator is set. */
rbicg_status rbicg_update_recycle(rbicg_handle h, const rbicg_csr *A);

/* Solve one dual pair with Algorithm 2.  A: the operator, or NULL to reuse the one set by
 * the last rbicg_update_recycle / rbicg_solve_pair (a different A triggers an implicit
 * rbicg_update_recycle).  b, bt: right-hand sides (n values each).  x, xt: in = x_{-1},
 * xt_{-1} (initial guesses of eq. (minusXR)); out = the solutions (step 7).  bt may be all
 * zeros (the dual test is then skipped).  Every s iterations the recycle space for the next
 * pair is refreshed (Sections 4.1-4.3); if the pair converges in fewer than s iterations the
 * previous space is kept (Section 6.2).  res receives counters and residuals. */
rbicg_status rbicg_solve_pair(rbicg_handle h, const rbicg_csr *A, const void *b, const void *bt,
                              void *x, void *xt, rbicg_result *res);

/* Solve `count` (<= 32) independent dual pairs, one per handle, together on the first handle's
 * stream through a continuous-batching engine (below): each iteration phase is one launch for
 * all FP64 pairs; each handle keeps its own recycle space, stopping test and cycle refreshes.
 * Arrays are host arrays of length count holding the per-pair arguments of rbicg_solve_pair
 * (As[i] may be NULL to reuse the handle's operator).  Results are bit-identical to solving
 * each pair alone with rbicg_solve_pair.  A handle may appear only once. */
rbicg_status rbicg_solve_batch(rbicg_handle *hs, const rbicg_csr *const *As, const void *const *bs,
                               const void *const *bts, void *const *xs, void *const *xts, int count,
                               rbicg_result *res);

/* Continuous batching.  An engine advances the FP64 requests in flight by one cycle (s
 * iterations, Algorithm 2 step 5, plus each request's cycle refresh of Sections 4.1-4.3) per
 * rbicg_engine_step, with ONE launch per iteration phase for all of them; requests join at
 * submit time and leave when they finish, between steps.  Each request is one dual pair on its
 * own handle (at most one in flight per handle; at most 32 in flight), and its results are
 * bit-identical to rbicg_solve_pair on that handle: the batched launch gives every request its
 * own blocks, partial sums and reduction order.  FP32_REFINED requests step through the same
 * engine: their FP64 residual and correction steps run between engine steps and their inner
 * solves advance one cycle per step with the other requests.  The paper has no counterpart
 * (serving layer).  Buffers must stay valid until the
 * request is polled.  stream: the engine's cudaStream_t (NULL = legacy default stream); the
 * handles' own streams are used again once their requests finish. */
typedef struct rbicg_engine_s *rbicg_engine;
rbicg_status rbicg_engine_create(void *stream, rbicg_engine *out);
/* Start a request: operator update if A differs from the handle's (Section 4.3 system start),
 * initial projection (eq. (minusXR)); tag is returned by rbicg_engine_poll. */
rbicg_status rbicg_engine_submit(rbicg_engine e, rbicg_handle h, const rbicg_csr *A, const void *b,
                                 const void *bt, void *x, void *xt, int64_t tag);
/* One cycle for every request in flight; *in_flight receives the number still running. */
rbicg_status rbicg_engine_step(rbicg_engine e, int *in_flight);
/* Up to max finished requests (tags[i], res[i]); *count receives how many. */
rbicg_status rbicg_engine_poll(rbicg_engine e, int64_t *tags, rbicg_result *res, int max, int *count);
/* Finishes the requests in flight, then frees the engine. */
rbicg_status rbicg_engine_destroy(rbicg_engine e);

/* Autotuner (no counterpart in the paper).  Times the iteration phases of Algorithm 2 on the
 * operator A (plain iterations from a random start, tolerance 0, on a private stream) for the
 * candidate launch shapes {1, 2, 4, 8, 16} x SMs blocks (capped at ceil(n / 256)), keeps the
 * fastest in a process-wide cache keyed by (n, nnz, dtype, value type, k), and returns it in
 * *grid_blocks (with its time per iteration in *us_per_iter, which may be NULL).  A cached
 * shape is returned without new trials.  Set params->grid_blocks to use it. */
rbicg_status rbicg_autotune(const rbicg_params *params, rbicg_dtype dtype, const rbicg_csr *A, int trial_iters,
                            int *grid_blocks, double *us_per_iter);

/* Autotuner over three launch knobs (no counterpart in the paper): grid_blocks as rbicg_autotune
 * does; then, with that grid, setup_blocks in {4, 8, 12} x SMs and graphs in {1, 0}, each by timing
 * three cycles of recycled iterations with their refreshes (k, s from params, tolerance 0, on a
 * private stream, from a random start).  *out = *params with the three fields set to the fastest
 * (the grid from the cache when rbicg_autotune already tuned this shape); *us_per_iter (may be
 * NULL) the time per recycled iteration, refresh included. */
rbicg_status rbicg_autotune_params(const rbicg_params *params, rbicg_dtype dtype, const rbicg_csr *A,
                                   int trial_iters, rbicg_params *out, double *us_per_iter);

/* Copy the recycle space for the next pair into caller buffers U, Ut (device, n x k row-major,
 * k = params->k columns, unused columns zero); *p receives the number of valid columns. */
rbicg_status rbicg_export_recycle(rbicg_handle h, void *U, void *Ut, int *p);

/* Install a recycle space (device, n x p row-major, p <= k).  It is made bi-orthogonal for
 * the operator of the next rbicg_update_recycle / rbicg_solve_pair call. */
rbicg_status rbicg_import_recycle(rbicg_handle h, const void *U, const void *Ut, int p);

/* Drop the recycle space: the next pair is solved as a first system (Algorithm 2 step 1). */
rbicg_status rbicg_reset(rbicg_handle h);

/* Set rbicg_params.refresh (0 or 1) for the handle's next solves (Section 6.2: recompute the
 * recycle space only for selected systems of a sequence). */
rbicg_status rbicg_set_refresh(rbicg_handle h, int refresh);

/* Measurement hook (no counterpart in the paper): the recurrence residual norms ||r_m|| of the last
 * FP64 solve on this handle (Algorithm 2 step 5; m = 0 is the norm after eq. (minusXR)), for its
 * last *count = min(max, 132, iterations + 1) iterations in iteration order, out[*count - 1] being
 * the last iteration's.  The values come from the device's ring of scalar histories; a pair that
 * restarted (guard, restarts) reports its last leg. */
rbicg_status rbicg_residual_history(rbicg_handle h, double *out, int max, int *count);

/* Free the handle and its device workspace. */
rbicg_status rbicg_destroy(rbicg_handle h);

/* Message of the last error on this handle (never NULL; "" when none).  With h == NULL,
 * the last error of a call that had no valid handle. */
const char *rbicg_last_error(rbicg_handle h);

/* Number of kernel launches made through this handle since it was created (for timing
 * reports). */
int64_t rbicg_launch_count(rbicg_handle h);

/* Measurement hooks (no counterpart in the paper): device time of each step of the solve,
 * taken with CUDA events on the handle's stream.  enable = 1 starts collection (clearing the
 * accumulators), 2 starts it with every cycle refresh run alone (the refresh waits for the
 * iteration stream and the iteration stream for the refresh, so each step's time is its own,
 * not shared with the concurrent next cycle), 0 stops it, -1 only reads.  ms_out / launches_out (host arrays of
 * RBICG_NPROF, may be NULL) receive the accumulated milliseconds and kernel launches per
 * slot: 0 dual SpMV + projections (Algorithm 2 step 5, lines 1-3; without a recycle space
 * also (pt, q) and alpha), 1 q and (pt, q) (iterations with a recycle space only),
 * 2 x / r updates and (rt, r), 3 refresh Gram (Section 4.1), 4 refresh eigen solve
 * (eq. (finalGenEigValue)), 5 refresh basis update and SVD (Section 4.3), 6 system start
 * (Section 4.3 last paragraph), 7 initial projection / step 7 / A^H construction. */
#define RBICG_NPROF 8
rbicg_status rbicg_profile(rbicg_handle h, int enable, double *ms_out, int64_t *launches_out);
/* With profiling on: the projection width (columns of C, Ct) summed over the slot-0 launches,
 * so that their algorithmic work (2 SpMVs and 2 k-column projections each) can be counted. */
rbicg_status rbicg_profile_columns(rbicg_handle h, int64_t *cols);
/* With profiling on: the column pairs mx x my summed over the slot-3 launches (the Gram
 * Psit^H [Psi U_{j-1}] of Section 4.1), so that their algorithmic work, mx my n multiply-adds
 * each, can be counted. */
rbicg_status rbicg_profile_gram_pairs(rbicg_handle h, int64_t *pairs);

/* ---------------------------------------------------------------------------------------
 * Component entry points.  Each runs one step of the hot path on caller-provided device
 * buffers, synchronously on `stream`, so that the step can be checked or used on its own.
 * ------------------------------------------------------------------------------------- */

/* Algorithm 2 step 5, first two lines: p = r + beta p_old, pt = rt + conj(beta) pt_old,
 * z = Op p, zt = Op^H pt (Op = A or shift I - A), and the projections
 * zeta = D_c^{-1} Ct^H z, zetat = D_c^{-1} C^H zt (eq. (CcheckChat): zeta = Chat^H z,
 * zetat = Ccheck^H zt).  C, Ct: n x k row-major (ldc >= k) or NULL with k = 0; Dc: k
 * doubles (host).  beta: (re, im) on the host.  zeta_host, zetat_host: k values each
 * (complex when dtype is C128) written on the host.  p_out, pt_out, z, zt: n values. */
rbicg_status rbicg_op_dual_spmv_project(const rbicg_csr *A, rbicg_dtype dtype, const void *r,
                                        const void *rt, const void *p_old, const void *pt_old,
                                        double beta_re, double beta_im, const void *C,
                                        const void *Ct, int k, int ldc, const double *Dc_host,
                                        void *p_out, void *pt_out, void *z, void *zt,
                                        void *zeta_host, void *zetat_host, void *stream);

/* Tall-skinny Gram G = X^H Y (Section 4.1 Grams Psit^H Psi, Psit^H Phi; Section 4.3
 * Ct^H C).  X: n x mx, Y: n x my, both row-major with leading dimensions ldx, ldy; G_host:
 * mx x my row-major on the host (complex when dtype is C128).  fp32: 1 to multiply in FP32
 * (FP64 accumulation across row blocks), 0 for FP64. */
rbicg_status rbicg_op_gram(rbicg_dtype dtype, int64_t n, const void *X, int mx, int ldx,
                           const void *Y, int my, int ldy, int fp32, void *G_host, void *stream);

/* Generalised eigenproblem L w = lambda R w of eq. (finalGenEigValue), order m <= 80, in
 * FP64 on one thread block: selects the k eigenvalues closest to the origin (a conjugate
 * pair of a real problem is kept together as real and imaginary parts, k-1 columns if the
 * pair straddles the cut) and returns the right eigenvectors W (m x kk) and the matching
 * left eigenvectors Wt (m x kk), column-major on the host, and the eigenvalues (complex,
 * kk).  L, R: m x m column-major on the host.  R = NULL means the standard problem L w =
 * lambda w (Section 4.2, first cycle).  *kk receives the number of columns. */
rbicg_status rbicg_op_eig_select(rbicg_dtype dtype, int m, const void *L_host, const void *R_host,
                                 int k, void *W_host, void *Wt_host, double *lam_host, int *kk,
                                 void *stream);

/* SVD S = M Sigma N^H of a k x k matrix (Section 4.3, eq. (equationSVD)) in FP64 on one
 * thread block (one-sided Jacobi).  S, M, N: column-major on the host; sigma: k values in
 * descending order. */
rbicg_status rbicg_op_svd(rbicg_dtype dtype, int k, const void *S_host, void *M_host, double *sigma,
                          void *N_host, void *stream);

/* Allocation-free variant of rbicg_op_gram (the paper has no counterpart): G = X^H Y with X
 * n x mx, Y n x my (row-major, leading dimensions ldx, ldy) and G an mx x my row-major DEVICE
 * output (doubles, or complex doubles for C128), computed on `stream` without allocating any
 * device memory.  It serves callers that must not allocate behind their back: a runtime that
 * reserves the device memory up front and forbids hidden allocations, or a latency-critical
 * caller that cannot afford cudaMalloc / cudaFree and the synchronisation they imply.
 * Limits: 1 <= mx, my <= 64 (larger sizes return RBICG_ERR_ARG).  The partial sums live in one
 * fixed 8 MiB device array inside the library, which every GPU that loads the library holds
 * until the process exits.  The first call on a device looks up that array's device address
 * (once per device, with the device current); make that first call before any stream capture.
 * All calls share the array and each call overwrites it, so calls that overlap on the GPU
 * (on different streams or from different threads) race; serialise them.  The call returns
 * once the work is queued; synchronise `stream` before reading G. */
rbicg_status rbicg_op_gram_noalloc(rbicg_dtype dtype, int64_t n, const void *X, int mx, int ldx,
                                   const void *Y, int my, int ldy, int fp32, void *G, void *stream);

/* ---------------------------------------------------------------------------------------
 * Applications built on solved dual pairs.
 * ------------------------------------------------------------------------------------- */

/* Bilinear form u^H Op^{-1} w from a solved dual pair (Section 1: bilinear forms u^* A^{-1} w,
 * e.g. in QMC, are evaluated from the primal and the dual system, with an error bound that is
 * quadratic in the residuals).  x solves Op x = w and xt solves Op^H xt = u (for example
 * rbicg_solve_pair with b = w, bt = u); Op = A or (shift I - A) as in rbicg_csr.  u, w, x, xt:
 * n device values of the dtype.  out_host receives three complex values (re, im interleaved; the
 * imaginary parts are 0 for R64): u^H x, xt^H w, and the corrected estimate
 * u^H x + xt^H (w - Op x), whose error u^H Op^{-1} w - estimate equals
 * (u - Op^H xt)^H Op^{-1} (w - Op x).  Sums are taken in FP64 in a fixed order (reproducible).
 * Synchronous on `stream`; allocates a small device buffer for the block partial sums. */
rbicg_status rbicg_bilinear_form(const rbicg_csr *A, rbicg_dtype dtype, const void *u, const void *w,
                                 const void *x, const void *xt, double *out_host, void *stream);

/* IRKA (Algorithm 3, Section 5) for the SISO system G(s) = c^H (s I - A)^{-1} b with E = I:
 * dual shifted systems (sigma_i I - A) v_i = b, (sigma_i I - A)^H w_i = c solved with RBiCG,
 * reduced model E_r = W^H V, A_r = W^H A V, b_r = W^H b, c_r = V^H c (eq. (red_projection); the
 * algorithm's listing prints W^H A V for E_r and V^H c_r for c_r), new shifts
 * sigma_i <- -lambda_i(A_r, E_r) until they stop moving.  Shifts are kept in ascending modulus
 * (the larger imaginary part first among equal moduli), and for real A, b, c the new set is made
 * exactly closed under conjugation (rounding removed).  Recycling (Section 5.3): */
typedef struct {
  int r;               /* reduced order = number of shifts, 1..32 */
  int max_steps;       /* bound on IRKA steps (reduced models formed) */
  double shift_tol;    /* converged when max_i |sigma_i' - sigma_i| / |sigma_i| < shift_tol (the
                          paper's experiments: 1e-6) */
  int strategy;        /* 0: no recycling (BiCG); 1: shift index i recycles from index i of the
                          previous step; 2: each solve recycles from the previous shift's solve
                          (within a step, and from the last shift of a step to the first of the
                          next); 3: the space of the pooled system (previous step's shifts and this
                          step's earlier ones) with the smallest relative shift change, if below
                          pool_tol, else none; 4: one recycle space shared by all shifts (E = I:
                          sigma I - A has A's eigenvectors, Section 5.3), computed by the solve of
                          the smallest shift and used by every shift in the next step, so one
                          refresh chain runs per step instead of r */
  int recycle_count;   /* recycle only for the recycle_count shifts of smallest modulus (0: all;
                          Section 6.2 recycles for the small shifts only) */
  int refresh_every;   /* compute new recycle spaces only on steps m with m % refresh_every == 0,
                          else solve with the carried spaces (Section 6.2: every fifth step) */
  double pool_tol;     /* strategy 3 threshold on the relative shift change */
  int batched;         /* strategies 0, 1 and 4: the r solves of a step in one rbicg_solve_batch */
  int conj_pairs;      /* 1: of each conjugate pair of shifts only the one with positive imaginary
                          part is solved; the other's v and w are the complex conjugates (exact for
                          real A, b, c), reported with 0 iterations; 0: every shift is solved */
} rbicg_irka_params;

typedef struct {
  int steps;               /* reduced models formed */
  int converged;           /* 1 if the shift change fell below shift_tol */
  double last_change;      /* max relative shift change of the last step */
  int64_t iters;           /* iterations summed over all solves (primal and dual pair counted once) */
  int failed_solves;       /* solves that ended with a status other than OK / RECYCLE_EMPTY */
  double model_shifts[64]; /* the r shifts (re, im) the returned reduced model interpolates at */
} rbicg_irka_result;

/* Fill *p with the defaults: r = 8, max_steps = 10, shift_tol = 1e-6, strategy = 1,
 * recycle_count = 0, refresh_every = 1, pool_tol = 0.5, batched = 1, conj_pairs = 1. */
void rbicg_irka_default_params(rbicg_irka_params *p);

/* Run IRKA.  sp: the RBiCG parameters of every solve (complex double vectors, C128).  A: the real
 * system matrix (val_complex = 0, has_shift = 0), device CSR.  b, c: n doubles each (device).
 * shifts_in: r initial shifts (re, im) on the host.  On return: shifts_out (host, r complex) the
 * shifts after the last step; Ar_out, Er_out (host, r x r complex, column-major) and br_out,
 * cr_out (host, r complex) the reduced model of the last step, which interpolates G at
 * res->model_shifts; iters_out (host, max_steps x r ints, may be NULL) the iterations of every
 * solve, step-major.  The output pointers other than shifts_out may be NULL.  Work runs on
 * `stream`; device memory for V, W, A V and the recycle pools is allocated and freed inside.
 * Returns a negative status on error (a failed solve is not an error: res->failed_solves counts
 * them), RBICG_ERR_EIG if the reduced pencil's eigenvalues could not be computed. */
rbicg_status rbicg_irka(const rbicg_params *sp, const rbicg_irka_params *ip, const rbicg_csr *A,
                        const double *b, const double *c, const double *shifts_in, void *stream,
                        double *shifts_out, double *Ar_out, double *Er_out, double *br_out, double *cr_out,
                        int *iters_out, rbicg_irka_result *res);

#ifdef __cplusplus
}
#endif

#endif /* RBICG_H */
