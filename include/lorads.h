/*
 * lorads.h - C ABI of the GB300 (sm_103a) LoRADS hot path.
 *
 * Problem (Eq. (1.1) of arXiv 2407.15049):
 *     min <C, X>  s.t.  <A_k, X> = b_k (k = 0..m-1),  X positive semidefinite,
 * solved through the Burer-Monteiro factorisation X = R R^T (Sec. 1, Sec. 2.1):
 * an augmented-Lagrangian outer loop, the L-BFGS inner solver of Algorithm 1,
 * the exact quartic line search of App. A.2 and the dynamic rank rule of
 * App. A.1.
 *
 * Sign convention.  y is the standard dual multiplier (y = -lambda of the
 * paper's Eq. (1.2)):
 *     L_rho(R, y) = <C, RR^T> - y^T (A(RR^T) - b) + rho/2 ||A(RR^T) - b||^2,
 *     grad_R L    = 2 (C - A*(y~)) R  with  y~ = y - rho (A(RR^T) - b),
 * and the multiplier step of Sec. 2.1 is y <- y~.  The error measures of
 * Sec. 4.2 (err1, err2, err3) are written with the dual slack C - A*(y).
 *
 * Constraint convention (SDPA-style triplets).  Constraint k is the sum of
 * its triplets (i <= j, a), each contributing a X_ii (i == j) or 2 a X_ij
 * (i < j) to <A_k, X>.  One triplet per constraint covers the MaxCut SDP of
 * Sec. 4.3 (X_ii = 1) and the matrix-completion SDP of Sec. 4.4.  Constraints
 * with several triplets, and several constraints on one entry (the general
 * sparse SDPs of Sec. 4.5), are accepted by lorads_create and every
 * single-instance entry point except lorads_admm_operator, which returns
 * LORADS_ERR_UNSUPPORTED for them; the batched solve and
 * lorads_linesearch_coeffs_noalloc take one triplet per constraint.
 *
 * Layout.  Every n x r factor (R, D, U, V, outputs) is row-major with a
 * leading dimension `ld` (elements): element (i, c) lives at p[i*ld + c].
 * `ld` must be a multiple of 4 (at most 512), and every device pointer must be
 * 16-byte aligned.  The kernels process all `ld` columns; the caller keeps
 * columns r..ld-1 at zero (they stay zero: C*0 = 0), `r` is informational.
 *
 * Precision (argument `prec`): LORADS_FP64 - double in, double out;
 * LORADS_FP32 - float in, float out (products in FP32, reductions in FP64);
 * LORADS_BF16 - bfloat16 in, float out.  Scalars and multipliers are double.
 *
 * Streams and ownership.  lorads_create copies every host input to device
 * memory owned by the context and allocates all scratch space; the caller may
 * free its buffers when it returns.  All entry points run on the context's
 * CUDA stream (the one given to lorads_create; NULL = legacy default stream).
 * Entry points taking device pointers do not allocate; pointers stay owned by
 * the caller and must stay valid until the stream has finished the call.
 *
 * Errors.  Every call returns a status; nothing throws or exits.  The message
 * of the last failure is available from lorads_last_error (per context, not
 * thread-safe).  A CUDA failure returns LORADS_ERR_CUDA; after a sticky CUDA
 * error the context is unusable and should be destroyed.
 */
#ifndef LORADS_H
#define LORADS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lorads_ctx lorads_ctx;

typedef enum {
    LORADS_OK = 0,
    LORADS_ERR_INVALID_ARG = 1,   /* bad size, pointer, index, layout or non-finite value */
    LORADS_ERR_NOT_SYMMETRIC = 2, /* C is not a symmetric CSR matrix */
    LORADS_ERR_OOM = 3,           /* device or host allocation failed */
    LORADS_ERR_CUDA = 4,          /* a CUDA runtime call failed */
    LORADS_ERR_NUMERIC = 5,       /* NaN/Inf reached the iteration */
    LORADS_ERR_MAXITER = 6,       /* max_outer reached before the tolerance */
    LORADS_ERR_TIMEOUT = 7,       /* time_limit reached */
    LORADS_ERR_UNSUPPORTED = 8    /* valid input outside what this library implements */
} lorads_status;

typedef enum {
    LORADS_FP64 = 0,
    LORADS_FP32 = 1,
    LORADS_BF16 = 2,
    LORADS_MIXED = 3,  /* solve only: double-float R and C*R, FP32 direction/gradient/history */
    LORADS_DF64 = 4,   /* solve only: double-float (hi, lo float pairs, ~48-bit) everywhere */
    LORADS_MIXED_BF16 = 5  /* solve only: MIXED with the search direction D and the stored L-BFGS pairs
                              in bf16 (each rounded once when formed; the C D product, line search and
                              step use the rounded direction, the Gram dots and the two-loop recursion
                              the rounded pairs); the gradient and C D stay FP32 */
} lorads_prec;

/* Solver constants.  The paper fixes tol (Sec. 4.2), the time limit (Sec. 4.2)
 * and the rank rule (App. A.1); the remaining values are this library's
 * readings of what the paper leaves open.  lorads_create and lorads_batch_create
 * refuse (LORADS_ERR_INVALID_ARG, message naming the field): tol not finite and
 * > 0; time_limit not > 0; lbfgs_mem outside [1, 4]; max_inner, max_outer,
 * rank_update_threshold or lanczos_steps below 1; rho0 not finite; rho_growth
 * not finite and >= 1; rho_max not > 0; infeas_decrease not finite and >= 0;
 * inner_rel or inner_progress not finite and > 0; lbfgs_scaling outside {0, 1};
 * rho_policy or inner_scale outside {0, 1, 2}; admm_switch < 0; cg_rel outside
 * (0, 1); cg_max < 1; admm_max_iter < 0; reopt_level outside [0, 2];
 * max_reopt < 0; reopt_factor outside (0, 1). */
typedef struct {
    double  tol;               /* 1e-5: err1 (1+||b||_inf normalisation) and |err3| */
    double  time_limit;        /* seconds, 1e4 */
    int32_t lbfgs_mem;         /* T of Algorithm 1, 1..4 (default 4) */
    int32_t max_inner;         /* K of Algorithm 1 per outer step (default 500) */
    int32_t max_outer;         /* default 200 */
    int32_t rank_update_threshold; /* outer steps in a row hitting max_inner before r grows (3) */
    double  rho0;              /* <= 0: 1 / mean |C_ij| over the stored entries */
    double  rho_growth;        /* 2 */
    double  rho_max;           /* 1e12 */
    double  infeas_decrease;   /* 0.25: rho grows unless err1 shrank by this factor */
    double  inner_rel;         /* 1.0: scale of the inner stopping threshold (see inner_scale) */
    double  inner_progress;    /* 0.1: inner_scale 2 also stops once ||G|| <= inner_progress ||G at loop start|| */
    int32_t prec;              /* lorads_prec of the solve: FP64, MIXED, DF64, FP32 or MIXED_BF16 */
    int32_t check_every;       /* iterations between host polls of the device status (16) */
    uint64_t seed;             /* seed of the rank-update columns (SplitMix64 + Box-Muller) */
    int32_t compute_err2;      /* 1: evaluate err2 (Lanczos on C - A*(y)) at the end */
    int32_t lanczos_steps;     /* Krylov dimension of that Lanczos run (default 200) */
    int32_t verbose;           /* 1: progress line per outer step on stderr; 2: per-kernel CUDA-event timing */
    int32_t reserved;
    int32_t lbfgs_scaling;     /* 0: initial matrix I (Algorithm 1 as printed); 1 (default): gamma I, gamma = <s,y>/<y,y> */
    int32_t rho_policy;        /* rho grows when err1 did not shrink by infeas_decrease: 0 always; 1 only
                                  after a converged inner loop; 2 (default) also after a capped loop that raised err1 */
    int32_t kernel_variant;    /* kernel forms, bit flags (bit 0 unused): bits 1, 2: the register-staged step
                                  update with 1 or 2 more resident blocks per SM (bit 1: one more block,
                                  measured 16% faster at n = 1e7); bit 3: the line-search SpMM loads each row
                                  group's next row bounds one iteration ahead and prefetches that row's
                                  entries, rows and scalars into L2 (measured 6% faster at n = 1e7); bit 4:
                                  the step update (with bit 1 or 2) prefetches each group's next row into L2
                                  (measured 1% slower); bit 5: the line-search SpMM with the fewest lanes
                                  per row that leaves none idle (ld = 24: 2 lanes x 3 units, 16 rows per
                                  warp; measured 2.6% slower at n = 1e7); bit 6 (with bit 3): the
                                  line-search SpMM loads row bounds two rows ahead and prefetches one
                                  neighbour row of the next row per lane into L2; bit 7 (with bit 1): the
                                  step update in packed row groups of ld/4 lanes where that keeps more lanes
                                  busy (ld = 24: 5 rows of 6 lanes per warp instead of 4 rows of 8 lanes);
                                  bit 8 (without bit 5): the same packed groups in the line-search SpMM.
                                  Bits 3, 4 and 6 change no arithmetic, bit 5 only the order of the
                                  epilogue's sums, bits 7 and 8 the order of the row sums and of the
                                  partial sums.
                                  Default 394 = bits 1, 3, 7 and 8 (at n = 1e7, ld = 24: step update 4.09 ->
                                  3.81 ms, line-search SpMM 2.58 -> 2.46 ms). */
    int32_t inner_scale;       /* inner stop ||G||_F <= thr, z = A(RR^T) - b, e = tol (1 + ||b||_inf):
                                  0: thr = inner_rel max(||z||, e);  1: thr = inner_rel max(rho ||z||, e);
                                  2 (default): thr = max(e, min(inner_rel rho ||z||, inner_progress ||G_0||)) */
    double  admm_switch;       /* two-stage solve (Sec. 2): 0 (default) runs the ALM stage alone; > 0 stops the
                                  ALM stage once err1 and |err3| <= max(admm_switch, tol) and finishes with the
                                  splitting ADMM stage of Sec. 2.2 from U = V = R, the ALM stage's y and rho */
    double  cg_rel;            /* ADMM block steps: conjugate gradients (Algorithm 2) stop at ||r|| <= cg_rel ||r_0|| (1e-2) */
    int32_t cg_max;            /* ... or after cg_max steps (50) */
    int32_t admm_max_iter;     /* ADMM iterations (U step, V step, multiplier step) at most (20000) */
    int32_t reopt_level;       /* re-opt of Sec. 4.1 with the final criteria of Sec. 4.2: 0 (default) off; 1: the ALM
                                  solve stops on err1 <= tol alone, then while err1 (1 + ||b||_1 normalisation)
                                  or |err3| of the original problem exceed tol, C is scaled by reopt_factor
                                  (compounding) and the scaled problem is solved again from R, rho and the scaled
                                  y; 2: err2 must hold too (GPU Lanczos).  Takes precedence over admm_switch. */
    int32_t max_reopt;         /* re-opt rounds at most (5) */
    double  reopt_factor;      /* scale of C per round, in (0, 1) (0.1) */
} lorads_params;

typedef struct {
    double  primal_obj;        /* <C, R R^T> */
    double  dual_obj;          /* b^T y */
    double  err1;              /* ||A(RR^T) - b||_2 / (1 + ||b||_inf) */
    double  err2;              /* |min(0, sigma_min(C - A*(y)))| / (1 + ||vec C||_1), -1 if not evaluated */
    double  err3;              /* (<C,X> - b^T y) / (1 + |<C,X>| + |b^T y|) */
    double  sigma_min;         /* Lanczos estimate of sigma_min(C - A*(y)) */
    double  rho;               /* final penalty */
    double  seconds;           /* wall time of lorads_solve */
    int32_t rank;              /* final r */
    int32_t outer_iters;
    int32_t inner_iters;       /* L-BFGS directions computed, all outer steps */
    int32_t status;            /* lorads_status of the solve */
    int64_t kernel_launches;   /* kernels this library launched during the solve (graph nodes included) */
    int32_t admm_iters;        /* iterations of the ADMM stage (0: the ALM stage met the tolerance or admm_switch = 0) */
    int32_t cg_steps;          /* conjugate-gradient steps of the ADMM stage, both block steps summed */
    int32_t reopt_rounds;      /* re-opt rounds taken */
    int32_t reserved_r;
    double  reopt_scale;       /* final scale of C in the re-opt rounds (1: none) */
} lorads_result;

/* Fills *p with the defaults listed above. */
void lorads_default_params(lorads_params* p);

/* Uploads the primal SDP of Eq. (1.1).
 *   n                          order of X (>= 1)
 *   c_rowptr[n+1], c_colind[nnz], c_val[nnz]   C as a full symmetric CSR matrix, host,
 *                              rowptr[0] = 0, nondecreasing, column indices sorted and
 *                              distinct within each row, values finite; C must equal C^T.
 *   m                          number of constraints (>= 1)
 *   nnz_a, a_con, a_row, a_col, a_val          constraint triplets, host; a_con in [0,m),
 *                              a_row <= a_col < n, every constraint at least one triplet,
 *                              no entry (i, j) twice in one constraint.
 *   b[m]                       right-hand side, host.
 *   p                          parameters (NULL = defaults), copied; a value outside the
 *                              ranges listed with lorads_params is refused (INVALID_ARG).
 *   cuda_stream                cudaStream_t the context uses (NULL = default stream).
 * On success *out receives a new context (free with lorads_destroy).  On failure *out
 * is NULL and the status says why (INVALID_ARG, NOT_SYMMETRIC, UNSUPPORTED, OOM, CUDA). */
lorads_status lorads_create(lorads_ctx** out, int64_t n,
                            const int64_t* c_rowptr, const int32_t* c_colind, const double* c_val,
                            int64_t m, int64_t nnz_a,
                            const int32_t* a_con, const int32_t* a_row, const int32_t* a_col,
                            const double* a_val, const double* b,
                            const lorads_params* p, void* cuda_stream);

/* out = (C - A*(v)) R  (the sparse-times-tall-skinny product of the gradient, Sec. 2;
 * Eq. (3.1) with the multiplier folded into the values of the fixed pattern).
 *   R, out      device, n x ld (prec: FP64 double->double, FP32 float->float,
 *               BF16 bf16->float); out must not alias R.
 *   v           device double[m] or NULL (NULL: out = C R).
 * Asynchronous on the context stream. */
lorads_status lorads_spmm(lorads_ctx* ctx, const void* R, int32_t r, int32_t ld,
                          const double* v, void* out, int32_t prec);

/* out_k = <A_k, U V^T>  for k = 0..m-1 (the constraint map evaluated as one gathered
 * row dot per constraint: Sec. 3.4's compressed outer product; diag(RR^T) for MaxCut).
 *   U, V        device, n x ld, element type by prec (FP64, FP32 or BF16); may be equal.
 *   out         device double[m].  Products in the element precision, sum in FP64
 *               for FP64 and in FP32 otherwise, output FP64.
 * Asynchronous on the context stream. */
lorads_status lorads_constraint_eval(lorads_ctx* ctx, const void* U, const void* V,
                                     int32_t r, int32_t ld, double* out, int32_t prec);

/* Exact line search along D at R (App. A.2), lambda := y:
 *   p1 = <C, RD^T + DR^T>, p2 = <C, DD^T>, q0 = b - A(RR^T), q1 = A(RD^T + DR^T), q2 = A(DD^T)
 *   a1 = rho/2 ||q2||^2, a2 = rho q1^T q2, a3 = p2 - (y + rho q0)^T q2 + rho/2 ||q1||^2,
 *   a4 = p1 - (y + rho q0)^T q1
 * and tau* = the positive real root of 4a1 t^3 + 3a2 t^2 + 2a3 t + a4 with the lowest
 * quartic value (0 if none lowers it).
 *   R, D        device, n x ld, element type by prec (FP64, FP32 or BF16).
 *   y           device double[m].
 *   a_out[4]    host, receives a1..a4 (FP64 reductions).   tau_out: host, may be NULL.
 * Synchronous: returns after the stream has produced the results. */
lorads_status lorads_linesearch_coeffs(lorads_ctx* ctx, const void* R, const void* D,
                                       int32_t r, int32_t ld, const double* y, double rho,
                                       double* a_out, double* tau_out, int32_t prec);

/* Runs the solver (Sec. 2.1 ALM + Algorithm 1 + App. A.1/A.2) from R0 and y0.
 *   R0          n x r0 row-major (leading dimension r0), FP64; host if r0_on_device == 0,
 *               device otherwise; NULL: rows drawn on the device (SplitMix64 normals,
 *               unit rows for diagonal constraints) with r0 = ceil(log2 m) if r0 <= 0.
 *   y0          host double[m] or NULL (zeros).
 *   res         host, receives the result (also on failure, with res->status).
 * The solution stays in the context (lorads_get_solution). Synchronous. */
lorads_status lorads_solve(lorads_ctx* ctx, const double* R0, int32_t r0, int32_t r0_on_device,
                           const double* y0, lorads_result* res);

/* ------------------------------------------------------------------ splitting (ADMM) stage
 * Sec. 2.2: with X = U V^T and L_rho(U, V, y) = <C, U V^T> - y^T (A(U V^T) - b)
 * + rho/2 ||A(U V^T) - b||^2 + rho/2 ||U - V||_F^2 (Eq. (1.3) in the sign of y), the steps of
 * Eq. (2.2) are U <- argmin_U L_rho, V <- argmin_V L_rho, y <- y - rho (A(U V^T) - b); each
 * argmin is the positive definite system of Eq. (2.3), for the U step
 *     frakA_V(U) = rho A*(A(U V^T)) V + rho U  =  frakb_V = -C V + A*(y) V + rho A*(b) V + rho V,
 * solved by the conjugate gradients of Algorithm 2 from the current iterate (the V step
 * exchanges U and V).  The stage reports R = (U + V)/2 and stops when err1 and |err3| of
 * Sec. 4.2 at R are <= tol. */

/* out = frakA_V(X) = rho A*(A(X V^T)) V + rho X (the left side of Eq. (2.3)).
 *   V, X, out   device, n x ld, double (prec LORADS_FP64) or float (LORADS_FP32); out must
 *               alias neither V nor X.   rho > 0.
 * Asynchronous on the context stream; allocates nothing. */
lorads_status lorads_admm_operator(lorads_ctx* ctx, const void* V, const void* X, int32_t r, int32_t ld,
                                   double rho, void* out, int32_t prec);

/* Solves frakA_V(X) = frakb_V(y) by Algorithm 2 in place, from the X given: stops at
 * ||r|| <= cg_rel ||r_0|| or after cg_max steps (the parameters of the stage).
 *   V, X        device, n x ld, double (LORADS_FP64) or float (LORADS_FP32); X is overwritten.
 *   y           device double[m].   rho > 0.   steps_out (host, may be NULL): CG steps taken.
 * The work arrays (three n x ld vectors and one m-vector) are allocated on the first call
 * and kept by the context for later calls and solves.  Synchronous. */
lorads_status lorads_admm_cg(lorads_ctx* ctx, const void* V, void* X, const double* y, double rho, int32_t r,
                             int32_t ld, double cg_rel, int32_t cg_max, int32_t* steps_out, int32_t prec);

/* Runs the ADMM stage alone from U = V = R0 with multiplier y0 and penalty rho (held fixed),
 * in the precision form of params.prec, for at most params.admm_max_iter iterations with
 * params.cg_rel / params.cg_max.  R0, r0, r0_on_device, y0 as in lorads_solve (y0 host, NULL:
 * zeros).  res: R = (U + V)/2 and y stay in the context (lorads_get_solution); inner_iters = 0.
 * Synchronous. */
lorads_status lorads_admm_stage(lorads_ctx* ctx, const double* R0, int32_t r0, int32_t r0_on_device,
                                const double* y0, double rho, lorads_result* res);

/* sigma_min(C - A*(y)), the dual-slack eigenvalue behind err2 of Sec. 4.2 (which the
 * paper evaluates on the CPU), by a `steps`-step Lanczos run on the GPU with the
 * library's FP64 SpMM; the start vector is drawn from SplitMix64(seed).  The smallest
 * Ritz value is returned (an upper bound that converges to sigma_min).
 *   y          device double[m], or NULL for the multipliers of the last solve.
 *   sigma_out  host.   Synchronous. */
lorads_status lorads_dual_min_eig(lorads_ctx* ctx, const double* y, int32_t steps, uint64_t seed,
                                  double* sigma_out);

/* Copies the last solution to the host.  R_host (n x rank, leading dimension rank) and
 * y_host (m) may be NULL; R_capacity is the number of doubles R_host can hold.
 * *rank_out (may be NULL) receives the rank.  Synchronous. */
lorads_status lorads_get_solution(lorads_ctx* ctx, double* R_host, int64_t R_capacity,
                                  int32_t* rank_out, double* y_host);

/* Message of the last failure on this context ("" if none).  Valid until the next call. */
const char* lorads_last_error(const lorads_ctx* ctx);

/* Message of the last lorads_create failure in this thread. */
const char* lorads_create_error(void);

/* Frees the context and everything it owns.  NULL-safe. */
void lorads_destroy(lorads_ctx* ctx);

/* Sizes of the uploaded problem: n, m, nnz(C), number of diagonal and off-diagonal
 * constraints.  Any pointer may be NULL. */
lorads_status lorads_problem_info(const lorads_ctx* ctx, int64_t* n, int64_t* m, int64_t* nnz_c,
                                  int64_t* m_diag, int64_t* m_offdiag);

/* Average duration (ms) of each kernel family launched by the last lorads_solve that ran
 * with params.verbose >= 2.  That solve runs host-stepped (no CUDA graph, same kernels and
 * decisions) with a CUDA event pair around every launch on the solve stream.  names/ms
 * have `cap` entries (names are static strings); returns the number written, 0 when no
 * profiled solve has run. */
int32_t lorads_kernel_times(const lorads_ctx* ctx, const char** names, double* ms, int32_t cap);

/* Caps the total number of L-BFGS iterations of the next solves (0: no cap); a capped
 * solve ends with LORADS_ERR_MAXITER.  Used to time a fixed slice of a solve. */
lorads_status lorads_set_iteration_limit(lorads_ctx* ctx, int64_t max_total_inner);

/* Launch counts of the same profiled solve, by kernel family (same order as
 * lorads_kernel_times). */
int32_t lorads_kernel_counts(const lorads_ctx* ctx, const char** names, int64_t* counts, int32_t cap);

/* Exact line-search coefficients for callers that cannot allocate device memory.
 * The paper has no counterpart: this is a deployment variant of
 * lorads_linesearch_coeffs (FP64) that needs no context and allocates nothing.  It is
 * for callers that cannot call cudaMalloc where they need the step: frameworks whose
 * caching allocator owns the device memory (an allocation outside it can fail or
 * fragment what the framework holds), and latency-critical loops that cannot take the
 * device-wide synchronisation cudaMalloc and cudaFree may imply.
 *   n, c_rowptr[n+1] (int64), c_colind, c_val   C as full symmetric CSR, device.
 *   m, a_con, a_row, a_col, a_val (m triplets, one per constraint, row <= col), b[m]:
 *                     device; a_con is the constraint index of each triplet.
 *   R, D              device FP64, n x ld (ld a multiple of 4, at most 512), 16-byte aligned.
 *   y                 device double[m].   rho >= 0.
 *   out               device double[5]: a1, a2, a3, a4, tau (as lorads_linesearch_coeffs).
 *   cuda_stream       stream to run on (NULL = legacy default stream).  Asynchronous.
 * Inputs are not validated beyond sizes and pointers: pass what lorads_create accepts.
 * In particular every constraint must have exactly one triplet: the per-constraint
 * products of the line search are formed per triplet, so a constraint with several
 * triplets gives wrong coefficients (no error is returned).
 * Scratch: one fixed device array inside the library (2 x 1024 x 7 doubles, 114,688
 * bytes) that every GPU loading the library keeps until exit.  It is shared by all
 * calls on a device, so calls that overlap on the GPU race and must be ordered by the
 * caller; nothing needs clearing between calls.  The first call on each device looks
 * up the array's device address (cudaGetSymbolAddress, with that device current) and
 * caches it per device ordinal; make that first call before starting any stream
 * capture.  The kernels it launches are loaded on their first launch, one variant per
 * row width, so the first call with each ld takes longer than the calls after it.
 * After cudaDeviceReset on a device the cached address is stale: do not
 * call this entry point on that device again in the same process.  Sizes beyond the
 * limits above return LORADS_ERR_INVALID_ARG; the message is in lorads_noalloc_error().
 * Calls no allocation routine. */
lorads_status lorads_linesearch_coeffs_noalloc(int64_t n, const int64_t* c_rowptr, const int32_t* c_colind,
                                               const double* c_val, int64_t m, const int32_t* a_con,
                                               const int32_t* a_row, const int32_t* a_col, const double* a_val,
                                               const double* b, const double* R, const double* D, int32_t r,
                                               int32_t ld, const double* y, double rho, double* out,
                                               void* cuda_stream);

/* Message of the last lorads_linesearch_coeffs_noalloc failure in this thread. */
const char* lorads_noalloc_error(void);

/* ------------------------------------------------------------------ batched solve
 * Many independent instances of Eq. (1.1) solved by ONE persistent kernel launch
 * (captured in a CUDA graph).  The paper solves one instance at a time; this is the
 * serving form of the same method: every block of the launch takes the next instance
 * from a device work queue and runs the whole solve of lorads_solve on it (ALM of
 * Sec. 2.1, Algorithm 1, App. A.1/A.2) with block-wide reductions, taking the same
 * decisions from the same sums.  Instances are independent units: no communication.
 * Every instance keeps its problem arrays and iterate in device memory owned by the
 * batch; the iterate of each instance is allocated for up to two rank updates
 * (r0 -> ceil(1.5 r0) -> ceil(1.5 ceil(1.5 r0)), at most ceil(sqrt(2m)) and 128); a rank
 * request beyond that is dropped and the solve continues at the current rank. */
typedef struct lorads_batch lorads_batch;

/* Launch shape of the persistent kernel (lorads_batch_tune picks one). */
typedef struct {
    int32_t ctas_per_sm;    /* resident solver blocks per SM; grid = SMs x this (1..4) */
    int32_t rows_per_warp;  /* rows a warp works on at once: 1, 2, 4 or 8; lanes per row =
                               max(32 / rows_per_warp, smallest power of two >= ld/4) */
    int32_t order;          /* queue order: 0 input order, 1 largest estimated work first */
    int32_t threads;        /* threads per block: 256 or 512 (0 = 256) */
    int32_t cluster;        /* 1 (or 0): one block per instance; 2, 4 or 8: thread-block clusters of that
                               size solve the first team_count instances of the queue together (their
                               blocks split rows and constraints and reduce through distributed shared
                               memory), then their blocks take the remaining instances one each */
    int32_t team_count;     /* instances solved by a whole cluster (cluster > 1) */
} lorads_batch_shape;

typedef struct {
    double  seconds;          /* device time of the launch (CUDA events around the graph) */
    double  instances_per_s;  /* count / seconds */
    double  latency_p50_ms;   /* per-instance completion time after the first block started */
    double  latency_p99_ms;
    double  latency_max_ms;
    int64_t inner_iters;      /* L-BFGS iterations over all instances */
    int32_t solved;           /* instances that ended with LORADS_OK */
    int32_t grid;             /* blocks launched */
    lorads_batch_shape shape; /* shape of the launch */
} lorads_batch_stats;

/* Uploads `count` instances, each in the format of lorads_create, concatenated:
 *   n[count], m[count]        order of X and number of constraints of each instance.
 *   c_rowptr                  the n_i + 1 row pointers of each instance one after the other
 *                             (each list starts at 0); c_colind / c_val: the nnz_i = rowptr_i[n_i]
 *                             entries of each instance one after the other.
 *   a_con, a_row, a_col, a_val, b:  the m_i triplets / right-hand sides of each instance in
 *                             turn (one triplet per constraint; indices local to the instance).
 *   r0[count]                 starting rank of each instance, or NULL: ceil(log2 m_i) (>= 1).
 *   R0                        NULL (rows drawn on the device as in lorads_solve) or the
 *                             n_i x r0_i row-major FP64 starting factors one after the other.
 *   p                         parameters (NULL = defaults); prec must be LORADS_FP64,
 *                             LORADS_MIXED or LORADS_FP32; compute_err2, check_every,
 *                             kernel_variant and reopt_level do not apply; admm_switch > 0 runs
 *                             the ADMM stage of Sec. 2.2 after each instance's ALM stage, inside
 *                             the same launch (single-triplet constraints only, as below).
 * All inputs are host memory and are copied.  Each instance is validated as by
 * lorads_create; the first failure names the instance (lorads_batch_create_error). */
lorads_status lorads_batch_create(lorads_batch** out, int32_t count, const int64_t* n, const int64_t* m,
                                  const int64_t* c_rowptr, const int32_t* c_colind, const double* c_val,
                                  const int32_t* a_con, const int32_t* a_row, const int32_t* a_col,
                                  const double* a_val, const double* b, const int32_t* r0, const double* R0,
                                  const lorads_params* p, void* cuda_stream);

/* Solves every instance in one launch of the persistent kernel (shape: the last one set
 * or tuned; default 256 threads, 2 blocks per SM, 8 rows per warp, largest first).  Each instance
 * starts again from its starting point.  results[count] (host, may be NULL) receive one
 * lorads_result per instance in input order (seconds = that instance's own solve time,
 * err2 = -1); stats (host, may be NULL) the launch figures.  Returns LORADS_OK when the
 * launch completed, whatever the instances' statuses.  Synchronous. */
lorads_status lorads_batch_solve(lorads_batch* b, lorads_result* results, lorads_batch_stats* stats);

/* Times the persistent launch for each candidate shape (threads per block x blocks per SM
 * allowed by the kernel's occupancy x rows per warp x queue order, then clusters of 2, 4
 * and 8 blocks for the 1, 2 or 4 x (clusters resident) largest instances) with every
 * instance capped at probe_iters L-BFGS iterations, keeps the fastest as the batch's
 * shape and writes it to *best (may be NULL).  Synchronous. */
lorads_status lorads_batch_tune(lorads_batch* b, int32_t probe_iters, lorads_batch_shape* best);

/* Sets the launch shape used by the next lorads_batch_solve. */
lorads_status lorads_batch_set_shape(lorads_batch* b, const lorads_batch_shape* shape);

/* Caps every instance's total L-BFGS iterations in the next solves (0: no cap). */
lorads_status lorads_batch_set_iteration_limit(lorads_batch* b, int64_t max_total_inner);

/* Copies instance i's last solution to the host (as lorads_get_solution). */
lorads_status lorads_batch_get_solution(lorads_batch* b, int32_t i, double* R_host, int64_t R_capacity,
                                        int32_t* rank_out, double* y_host);

/* Device time (ms, %globaltimer at the block's barriers) that the last lorads_batch_solve
 * spent in each phase of instance i's solve (i = -1: summed over all instances): init,
 * direction, spmm_ls, cons_ls, root, step, ytil, spmm_a, update, hist, outer,
 * outer_gradient, rank_update.  names (static strings) and ms have cap entries (either may
 * be NULL); returns the number written (0 before a solve). */
int32_t lorads_batch_phase_times(const lorads_batch* b, int32_t i, const char** names, double* ms, int32_t cap);

/* Message of the last lorads_batch_create failure in this thread. */
const char* lorads_batch_create_error(void);

/* Message of the last failure on this batch ("" if none). */
const char* lorads_batch_last_error(const lorads_batch* b);

/* Frees the batch and everything it owns.  NULL-safe. */
void lorads_batch_destroy(lorads_batch* b);

/* ------------------------------------------------------------------ learned warm start
 * A small message-passing network that predicts a starting factor R0 (unit rows, the
 * feasible set of the MaxCut constraints X_ii = 1 of Sec. 4.3) from the pattern of C, to
 * replace the random start of the solve.  The paper has no such network; it is trained
 * on the factors R* that lorads_solve / lorads_batch_solve return.  Definition (F = 16,
 * H = 32, w_ij = C_ij for i != j, s_i = sum_j |w_ij|, deg_i = #{j != i: C_ij stored}):
 *   x_i   = [1, log(1 + deg_i)/4, sum_j w_ij / s_i, C_ii / s_i, g_i1..g_i12]  (ratios 0 if s_i = 0),
 *           g_ik = standard normal number e = 12 i + k - 1 of the SplitMix64 / Box-Muller stream
 *           of lorads_solve's start draws with base seed ^ (0x474E4E * 0x9E3779B97F4A7C15);
 *   layer l = 1..3:  m_i = sum_{j != i} (w_ij / s_i) h_j,  h_i <- relu(W_s h_i + W_n m_i + b);
 *   o_i = W_o h_i + b_o (r_out values),  r_hat_i = o_i / ||o_i||;
 *   loss = (1/|E|) sum over stored pairs i < j of (r_hat_i . r_hat_j - X*_ij)^2,
 *           X*_ij = r*_i . r*_j  (invariant to rotations of R*).
 * Parameters: one float vector, for l = 1..3: W_s (H x F_in row-major, F_in = 16 then 32),
 * W_n (H x F_in), b (H); then W_o (r_out x H), b_o (r_out).
 * Graph arguments are C as a symmetric CSR matrix in DEVICE memory (n, rowptr int64,
 * colind int32, val double: the arrays lorads_create accepts, uploaded by the caller).
 * Activations are stored in bf16 (act_prec LORADS_BF16; weights rounded to bf16 for the
 * forward pass) or float (LORADS_FP32); arithmetic and gradients are float; Adam
 * (beta1 0.9, beta2 0.999, eps 1e-8) updates float master weights.  All calls run on the
 * network's stream and are asynchronous unless stated. */
typedef struct lorads_gnn lorads_gnn;

/* Number of parameters for r_out outputs (1..32), or -1. */
int64_t lorads_gnn_param_count(int32_t r_out);

/* New network with parameters theta0 (host, lorads_gnn_param_count(r_out) floats). */
lorads_status lorads_gnn_create(lorads_gnn** out, int32_t r_out, int32_t act_prec, const float* theta0,
                                void* cuda_stream);

/* Copies the parameters to / from the host (count >= the parameter count); set also resets
 * the Adam moments.  Synchronous. */
lorads_status lorads_gnn_get_params(lorads_gnn* g, float* theta_host, int64_t count);
lorads_status lorads_gnn_set_params(lorads_gnn* g, const float* theta_host, int64_t count);

/* Forward pass on the graph of C: R_out (device, n x ld FP64, ld >= r_out) receives
 * r_hat in columns 0..r_out-1 and zeros after. */
lorads_status lorads_gnn_predict(lorads_gnn* g, int64_t n, const int64_t* c_rowptr, const int32_t* c_colind,
                                 const double* c_val, uint64_t feature_seed, int32_t ld, double* R_out);

/* Training targets: targets[e] = r_i . r_j for every stored entry e = (i, j) of C
 * (0 on the diagonal).  R: device n x ld FP64 (columns 0..r-1 used); targets: device
 * float[nnz(C)].  Runs on cuda_stream. */
lorads_status lorads_gnn_edge_targets(int64_t n, const int64_t* c_rowptr, const int32_t* c_colind, const double* R,
                                      int32_t r, int32_t ld, float* targets, void* cuda_stream);

/* One training step on one graph: forward, loss, hand-written backward, then an Adam
 * step with learning rate lr (lr = 0: no update).  n_edges = number of pairs i < j with
 * C_ij stored.  loss_out (host, may be NULL; synchronises when given) receives the loss
 * before the update; grad_out (device, may be NULL) the gradient. */
lorads_status lorads_gnn_train_step(lorads_gnn* g, int64_t n, const int64_t* c_rowptr, const int32_t* c_colind,
                                    const double* c_val, uint64_t feature_seed, const float* targets,
                                    int64_t n_edges, float lr, double* loss_out, float* grad_out);

/* Message of the last failure on this network / of the last lorads_gnn_create. */
const char* lorads_gnn_last_error(const lorads_gnn* g);
const char* lorads_gnn_create_error(void);

/* Frees the network.  NULL-safe. */
void lorads_gnn_destroy(lorads_gnn* g);

#ifdef __cplusplus
}
#endif

#endif /* LORADS_H */
