/*
 * ncl_kkt.h -- C ABI of the GB300 sparse LDL^T library for the KKT systems
 * of Algorithm NCL (MadNCL, arXiv 2510.05885).
 *
 * The library factors and solves, on one GPU, the two regular forms of the
 * NCL Newton system derived in Section 3 of the paper:
 *
 *   stabilized (Section 3.2, Eq. K2r), dimension n+m:
 *       [ H + Sigma + delta I    J^T       ] [u]   [f]
 *       [ J                     -rho^-1 I  ] [v] = [g]
 *   condensed (Section 3.3, Eq. K1), dimension n:
 *       K = H + Sigma + delta I + rho J^T J
 *
 * by a supernodal multifrontal LDL^T with D diagonal and static pivoting
 * (Section 3.1, "Sparse LDL^T factorization"): any symmetric permutation of a
 * symmetric quasi-definite matrix has such a factorisation (Section 3.2), so
 * the ordering is free to minimise fill.  A pivot with |d| <= pivot_eps is
 * replaced by +-pivot_eps, the sign being that of the block (primal +,
 * dual -) the index belongs to before reordering (Section 3.1 case (ii);
 * eps = 1e-10 in Section 4.3), and the solution of the unperturbed system
 * is recovered by iterative refinement (Section 4.3).  The inertia of the
 * factored matrix is returned; (n, m, 0) for K2r and (n, 0, 0) for K are
 * equivalent to a correct inertia of the full system K2 (Section 3.4).
 *
 * The caller passes rho as one scalar: -1/rho goes in the dual block of
 * K2r, +rho multiplies J^T J in K.  (The paper writes rho-hat = rho + delta
 * there; a caller following it passes rho-hat.)
 *
 * Around these: the condensed form with slacks (Section 3.3, Eq. K1s;
 * ncl_kkt_factor_k1s and its right-hand side and slack step), the inertia
 * correction of Section 3.1 (ncl_kkt_factor_regularize), the right-hand side
 * of the Newton step and the recovery of its other components (Sections
 * 3.1-3.3; ncl_kkt_newton_rhs / ncl_kkt_newton_recover), the adjoint, and
 * batches of independent instances in one handle.
 *
 * Conventions shared by every entry point
 *   - Pattern arrays (CSR row pointers and column indices) are HOST memory.
 *     Value arrays, right-hand sides and solutions are DEVICE memory, FP64.
 *   - H is passed as its lower triangle by rows (column <= row), column
 *     indices sorted and unique within each row; each off-diagonal value
 *     stands for both (i,j) and (j,i).  The diagonal of H may be absent
 *     (Sigma + delta is always on the diagonal).
 *   - J is m x n CSR, column indices sorted and unique within each row.
 *   - Value arrays follow the order of the pattern given to analyze.
 *   - Multi-RHS blocks are column-major: column k of B starts at B + k*ldb.
 *   - The caller owns every buffer it passes; the handle owns the plan, the
 *     factors and all workspace.  Nothing is retained after a call returns.
 *   - Errors are status codes; nothing is thrown across the ABI.  On error
 *     ncl_kkt_last_error() returns a message for the calling thread.
 *   - A handle is used by one host thread at a time, and all its work is
 *     issued on the stream passed to each call (NULL = the legacy default
 *     stream).  Calls return after their work is complete.
 */
#ifndef NCL_KKT_H
#define NCL_KKT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ncl_kkt_s* ncl_kkt_t;   /* opaque handle: plan + factors */
typedef void* ncl_stream_t;            /* a cudaStream_t */

typedef enum {
    NCL_KKT_STABILIZED = 0,   /* K2r, Section 3.2 */
    NCL_KKT_CONDENSED = 1     /* K1,  Section 3.3 */
} ncl_kkt_form;

typedef enum {
    NCL_PREC_FP64 = 0,        /* factor and solve in FP64 */
    NCL_PREC_FP32_IR = 1      /* FP32 factor (split-TF32 tensor-core updates),
                                 FP64 residual and refinement */
} ncl_kkt_prec;

typedef enum {
    NCL_PIVOT_PERTURB = 0,    /* Section 3.1 case (ii): replace by +-eps, go on */
    NCL_PIVOT_STOP = 1        /* Section 3.1 case (i): report the tiny pivots
                                 as zero eigenvalues and NCL_ERR_ZERO_PIVOT */
} ncl_pivot_policy;

typedef enum {
    NCL_OK = 0,
    NCL_ERR_INVALID_ARG = 1,      /* NULL pointer, negative size, bad enum */
    NCL_ERR_PATTERN = 2,          /* unsorted / out-of-range / upper-triangle index */
    NCL_ERR_OOM = 3,              /* device or host allocation failed, or over
                                     options.max_device_bytes */
    NCL_ERR_CUDA = 4,             /* a CUDA call failed (message has the code) */
    NCL_ERR_STATE = 5,            /* solve/adjoint before a successful factor */
    NCL_ERR_ZERO_PIVOT = 6,       /* policy STOP and a pivot with |d| <= eps */
    NCL_ERR_NUMERIC = 7,          /* a NaN or Inf pivot or solution */
    NCL_ERR_IR_NOT_CONVERGED = 8, /* refinement reached ir_max_iter above ir_tol;
                                     the best iterate is still returned */
    NCL_ERR_TIMEOUT = 9,          /* a bounded device wait ran out */
    NCL_ERR_INERTIA = 10          /* ncl_kkt_factor_regularize: an instance's inertia
                                     is still irregular after max_tries factorisations */
} ncl_status;

typedef struct {
    int32_t prec;             /* ncl_kkt_prec, default NCL_PREC_FP32_IR */
    int32_t pivot_policy;     /* ncl_pivot_policy, default PERTURB */
    double pivot_eps;         /* default 1e-10 (Section 4.3) */
    double ir_tol;            /* target normwise backward error
                                 ||b-Kx||_inf/(||K||_inf||x||_inf+||b||_inf);
                                 <= 0 selects 1e-10 (FP32_IR) or 1e-12 (FP64) */
    int32_t ir_max_iter;      /* refinement steps; < 0 selects 10 (FP32_IR) or 3 (FP64) */
    int32_t use_fgmres;       /* 1: FGMRES-IR when Richardson stagnates (default 1) */
    int32_t use_tensor_cores; /* FP32_IR, fronts with >= tc_min_pivots pivots: 2
                                 (default) tcgen05 split-TF32 update blocks and panel
                                 trailing updates; 1: update blocks only; 0: SIMT
                                 FP32 everywhere */
    int32_t leaf_size;        /* nested-dissection leaf size (default 96) */
    int32_t host_only;        /* 1: symbolic analysis only, no device memory; the
                                 handle then answers only the get_* queries */
    int32_t precision_fallback; /* FP32_IR: 1 (default) refactor the same FP64 values in
                                 FP64 when the FP32 factor cannot be trusted (an
                                 inertia other than (n,m,0) / (n,0,0), which FP32
                                 produces when rho*||J||^2 swamps H+Sigma+delta I) or
                                 when refinement cannot reach ir_tol, and remember,
                                 per instance, the penalty rho of such a fallback
                                 whose FP64 factors were regular: a later
                                 factorisation in which some instance's rho is at
                                 least its remembered one starts in FP64 directly
                                 (fp64_fallback = 2; the penalty of the NCL outer
                                 loop only grows, Algorithm 1); 2: fall back the
                                 same way but remember nothing (every factorisation
                                 tries FP32 first); 0: never */
    int64_t max_device_bytes; /* 0 = no limit */
    int64_t wait_cycles;      /* bound, in SM clock cycles, of every wait of one CTA
                                 on another inside a kernel (the panel factorisation's
                                 rows waiting for the diagonal block, the chained
                                 triangular sweeps, the tensor-core pipeline); past it
                                 the kernel sets an error flag, finishes without the
                                 awaited data and the call returns NCL_ERR_TIMEOUT.
                                 <= 0 selects 4e9 (about 2 s) */
    int32_t persistent_fronts; /* 1: the large fronts of each level are factored by
                                 one persistent launch whose CTAs take panel, row
                                 and trailing-update tile tasks from a
                                 dependency-ordered list; 0 (default): one launch
                                 per 128-column panel step plus one per trailing
                                 update (measured a few percent faster on every
                                 workload of the autotuner's classes) */
    double ir_switch;         /* single-instance handles with use_fgmres: Richardson
                                 hands over to FGMRES as soon as a step reduces the
                                 backward error by less than this factor (default
                                 0.5; values outside (0, 1] select it) */
    int32_t subtree_sweeps;   /* 1 (default): every maximal subtree of supernodes with
                                 at most 32 pivots (and a front that fits the
                                 shared-memory front) is factored by one CTA and, in
                                 the triangular sweeps, swept by one warp (one launch
                                 each for all of them, largest subtrees first); 0:
                                 those supernodes go through the per-level launches
                                 like the others */
    int32_t tc_min_pivots;    /* FP32_IR: large fronts with at least this many pivots
                                 get split TF32 operands and tensor-core updates
                                 (default 256, >= 32) */
    const char* autotune_path; /* NULL (default), or a table written by the autotuner
                                 (paper_2510_05885_gb300/autotune.py): at analysis the
                                 first line whose form, dimension range and
                                 instance-count range match sets persistent_fronts,
                                 subtree_sweeps, use_tensor_cores and tc_min_pivots
                                 (lines "form dim_lo dim_hi count_lo count_hi
                                 persistent subtree tensor_cores tc_min_pivots",
                                 dim_hi exclusive, '#' comments).  Read once during
                                 the call; an unreadable file or a bad line is
                                 INVALID_ARG */
} ncl_kkt_options;

typedef struct {
    int64_t n_pos, n_neg, n_zero;  /* inertia of the factored matrix */
    int64_t n_perturbed;           /* pivots replaced by +-eps */
    int64_t nnz_L;                 /* strictly-lower nonzeros of L (no padding) */
    double flops;                  /* sum_j (c_j^2 + 3 c_j), c_j = nnz of column j of L
                                      below the diagonal */
    float ms;                      /* device time of the call */
    int32_t fp64_fallback;         /* 0: FP32 factors (or an FP64 handle); 1: the FP64
                                      refactorisation after an untrusted FP32 one;
                                      2: FP64 factors started directly (the penalty
                                      is at least one where FP32 failed before) */
} ncl_kkt_factor_info;

typedef struct {
    int32_t ir_iters;              /* refinement steps taken */
    int32_t used_fgmres;           /* 1 if the FGMRES fallback ran */
    double backward_err;           /* final normwise backward error (max over RHS) */
    float ms;                      /* device time of the call */
    int32_t fp64_fallback;         /* 1 if the FP64 refactorisation solved it */
} ncl_kkt_solve_info;

typedef struct {
    int64_t dim;                   /* n+m (K2r) or n (K), summed over instances */
    int64_t nnz_A;                 /* lower-triangle nonzeros of the KKT matrix */
    int64_t nnz_L;                 /* strictly-lower nonzeros of L (no padding) */
    int64_t nnz_L_stored;          /* stored factor entries incl. supernode padding */
    int64_t update_entries;        /* stored multifrontal update-matrix entries */
    int64_t n_supernodes, n_levels, max_front, max_pivots;
    int64_t device_bytes;          /* device memory held by the handle */
    double flops;                  /* algorithmic factorisation flops */
    double analyze_ms;             /* host time of analyze */
} ncl_kkt_analysis_info;

/* Fill *opt with the defaults listed above. */
void ncl_kkt_default_options(ncl_kkt_options* opt);

/*
 * ncl_kkt_analyze -- symbolic phase, once per pattern (the paper reuses the
 * symbolic factorisation across Newton steps, Section 4.1).
 *   form       ncl_kkt_form
 *   n, m       primal / dual sizes (m may be 0)
 *   H_rowptr   host int32[n+1], H_colind host int32[H_rowptr[n]] (lower, sorted)
 *   J_rowptr   host int32[m+1], J_colind host int32[J_rowptr[m]] (sorted)
 *   opt        NULL for defaults
 *   out        receives the handle
 * Builds the KKT pattern, a nested-dissection ordering, the elimination
 * tree, relaxed supernodes and the multifrontal schedule, and allocates all
 * device memory the numeric phase needs.  Uses the current CUDA device.
 * Errors: INVALID_ARG, PATTERN, OOM, CUDA.
 */
ncl_status ncl_kkt_analyze(int32_t form, int32_t n, int32_t m,
                           const int32_t* H_rowptr, const int32_t* H_colind,
                           const int32_t* J_rowptr, const int32_t* J_colind,
                           const ncl_kkt_options* opt, ncl_kkt_t* out);

/*
 * ncl_kkt_analyze_like -- a new handle with the options opt (e.g. another
 * precision or pivot policy) on the analysis of an existing handle src: the
 * pattern, ordering, supernodes and schedule are copied, not recomputed
 * (analyse once, factor in several precisions).  opt->leaf_size is not used.
 * src is not modified and may be destroyed afterwards.  Uses the current
 * CUDA device.  Errors: INVALID_ARG, OOM, CUDA.
 */
ncl_status ncl_kkt_analyze_like(ncl_kkt_t src, const ncl_kkt_options* opt, ncl_kkt_t* out);

/*
 * ncl_kkt_factor -- numeric LDL^T of the KKT matrix for new values on the
 * analysed pattern (every Newton step).
 *   H_val   device double[nnz(H)], J_val device double[nnz(J)],
 *   Sigma   device double[n] (the diagonal of Section 3.1, Eq. K2unreg),
 *   delta   primal regularisation, rho penalty (> 0)
 *   info    may be NULL; receives inertia, perturbed count, flops, time
 * The FP64 KKT values are assembled on the device (rho J^T J as a sparse
 * product in FP64 for K), then factored in the handle's precision.
 * Returns NCL_OK even for a wrong inertia (the caller raises delta, Section
 * 3.1); ZERO_PIVOT under the STOP policy; NUMERIC for a NaN/Inf pivot.
 */
ncl_status ncl_kkt_factor(ncl_kkt_t h, const double* H_val, const double* J_val,
                          const double* Sigma, double delta, double rho,
                          ncl_stream_t stream, ncl_kkt_factor_info* info);

/*
 * ncl_kkt_solve -- X = K^{-1} B for nrhs >= 1 right-hand sides, using the
 * current factors, with FP64 iterative refinement on the FP64 matrix
 * (Section 4.3) until the backward error is <= ir_tol.
 *   B  device double, dim x nrhs, column-major, leading dimension ldb >= dim
 *   X  device double, dim x nrhs, leading dimension ldx >= dim (may not alias B)
 * Errors: STATE (no factor), IR_NOT_CONVERGED (X still holds the best iterate).
 */
ncl_status ncl_kkt_solve(ncl_kkt_t h, int32_t nrhs, const double* B, int64_t ldb,
                         double* X, int64_t ldx, ncl_stream_t stream,
                         ncl_kkt_solve_info* info);

/*
 * ncl_kkt_adjoint -- reverse-mode derivative of X = K^{-1} B.
 * Given X (from ncl_kkt_solve) and GX = dl/dX, computes
 *   GB = K^{-1} GX   (K is symmetric; refined like a solve)
 *   dl/dK = -GB X^T folded onto the stored values:
 *     G_Hval  for an off-diagonal lower H value (i,j): -(gb_i x_j + gb_j x_i),
 *             on the diagonal -gb_i x_i
 *     G_Jval  K2r: -(gb_{n+r} x_c + gb_c x_{n+r});
 *             K:   -rho ((J gb)_r x_c + (J x)_r gb_c)
 *     G_Sigma -gb_i x_i
 *     G_scal  [0] = dl/ddelta = -sum_{i<n} gb_i x_i,
 *             [1] = dl/drho  = K2r: -(1/rho^2) sum_{dual} gb_i x_i;
 *                              K:   -(J gb).(J x)
 *   summed over the nrhs columns.  All arrays are device FP64 with the
 *   layouts of analyze/factor/solve; any gradient pointer may be NULL.
 */
ncl_status ncl_kkt_adjoint(ncl_kkt_t h, int32_t nrhs, const double* X, int64_t ldx,
                           const double* GX, int64_t ldgx, double* GB, int64_t ldgb,
                           double* G_Hval, double* G_Jval, double* G_Sigma, double* G_scal,
                           ncl_stream_t stream, ncl_kkt_solve_info* info);

/*
 * ncl_kkt_solve_noalloc -- ncl_kkt_solve without any memory allocation (the
 * paper has no counterpart).  It serves callers that cannot allocate at the
 * point where they solve: real-time loops that cannot afford an allocator
 * round trip, and processes whose device memory is committed elsewhere (for
 * instance a factorisation sized to max_device_bytes).  Same arguments and
 * results as ncl_kkt_solve on a handle that has been factored, with two
 * differences: it never refactors in FP64 (an FP32_IR handle whose
 * refinement falls short returns NCL_ERR_IR_NOT_CONVERGED with the best
 * iterate, where ncl_kkt_solve would escalate), and its FGMRES stage runs
 * only when the Krylov vectors also fit in the static array (else it is left
 * out of the call).  After an earlier precision fallback the FP64 factors
 * are used, on the same static array.
 * The sweep and refinement workspace comes from one static device array of
 * 8 MiB inside the library (held by every GPU that loads the library until
 * the process exits) instead of the handle's workspace.  It must hold
 * min(nrhs, 8) * (dim + update and partial-sum vectors) solve values plus
 * min(nrhs, 8) * dim FP64 residuals (about dim <= 100k at one right-hand
 * side in FP32); larger problems get NCL_ERR_INVALID_ARG with the required
 * size in ncl_kkt_last_error().  The FGMRES stage needs 41 * dim FP64
 * values more.  The first call on a device looks up the array's device
 * address.  Every call shares the one array, which keeps the last call's
 * contents (the call clears what must start at zero itself); calls whose
 * work overlapped on the GPU would race on it, so the library serialises
 * them on the host and each returns only after its work is complete.  The
 * refinement reads norms back to the host between steps, so a stream under
 * graph capture is refused (NCL_ERR_STATE), as is a handle with profiling on.
 */
ncl_status ncl_kkt_solve_noalloc(ncl_kkt_t h, int32_t nrhs, const double* B, int64_t ldb,
                                 double* X, int64_t ldx, ncl_stream_t stream,
                                 ncl_kkt_solve_info* info);

/* The options in effect for a handle (after the defaults, and after a
 * tuned table's line if one matched; autotune_path is returned NULL). */
ncl_status ncl_kkt_get_options(ncl_kkt_t h, ncl_kkt_options* out);

/* Sizes and counts of the analysis (host struct). */
ncl_status ncl_kkt_get_analysis_info(ncl_kkt_t h, ncl_kkt_analysis_info* out);

/* The fill-reducing permutation: perm[k] = original index of the k-th
 * pivot (host int32[dim]). */
ncl_status ncl_kkt_get_permutation(ncl_kkt_t h, int32_t* perm);

/* Free the handle and its device memory (NULL is ignored). */
void ncl_kkt_destroy(ncl_kkt_t h);

/* Static string naming a status code. */
const char* ncl_kkt_status_string(ncl_status st);

/* Detail message of the last error on the calling thread ("" if none). */
const char* ncl_kkt_last_error(void);

/* ------------------------------------------------------------------------
 * Batches: many independent KKT systems of uneven size and pattern (such as
 * the scenarios or contingencies of one network) factored and solved by one
 * handle.  The batch is one block-diagonal system: every kernel launch of a
 * factorisation or solve covers all instances, and the whole factor + solve
 * is replayed from one captured CUDA graph.
 *
 * Instance i has form forms[i] (all equal), sizes n[i], m[i] and its own
 * pattern (pointers into host arrays).  Values are passed CONCATENATED in
 * instance order: H values of instance 0, then 1, ...; likewise J values,
 * Sigma (n[i] each) and right-hand sides (dim_i rows each, so B is the
 * concatenated dim x nrhs column-major block).  delta and rho are host
 * arrays with one entry per instance.
 * ------------------------------------------------------------------------ */

ncl_status ncl_kkt_batch_analyze(int32_t count, int32_t form, const int32_t* n, const int32_t* m,
                                 const int32_t* const* H_rowptr, const int32_t* const* H_colind,
                                 const int32_t* const* J_rowptr, const int32_t* const* J_colind,
                                 const ncl_kkt_options* opt, ncl_kkt_t* out);

/* Factor all instances (values concatenated; delta, rho host arrays of
 * length count).  infos (host, may be NULL) receives one struct per
 * instance; the status is the worst over instances. */
ncl_status ncl_kkt_batch_factor(ncl_kkt_t h, const double* H_val, const double* J_val,
                                const double* Sigma, const double* delta, const double* rho,
                                ncl_stream_t stream, ncl_kkt_factor_info* infos);

/*
 * ncl_kkt_factor_k1s -- the condensed system with slacks, Eq. K1s (Section
 * 3.3, proposition on the condensed KKT system): on a CONDENSED handle whose
 * J rows are the constraints h = (c_E, c_I) of an NCO problem (Section 3.3),
 * factor
 *   K = H + Sigma + delta I + sum_r w_r J_r^T J_r,
 *   w_r = rho for a row without slack, rho Omega_r for a row with slack,
 *   Omega_r = Sigma_s,r / (rho + Sigma_s,r)  (so Omega_r -> 1 as Sigma_s,r -> inf).
 *   Sigma_s  device double[m] (batch: concatenated by instance): the slack
 *            barrier term of each constraint row, >= 0, or +inf for a row
 *            without slack (an equality row)
 *   H_val, J_val, Sigma (= Sigma_t of the paper), delta, rho, infos: as in
 *            ncl_kkt_batch_factor (host arrays of length count; count = 1 for
 *            a single handle); rho is the penalty of the matrix (rho-hat)
 * ncl_kkt_k1s_rhs forms the right-hand side, ncl_kkt_solve then gives
 * Delta t and ncl_kkt_k1s_slack_step Delta s.  The adjoint of a
 * K1s factorisation differentiates through the weights (dl/dJ, dl/drho);
 * dl/dSigma_s is not computed.
 * Errors: INVALID_ARG (not a condensed handle, NULL Sigma_s), and those of
 * ncl_kkt_batch_factor.
 */
ncl_status ncl_kkt_factor_k1s(ncl_kkt_t h, const double* H_val, const double* J_val,
                              const double* Sigma, const double* Sigma_s, const double* delta,
                              const double* rho, ncl_stream_t stream, ncl_kkt_factor_info* infos);

/*
 * Newton step of Algorithm NCL around the factorisation (Section 3.1-3.3).
 * A Newton point holds device arrays over the concatenated primal variables
 * (n-vectors) and constraints (m-vectors) of the handle's instances:
 */
typedef struct {
    const double* grad_phi;   /* n: gradient of the objective at x */
    const double* x;          /* n: current point, strictly inside its bounds */
    const double* lower;      /* n: lower bounds l (-inf: none) */
    const double* upper;      /* n: upper bounds u (+inf: none) */
    const double* z_lower;    /* n: bound multipliers z_l (0 where l = -inf) */
    const double* z_upper;    /* n: bound multipliers z_u (0 where u = +inf) */
    const double* c;          /* m: constraint values c(x) */
    const double* y;          /* m: current multipliers y */
    const double* y_k;        /* m: multiplier estimate y_k of the outer iteration */
    const double* r;          /* m: current residual variables r */
} ncl_kkt_newton_point;

/*
 * ncl_kkt_newton_rhs -- the right-hand side of the factored system:
 *   K2r (Eq. K2r, unknown [Delta x; -Delta y]):
 *     -[grad_phi - J^T y - (X-L)^{-1} mu e + (U-X)^{-1} mu e ; c - (y_k - y)/rho]
 *   K   (Eq. K1, unknown Delta x):
 *     J^T (y_k - rho c) - (grad_phi - (X-L)^{-1} mu e + (U-X)^{-1} mu e)
 * with the J values and rho (= rho-hat) of the current factorisation; an
 * infinite bound contributes no barrier term.  Sigma passed to the factor is
 * the caller's (X-L)^{-1} Z_l + (U-X)^{-1} Z_u (Section 3.1).
 *   mu  host double[count]: barrier parameter per instance (>= 0)
 *   B   device double[dim] (KKT row order of ncl_kkt_solve)
 * Errors: INVALID_ARG, STATE (no factor).
 */
ncl_status ncl_kkt_newton_rhs(ncl_kkt_t h, const ncl_kkt_newton_point* pt, const double* mu,
                              double* B, ncl_stream_t stream);

/*
 * ncl_kkt_newton_recover -- the full Newton direction from the solution X
 * (device double[dim]) of the system ncl_kkt_newton_rhs set up:
 *   dx  = Delta x
 *   dy  = Delta y: minus the dual block of X (K2r), or
 *         -rho (J Delta x + c) + y_k - y (K, Eq. K1 elimination)
 *   dr  = (Delta y - y_k + y)/rho - r                (Eq. K2 elimination)
 *   dz_lower = -(X-L)^{-1} (Z_l Delta x - mu e) - z_l
 *   dz_upper =  (U-X)^{-1} (Z_u Delta x + mu e) - z_u  (eliminated from Eq. K3)
 * dx, dz_lower, dz_upper: device double[n]; dy, dr: device double[m]; any
 * of them may be NULL.  Errors: INVALID_ARG, STATE (no factor).
 */
ncl_status ncl_kkt_newton_recover(ncl_kkt_t h, const ncl_kkt_newton_point* pt, const double* mu,
                                  const double* X, double* dx, double* dy, double* dr,
                                  double* dz_lower, double* dz_upper, ncl_stream_t stream);

/*
 * ncl_kkt_k1s_rhs -- the right-hand side of Eq. K1s for the current
 * condensed factorisation, as the elimination of Delta s in the proof of the
 * proposition (Section 3.3) produces it:
 *   OUT = RT + rho J_I^T (Sigma_s + rho I)^{-1} RS
 * (the statement of Eq. K1s prints it without (Sigma_s + rho I)^{-1}; the
 * proof's own steps, and the unreduced system they start from, give it
 * with).  Rows without slack contribute nothing.
 *   RT   device double, dim x nrhs column-major (ldt >= dim): r_t
 *   RS   device double, m x nrhs (ldr >= m): r_s
 *   OUT  device double, dim x nrhs (ldo >= dim); may be RT itself
 * Errors: INVALID_ARG, STATE (no factor).
 */
ncl_status ncl_kkt_k1s_rhs(ncl_kkt_t h, int32_t nrhs, const double* RT, int64_t ldt,
                           const double* RS, int64_t ldr, double* OUT, int64_t ldo,
                           ncl_stream_t stream);

/*
 * ncl_kkt_k1s_slack_step -- the eliminated slack step of Eq. K1s:
 *   Delta s_r = (rho (J Delta t)_r + r_s,r) / (Sigma_s,r + rho)
 * for each row with slack, 0 for a row without (Sigma_s = +inf), with the
 * Sigma_s and rho of the current factorisation (plain condensed factors: no
 * row has a slack).
 *   DT  device double, dim x nrhs column-major (ldt >= dim): Delta t
 *   RS  device double, m x nrhs (ldr >= m): r_s (read on rows with slack)
 *   DS  device double, m x nrhs (lds >= m): receives Delta s
 * Errors: INVALID_ARG, STATE (no factor).
 */
ncl_status ncl_kkt_k1s_slack_step(ncl_kkt_t h, int32_t nrhs, const double* DT, int64_t ldt,
                                  const double* RS, int64_t ldr, double* DS, int64_t lds,
                                  ncl_stream_t stream);

/*
 * ncl_kkt_factor_regularize -- the inertia correction of Section 3.1
 * (regularised matrix Eq. K2): factor with the primal regularisation
 * delta[i]; while instance i's inertia is not the regular one, (n_i, m_i, 0)
 * for K2r or (n_i, 0, 0) for K, raise delta[i] and refactor on the same
 * analysis.  As in Section 3.1 the regularisation also enters the penalty:
 * the matrix uses rho-hat_i = rho[i] + delta[i] (the dual block -1/rho-hat of
 * K2r, the rho-hat J^T J of K), so here rho[i] is the unregularised penalty.
 * Works on single and batch handles (count = 1 for a single handle).
 *   delta        host double[count]: in, the first delta of each instance
 *                (>= 0); out, the delta of the factors in use
 *   rho          host double[count], > 0
 *   delta_first  the delta tried after a zero one (> 0)
 *   growth       factor applied to a nonzero delta at each retry (> 1)
 *   max_tries    factorisations at most (>= 1)
 *   infos        host, may be NULL: the last factorisation's info per instance
 *   tries        host, may be NULL: the number of factorisations done
 * On an FP32_IR handle with precision_fallback, a try whose FP32 inertia is
 * irregular is refactored in FP64 before its inertia is trusted, so each
 * failed try costs an FP64 factorisation there; with precision_fallback = 0
 * the FP32 inertia decides.  The paper fixes no growth schedule.
 * Errors: INVALID_ARG (bad schedule or delta < 0), INERTIA (the factors of
 * the last try stay usable; delta holds its values), and those of
 * ncl_kkt_batch_factor.
 */
ncl_status ncl_kkt_factor_regularize(ncl_kkt_t h, const double* H_val, const double* J_val,
                                     const double* Sigma, double* delta, const double* rho,
                                     double delta_first, double growth, int32_t max_tries,
                                     ncl_stream_t stream, ncl_kkt_factor_info* infos,
                                     int32_t* tries);

/* Factor + solve in one call; with the same handle, values and nrhs the
 * whole sequence is one CUDA-graph launch after the first call.
 * sinfo->backward_err is the worst over instances. */
ncl_status ncl_kkt_batch_factor_solve(ncl_kkt_t h, const double* H_val, const double* J_val,
                                      const double* Sigma, const double* delta, const double* rho,
                                      int32_t nrhs, const double* B, int64_t ldb,
                                      double* X, int64_t ldx, ncl_stream_t stream,
                                      ncl_kkt_factor_info* infos, ncl_kkt_solve_info* sinfo);

/* Supernode partition of the permuted matrix: col0[s] is the first pivot of
 * supernode s (col0 host int32[ns+1], col0[ns] = dim), parent[s] its
 * parent in the assembly tree or -1 (host int32[ns]), nrow[s] the number of
 * rows of its front (host int32[ns]).  Any pointer may be NULL.  ns is
 * ncl_kkt_analysis_info.n_supernodes. */
ncl_status ncl_kkt_get_supernodes(ncl_kkt_t h, int32_t* col0, int32_t* parent, int32_t* nrow);

/* ------------------------------------------------------------------------
 * Diagnostics
 * ------------------------------------------------------------------------ */

/* Number of CUDA kernels the library has launched in this process. */
int64_t ncl_kkt_kernel_launches(void);

/* Per-kernel timing of a handle.  With enable = 1 every later factor/solve
 * call brackets each kernel launch with CUDA events on the call's stream
 * (this adds a little time per launch) and accumulates, per kernel name,
 * the launches, the summed device time and the kernel's arithmetic (flops
 * on the stored supernodal blocks) and minimum memory traffic (bytes).
 * enable = 0 stops recording; enable = -1 clears the totals. */
ncl_status ncl_kkt_profile(ncl_kkt_t h, int32_t enable);

/* Write the accumulated per-kernel totals as a JSON object
 * {"name": {"launches": L, "ms": T, "flops": F, "bytes": B}, ...} into buf
 * (NUL-terminated, truncated to buflen).  Returns NCL_OK. */
ncl_status ncl_kkt_profile_report(ncl_kkt_t h, char* buf, int64_t buflen);

/* Run the tensor-core (tcgen05, split-TF32) update kernel of the FP32
 * factorisation on caller data, for testing it in isolation:
 *   C[i][j] -= sum_{k<K} L[row_a+i][k] d[k] L[row_b+j][k],  0 <= j <= min(i, N-1), i < M
 * L: device float, rows x ld row-major (ld >= K, ld % 4 == 0); d: device
 * float[K]; C: device float, M x ldc row-major (only its lower part is
 * touched).  N <= M, row_a + M <= rows, row_b + N <= rows.  Allocates its own
 * temporary buffers; returns after completion.  INVALID_ARG, OOM, CUDA,
 * TIMEOUT. */
ncl_status ncl_kkt_selftest_tensor_update(int32_t rows, int32_t ld, int32_t K, const float* L,
                                          const float* d, int32_t row_a, int32_t row_b, int32_t M,
                                          int32_t N, float* C, int32_t ldc, ncl_stream_t stream);

/* Make one bounded inter-CTA wait of a real kernel run out, to test the
 * failure path of options.wait_cycles without faulting or hanging anything:
 *   which = 0: the forward sweep's chain kernel on the block-rows of a
 *              supernode with more than one block-row (needs a factored
 *              handle); its ticket counter starts past block-row 0, so that
 *              block-row's flag is never published and the next one's CTA
 *              waits for it;
 *   which = 1: the first macro panel with rows below it; its ticket counter
 *              starts past the diagonal role, so the row CTAs wait for
 *              sub-block flags that are never published.  The handle's
 *              factors are void afterwards (factor again before solving).
 * Every wait of that launch is bounded by wait_cycles (> 0) SM clock cycles;
 * the kernel then finishes without the awaited data.  Returns
 * NCL_ERR_TIMEOUT when the wait ran out (the expected outcome), NCL_OK if it
 * did not, INVALID_ARG when the handle has no such supernode or panel, STATE
 * for a sweep test before a factor.  The error flags are cleared afterwards. */
ncl_status ncl_kkt_selftest_wait_timeout(ncl_kkt_t h, int32_t which, int64_t wait_cycles,
                                         ncl_stream_t stream);

/* Number of instances of a handle (1 for ncl_kkt_analyze). */
int32_t ncl_kkt_instance_count(ncl_kkt_t h);

#ifdef __cplusplus
}
#endif
#endif /* NCL_KKT_H */
