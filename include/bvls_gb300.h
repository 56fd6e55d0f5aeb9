/*
 * bvls_gb300.h -- C ABI of a GB300 (sm_103a) solver for box-constrained least squares
 * with dynamic Gap safe screening.
 *
 * Problem (Dantas, Soubies, Fevotte, "Accelerating Non-Negative and Bounded-Variable
 * Linear Regression Algorithms with Safe Screening", Section 2, Eq. (LR) with the
 * least-squares loss of Section 5):
 *
 *     x* in argmin_x 1/2 ||y - A x||_2^2   subject to  l <= x <= u,
 *
 * with l finite and u in R or +inf (NNLS: l = 0, u = +inf; BVLS: every u finite).
 *
 * The solver is an accelerated projected-gradient iteration (FISTA with gradient-based
 * adaptive restart) into which the screening procedure of Algorithm 1 (Algorithm 2 for
 * NNLS) is fused: the dual point of Section 4 (Eq. (BVLR_dual_up) for BVLS, the dual
 * translation of Eq. (BVLR_dual_up2) when some u_j = +inf), the duality gap of
 * Eq. (Dual_Gap), the Gap safe radius of Eq. (GAP_Safe_sph) and the sphere test of
 * Eq. (safe_rule), which fixes coordinates at their bounds and removes their columns from
 * every later product (Eq. (decmposition_fwd)).
 *
 * Conventions shared by every entry point
 *   - Matrices are column-major float32: column j of A starts at A + j*lda, lda >= m.
 *   - Pointers documented as "any" may point to device memory, pinned host memory or
 *     pageable host memory; the library copies through the CUDA runtime with unified
 *     addressing.  Pointers documented as "host" must be host memory.
 *   - The caller owns every pointer it passes; the library keeps no reference to a
 *     caller pointer after the call returns.  The handle owns its device workspace,
 *     including its own padded copy of A.
 *   - All device work of a handle is enqueued on the stream given to bvls_setup, in order
 *     after the work already queued there.  For stream 0 (the legacy default stream, which
 *     cannot be captured into a CUDA graph) the handle uses a stream of its own, ordered
 *     after the legacy stream by an event.  bvls_solve returns when its results are in the
 *     caller's buffers.
 *   - Every call returns a bvls_status and never aborts the process.  On BVLS_EINVAL,
 *     BVLS_ENONFINITE and BVLS_ENOTSUP nothing is written to the outputs.
 *     bvls_last_error() describes the last failure on the calling thread.
 *   - A handle may be used by one host thread at a time.
 */
#ifndef BVLS_GB300_H
#define BVLS_GB300_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define BVLS_API __attribute__((visibility("default")))
#else
#define BVLS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bvls_handle bvls_handle;

typedef enum {
  BVLS_OK = 0,
  BVLS_EINVAL = 1,      /* invalid argument (sizes, bounds with l > u or l not finite, ...) */
  BVLS_ENOMEM = 2,      /* a device allocation failed */
  BVLS_ECUDA = 3,       /* a CUDA runtime call failed */
  BVLS_EMAXITER = 4,    /* max_iter reached with gap >= tol; outputs hold the last evaluated
                           iterate, its gap and its screened set */
  BVLS_ENONFINITE = 5,  /* NaN or Inf found in A, y or x0 */
  BVLS_ENOTSUP = 6,     /* sizes beyond what this build supports (see bvls_setup) */
  BVLS_ETIMEOUT = 7     /* a bounded device-side wait gave up (about 2 s); outputs untouched */
} bvls_status;

/* Arithmetic of the two products over the preserved columns. */
enum {
  BVLS_PREC_FP32X2 = 0, /* float32 data, error-free products and double-float (about 48-bit)
                           accumulation; default */
  BVLS_PREC_FP32 = 1,   /* float32 data and plain float32 accumulation; faster, and the
                           rounding margins of the test are about 2^24 times wider */
  BVLS_PREC_MIXED = 2   /* float32 correlations a_j^T r; forward product A x with float32
                           sums over groups of at most 8 columns merged in double-float
                           (bvls_solve, bvls_solve_static): the residual, P(x) and the
                           certificate of the zero dual point are good to about 9 u relative
                           to sum_j |a_ij x_j| (FP32: about u per column); the correlations and
                           the screening margins are those of FP32.  bvls_solve_batched treats
                           it as FP32 */
};

/* Primal solver of bvls_solve. */
enum {
  BVLS_ALG_FISTA = 0,          /* accelerated projected gradient with adaptive restart (default) */
  BVLS_ALG_CHAMBOLLE_POCK = 1  /* the primal-dual iteration of Section 5's BVLS experiments
                                  (sigma = tau = 0.99 / sqrt(L)); screening uses its own dual
                                  iterate theta = -z.  BVLS only (every u_j finite), single-pass
                                  form, no dual_point; else BVLS_ENOTSUP */
};

/* Dual point used by the screening step (Section 4). */
enum {
  BVLS_DUAL_SCALING = 0,     /* every u_j finite: theta = y - A x (Eq. (BVLR_dual_up)) */
  BVLS_DUAL_TRANSLATION = 1, /* some u_j = +inf: theta = Xi_t(y - A x) (Eq. (BVLR_dual_up2)) */
  BVLS_DUAL_ZERO = 2         /* some u_j = +inf and no interior direction t was found:
                                theta = 0, the gap is P(x) and nothing is screened */
};

typedef struct {
  double tol;         /* stop when the gap bound < tol (absolute; Algorithm 1's until test) */
  int screen_every;   /* K >= 1: the gap and the screening step run every K iterations */
  int max_iter;       /* >= 1; rounded up to a multiple of screen_every */
  int screening;      /* 1: Algorithm 1; 0: the same iteration and gap with nothing fixed */
  int precision;      /* BVLS_PREC_* */
  int restart;        /* 1: gradient-based adaptive restart of the momentum */
  double lipschitz;   /* > 0: use this step constant L instead of the one from bvls_setup */
  int profile;        /* 1: time every product kernel with CUDA events (one chunk of
                         iterations captured into a plain graph with event nodes; fills the
                         *_ms fields of bvls_info); 2 (bvls_solve): launch every kernel directly
                         from the host, a chunk at a time, with no CUDA graph and no events */
  int single_pass;    /* 1 (default): when m <= 8192, one streaming read of the preserved
                         columns per iteration yields both products, and the K iterations
                         between two gap evaluations run in one persistent (cooperative)
                         launch when its shape fits one CTA per SM; 2: the same single pass
                         with two launches per iteration (pass, residual); 0: two passes
                         (A_S x_S, then A_S^T r), the form used for larger m */
  const double* dual_point; /* any; m doubles or NULL (default).  A fixed dual point used by
                         every screening step of bvls_solve in place of Theta(x_k): the
                         oracle-dual-point experiment of Section 5, where theta* informs the
                         test.  Translated into F_D along t when some a_j^T theta > 0 with
                         u_j = +inf; any dual-feasible point keeps the test safe.  Needs the
                         single-pass form and a dual mode other than BVLS_DUAL_ZERO
                         (else BVLS_ENOTSUP / BVLS_EINVAL).  Ignored by the other entry points. */
  int algorithm;      /* BVLS_ALG_*; bvls_solve only (the other entry points use FISTA) */
  int refine;         /* 1: after the solve, refine the returned x on its free set (the
                         optimality conditions of Section 3.2, Eq. (optimality2)): the
                         coordinates strictly inside the box solve the restricted normal
                         equations A_F^T A_F x_F = A_F^T (y - A_B x_B), by rounds of float64
                         residuals and float32 conjugate-gradient corrections; a coordinate
                         that leaves the box stops on its bound, a coordinate at a bound whose
                         a_j^T (y - A x) has the wrong sign joins F.  The refined x is returned
                         only when every preserved coordinate passes its optimality test within
                         the rounding bound of that test (eta_j = ||a_j|| (gamma ||r|| + ||e_r||),
                         plus 1e-12 ||a_j|| ||r|| of stationarity on F); otherwise the solver's
                         iterate is returned unchanged.  Coordinates fixed by the safe rule stay
                         at their bounds.  Declined when m > 8192, when |F| > min(m, 2048) (A_F
                         cannot have full column rank: the optimum is not unique) or after 10
                         rounds.  bvls_solve, bvls_solve_batched, bvls_solve_ragged; 0 (default):
                         off.  The gap fields keep the solver's certificate. */
} bvls_opts;

typedef struct {
  int iters;            /* iterations run (gradient evaluations) */
  int converged;        /* 1 when gap < tol */
  int n_preserved;      /* |preserved set| at the end */
  int dual_mode;        /* BVLS_DUAL_* */
  int gap_evals;        /* screening / gap evaluations */
  double gap;           /* rigorous upper bound of the duality gap at the returned x */
  double primal;        /* 1/2 ||y - A x||^2 at the iterate of the last gap evaluation, before
                           that evaluation set its screened coordinates to their bounds */
  double radius;        /* Gap safe radius of the last evaluation */
  double L;             /* step constant used */
  double sum_preserved; /* sum over iterations of |preserved set|: columns read by A_S^T r */
  double sum_nonzero;   /* sum over iterations of the preserved x_j != 0: columns read by
                           A_S x_S (zero coordinates contribute nothing and are skipped) */
  double fwd_ms, tr_ms; /* profile mode, total kernel time.  Persistent single pass: tr_ms =
                           the launches that run K iterations each (tr_launches of them),
                           fwd_ms = 0.  Single pass with two launches per iteration: tr_ms =
                           the pass that reads A_S once for both products, fwd_ms = the
                           residual kernel r = y' - q.  Two-pass iteration: fwd_ms = A_S x_S,
                           tr_ms = A_S^T r. */
  int fwd_launches, tr_launches;
  double kernel_launches; /* kernels this call launched (including ones that found the solve
                             already stopped and returned at entry) */
  int single_pass;        /* form of the iterations (see bvls_opts): 0 two passes, 1 single pass
                             with two launches per iteration, 2 single pass, persistent */
  int refined;            /* opts.refine: 1 when the refined x was returned */
  int refine_rounds;      /* refinement rounds run (each: float64 residual and correlations,
                             then a float32 correction on F) */
  int n_free;             /* |F| of the last refinement round */
  int refine_cg_iters;    /* conjugate-gradient iterations over all rounds */
  double kkt;             /* refinement: max over the preserved j of
                             |x_j - clip(x_j + a_j^T (y - A x), l_j, u_j)| at the returned x
                             (0 at an optimum; float64 evaluation) */
  double refine_ms;       /* refinement kernel time (CUDA events) */
  int refine_reason;      /* 0 refined or off, 1 declined after the last round, 2 declined
                             because |F| > min(m, 2048), 3 declined because m > 8192 */
  int t_choice;           /* translation direction t of the handle (Section 4.2): 0 the
                             caller's, 1 t = -1 (Proposition 2, case 3), 2 minus the mean column,
                             3 minus the column most correlated with all others, 4 the
                             least-squares solution of A^T t = -1 (Proposition 2, case 1);
                             -1 none (BVLS_DUAL_SCALING or BVLS_DUAL_ZERO) */
} bvls_info;

/* Fill *opts with the defaults: tol 1e-6, screen_every 10, max_iter 100000, screening 1,
   precision BVLS_PREC_FP32X2, restart 1, lipschitz 0 (use setup's), profile 0,
   single_pass 1, dual_point NULL, algorithm BVLS_ALG_FISTA, refine 0. */
BVLS_API void bvls_default_opts(bvls_opts* opts);

/*
 * Prepare a solver for the matrix A and the box [l, u].
 *   A       any; m x n column-major float32 with leading dimension lda >= m.  Copied into a
 *           handle-owned layout padded to a multiple of 32 rows.
 *   l, u    host; n doubles each, or NULL for l = 0 / u = +inf.  l must be finite, u may
 *           be +INFINITY, l_j <= u_j.
 *   t       host; m doubles: the translation direction of Section 4.2 for the columns
 *           with u_j = +inf, or NULL to choose one (t = -1, then minus the mean column,
 *           then minus the column most correlated with all others, per Proposition 2 and
 *           the choices of Section 5, then, when n <= m and n <= 1024, the least-squares
 *           solution of A^T t = -1 of Proposition 2, case 1, by float64 conjugate gradients
 *           on A^T A).  A given t must satisfy a_j^T t < 0 on every nonzero column with
 *           u_j = +inf, else BVLS_EINVAL.
 *   stream  a cudaStream_t (0 = legacy default stream).
 *   out     receives the handle.
 * Setup computes the column norms ||a_j||_2 (used by Eq. (safe_rule)), w = A^T t and the
 * step constant L (1.05 x the largest Ritz value of 20 Lanczos steps on A^T A, an estimate of
 * ||A||_2^2 from below; 100 power steps where the one-launch form does not fit).
 * Limits: 1 <= m <= 24576 (the residual is staged in shared memory), 1 <= n < 2^31,
 * lda*n*4 bytes addressable.  Errors: EINVAL, ENOTSUP, ENOMEM, ECUDA, ENONFINITE (A).
 */
BVLS_API bvls_status bvls_setup(const float* A, int m, int n, int lda, const double* l,
                       const double* u, const double* t, void* stream, bvls_handle** out);

/*
 * Solve for one right-hand side y with the handle's A and box.
 *   y             any; m float32.
 *   x0            any; n doubles, the starting point (projected onto [l, u]), or NULL for
 *                 the projection of 0 (Algorithm 1: initialise x in [l, u]).
 *   opts          host; NULL for the defaults.
 *   x_out         any; n doubles: the iterate at which the final gap was evaluated, with
 *                 every screened coordinate at its bound.
 *   screened_out  any; n bytes or NULL: 0 preserved, 1 fixed at l_j, 2 fixed at u_j.
 *   info          host; or NULL.
 * Returns BVLS_OK when the gap bound fell below tol, BVLS_EMAXITER otherwise (outputs
 * valid), or an error (outputs untouched).
 */
BVLS_API bvls_status bvls_solve(bvls_handle* h, const float* y, const double* x0, const bvls_opts* opts,
                       double* x_out, uint8_t* screened_out, bvls_info* info);

typedef struct {
  int iters_max;          /* largest per-instance iteration count */
  int n_converged;        /* instances with gap < tol */
  int gap_evals;          /* evaluations run (each covers every instance still active) */
  int dual_mode;          /* BVLS_DUAL_* */
  double L;               /* step constant used */
  double sum_step;        /* sum over tensor-core steps of the instances they advanced */
  double sum_eval;        /* sum over evaluations of the instances they covered */
  double sum_preserved;   /* sum over evaluations and instances of |preserved set| */
  double step_ms, eval_ms;  /* profile mode: total time of the step / evaluation kernels */
  int step_launches, eval_launches;
  double kernel_launches; /* kernels this call launched (including ones that returned at
                             entry because every instance had finished) */
  int n_refined;          /* opts.refine: instances whose refined x was returned */
  int refine_free_max;    /* largest |F| of a refined instance */
  double kkt_max;         /* largest kkt (see bvls_info) over the refined instances */
  double refine_ms;       /* refinement kernel time (CUDA events) */
  int refine_out_of_rounds; /* instances declined after the last round */
  int refine_not_unique;    /* instances declined because |F| > min(m, 2048) */
  int steps_persistent;     /* 1: the K - 1 tensor-core steps between two evaluations ran as
                               one cluster launch with the iteration state on chip */
  int pad0;
} bvls_batch_info;

/*
 * Solve B problems that share the handle's A and box: x_b* in argmin 1/2 ||y_b - A x||^2,
 * l <= x <= u, each with its own screened set, gap and stop (Algorithm 1 per instance).
 * The instances advance in lockstep; each leaves the active set at the first evaluation
 * whose gap bound is below tol.
 *   Y             any; B rows of m float32, row b at Y + b*ldy (ldy >= m).
 *   X0            any; B x n doubles (row b = instance b) or NULL for the projection of 0.
 *   opts          host or NULL.  screen_every = K: every K-th iteration (k = 0, K, 2K, ...)
 *                 is an evaluation: exact correlations g = A^T (y - A x_k) with float32
 *                 (BVLS_PREC_FP32) or double-float (BVLS_PREC_FP32X2) products, the gap,
 *                 the sphere test and the stop test.  The other iterations are tensor-core
 *                 steps: g_k = g_{k-1} - bf16(A^T A) bf16(x_k - x_{k-1}) for all active
 *                 instances in one tcgen05 GEMM with float32 accumulation, whose momentum
 *                 term also takes bf16(x_k - x_{k-1}).  max_iter is rounded up to a
 *                 multiple of K.  single_pass 1 (default) runs the K - 1 steps between two
 *                 evaluations as one launch of clusters of npad / 128 CTAs that keep x, g
 *                 and bf16(x_k - x_{k-1}) in tensor and shared memory (when npad <= 512);
 *                 0 or 2: one launch per step.  Both give the same iterates.
 *   X_out         any; B x n doubles: per instance, the iterate of its last evaluation with
 *                 screened coordinates at their bounds.
 *   screened_out  any; B x n bytes or NULL (0 preserved, 1 at l_j, 2 at u_j).
 *   gaps_out      any; B doubles or NULL: the gap bound at X_out.
 *   iters_out     any; B ints or NULL: the iteration index of that evaluation.
 *   status_out    any; B ints or NULL: BVLS_OK or BVLS_EMAXITER per instance.
 *   info          host or NULL.
 * The iterates are double-float pairs of float32 (about 48 significant bits), clipped to
 * the bounds in the same form; the gap, the radius and the test bound the rounding of
 * every evaluation product, so no coordinate is fixed unless the safe rule holds for the
 * exact problem.  Limits: m <= 1024, n <= 4096, 1 <= B <= 2^20.  The first call computes
 * and keeps bf16(A^T A) (n rounded up to 128 = npad, squared, 2 bytes each) and a
 * workspace of about 37 * B * npad + 8 * B * n bytes, reused by later calls with the same
 * or smaller B.
 * Returns BVLS_OK when every instance converged, BVLS_EMAXITER otherwise (all outputs
 * valid), or an error (outputs untouched).
 */
BVLS_API bvls_status bvls_solve_batched(bvls_handle* h, int B, const float* Y, int ldy, const double* X0,
                                        const bvls_opts* opts, double* X_out, uint8_t* screened_out,
                                        double* gaps_out, int* iters_out, int* status_out,
                                        bvls_batch_info* info);

typedef struct {
  double free_tol;      /* free set: l_j + free_tol (1 + |l_j|) < x_j < u_j - free_tol (1 + |u_j|);
                           default 1e-9 */
  double cg_tol;        /* CG stops when ||A_F^T A_F w - v_F|| <= cg_tol ||v_F||; default 1e-12 */
  int cg_max_iter;      /* CG iteration limit per instance; default 4000 */
} bvls_backward_opts;

typedef struct {
  int n_converged;      /* instances whose CG met cg_tol */
  int n_iter_limit;     /* instances that stopped at cg_max_iter (gradients approximate) */
  int n_too_large;      /* instances whose free set exceeds 1024 (zero gradients returned) */
  int n_not_unique;     /* instances whose free set exceeds m (zero gradients returned) */
  int max_free;         /* largest free set */
  int max_cg_iters;     /* most CG iterations of an instance */
  double cg_work;       /* sum over instances of CG iterations x |F| (each iteration applies
                           A_F^T A_F: 4 m |F| float64 flops) */
  double kernel_ms;     /* device time of the backward kernels (CUDA events) */
} bvls_backward_info;

/* Fill *opts with the defaults above. */
BVLS_API void bvls_backward_default_opts(bvls_backward_opts* opts);

/*
 * Gradients of a loss L(x*) through the solution map (y, A) -> x*(y, A) for B instances
 * that share the handle's A and box.  The paper has no backward pass; this follows from
 * the optimality conditions of Section 3.2: at a non-degenerate optimum (strict
 * complementarity, A_F of full column rank on the free set F) the coordinates outside F
 * sit at their bounds and x_F solves the restricted normal equations
 * A_F^T A_F x_F = A_F^T (y - A_B x_B).  With v = dL/dx and w = (A_F^T A_F)^{-1} v_F (zero
 * off F, found by conjugate gradients on the free set, float64):
 *     dL/dy_b = A_F w_b,     dL/dA = sum_b  r_b w_b^T - (A_F w_b) x_b^T,   r_b = y_b - A x_b.
 * Components of dL/dx on the fixed coordinates do not flow back.
 *   X        any; B x n doubles: the solutions (e.g. X_out of bvls_solve_batched).
 *   Y        any; B rows of m float32 at Y + b*ldy (ldy >= m): the right-hand sides.
 *   dLdX     any; B x n doubles.
 *   opts     host or NULL (defaults).
 *   dLdY     any; B x m doubles, or NULL.
 *   dLdA     any; m x n doubles, column-major (leading dimension m), summed over the batch,
 *            or NULL.
 *   status_out  any; B ints or NULL: 0 CG converged, 1 CG iteration limit, 2 free set
 *            larger than 1024, 3 free set larger than m (A_F cannot have full column rank:
 *            the optimum is not unique and has no derivative); with 2 and 3 that instance
 *            contributes zero gradients and runs no CG.
 *   info     host or NULL.
 * Limits: m <= 24576 (the handle's limit); free sets up to 1024 coordinates.  Returns
 * BVLS_OK, or an error (EINVAL, ENOMEM, ECUDA; outputs untouched).
 */
BVLS_API bvls_status bvls_backward(bvls_handle* h, int B, const double* X, const float* Y, int ldy,
                                   const double* dLdX, const bvls_backward_opts* opts, double* dLdY,
                                   double* dLdA, int* status_out, bvls_backward_info* info);

/* One problem of a ragged batch (bvls_solve_ragged). */
typedef struct {
  const float* A;       /* any; m x n column-major float32, leading dimension lda >= m */
  int m, n, lda;
  const float* y;       /* any; m float32 */
  const double* l;      /* host; n doubles or NULL (0) */
  const double* u;      /* host; n doubles or NULL (+inf); u_j may be +INFINITY */
} bvls_problem;

typedef struct {
  int iters_max;        /* largest per-instance iteration count */
  int n_converged;      /* instances with gap < tol */
  int n_translation;    /* instances screened with the dual translation (t = -1) */
  int n_zero;           /* instances with u_j = +inf and no interior t = -1: theta = 0 */
  int chunks;           /* chunks of iterations the device loop ran */
  int tiles_max;        /* work-list capacity (sum over instances of ceil(n / 8)) */
  double setup_ms;      /* copies, column norms, dual modes, 40 power iterations, autotuner */
  double solve_ms;      /* the solve graph (host wall clock around one graph launch) */
  int tile_cols;        /* columns per tile of the work list (8, 16 or 32), picked by timing */
  int screen_every;     /* the screening period used (the autotuner's when opts->screen_every = 0) */
  int tuned;            /* 1 when this call ran the autotuner (the choice is kept for later calls
                           on a batch of the same shape) */
  double tune_ms;       /* autotuner time (part of setup_ms) */
  int n_refined;        /* opts.refine: instances whose refined x was returned */
  int refine_free_max;  /* largest |F| of a refined instance */
  double kkt_max;       /* largest kkt (see bvls_info) over the refined instances */
  double refine_ms;     /* refinement kernel time (CUDA events) */
  int refine_out_of_rounds; /* instances declined after the last round */
  int refine_not_unique;    /* instances declined because |F| > min(m, 2048) */
  double sum_rows_cols;     /* sum over the solve's iterations and active instances of
                               m_k |S_k|: the elements of A_k read (4 bytes each) */
} bvls_ragged_info;

/*
 * Solve B independent problems of uneven sizes, each with its own A_k, y_k and box, in one
 * set of launches per iteration (Algorithm 1 per instance, lockstep iterations, retirement of
 * finished instances): the mixed NNLS / BVLS batch.  Per instance: the step constant is
 * 1.05 x a 40-step power-iteration estimate of ||A_k||_2^2; the dual point is the scaling
 * (every u_j finite), the translation with t = -1 when it is interior (Proposition 2), else
 * theta = 0.  Products are float32 data with double-float accumulation.
 *   probs         host; B problem descriptors (1 <= m_k <= 1024, n_k >= 1).
 *   opts          host or NULL: tol, screen_every, max_iter, screening, restart, refine and
 *                 profile (2: every kernel launched directly, no CUDA graph) are used;
 *                 screen_every = 0 lets the autotuner pick it from {5, 10, 20} by timing 20
 *                 iterations of each from the start point.  The tile width of the work list
 *                 is always picked by timing eight iterations with 8, 16 and 32 columns (the
 *                 iterates do not depend on it).  Choices are kept per batch shape for the
 *                 life of the process.
 *   stream        a cudaStream_t (0 allowed); the call returns when its outputs are written.
 *   x_out         host; B pointers (any memory) to n_k doubles each.
 *   screened_out  host; B pointers (any memory) to n_k bytes, or NULL.
 *   gaps_out, iters_out, status_out: host; B entries each, or NULL.
 *   info          host or NULL.
 * The call allocates its workspace (the A_k copies padded to a multiple of 4 rows, about 60
 * bytes per column and 40 bytes per row) and frees it before returning.
 * Returns BVLS_OK when every instance converged, BVLS_EMAXITER otherwise (outputs valid),
 * or an error (EINVAL, ENOTSUP, ENONFINITE, ENOMEM, ECUDA; outputs untouched).
 */
BVLS_API bvls_status bvls_solve_ragged(int B, const bvls_problem* probs, const bvls_opts* opts, void* stream,
                                       double* const* x_out, uint8_t* const* screened_out, double* gaps_out,
                                       int* iters_out, int* status_out, bvls_ragged_info* info);

/*
 * One-call solve that allocates nothing.  The paper has no counterpart: this is a service
 * for callers that cannot allocate device memory -- code that runs inside a memory pool or
 * allocator it does not own, or a plug-in whose host application forbids allocations after
 * start-up.  It uses the same per-iteration kernels as bvls_setup + bvls_solve, launched one
 * by one (the single pass and its residual, or the two passes, then the gap, test and
 * compaction kernels); the step constant comes from power steps, and neither the persistent
 * form nor CUDA graphs are used.  All scratch lives in one static device array of 8 MiB that
 * every GPU loading this library holds until the process exits; no cudaMalloc, cudaFree,
 * pinned host memory, CUDA graph or event is created.
 *   A             device memory, column-major float32, read in place; lda a multiple of 32;
 *                 rows m..lda-1 of each column are read and must be finite (zero them).
 *   l, u          host; n doubles or NULL (0 / +inf), as in bvls_setup.
 *   y             any; m float32.  x0: any; n doubles or NULL.
 *   opts          host or NULL (defaults).  opts->profile, opts->dual_point and opts->refine
 *                 are ignored; only FISTA runs here (another opts->algorithm gets
 *                 BVLS_ENOTSUP).
 *   stream        a cudaStream_t (0 allowed); the call returns when its outputs are written.
 *   x_out, screened_out, info: as in bvls_solve.
 * Limits: m <= 4096, n <= 16384 and a scratch layout that fits the 8 MiB array; larger
 * problems get BVLS_ENOTSUP with the size in bvls_last_error() (use bvls_setup then).
 * The translation direction for columns with u_j = +inf is t = -1 when it is interior,
 * else theta = 0 (bvls_setup also tries further candidates).  The step constant comes from
 * opts->lipschitz when > 0, else from 1.05 x a 101-step power-iteration estimate of ||A||_2^2.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current and keeps it for later calls on that device.  Every call
 * reuses the same array, which keeps the previous call's contents (each call clears what
 * must start at zero); calls whose GPU work overlaps -- from two threads or on two streams
 * -- race on it and must be serialised by the caller.
 */
BVLS_API bvls_status bvls_solve_static(const float* A, int m, int n, int lda, const double* l,
                                       const double* u, const float* y, const double* x0,
                                       const bvls_opts* opts, void* stream, double* x_out,
                                       uint8_t* screened_out, bvls_info* info);

/*
 * Testing hook of the failure path; the paper has no counterpart.  Sets the bound, in SM
 * clock cycles, of the grid-barrier waits of bvls_solve's persistent pass on this handle
 * (cycles <= 0 restores the default of 4e9 cycles, about 2 s).  A wait that runs out records
 * an error instead of waiting on: every CTA leaves its iteration loop at its next barrier,
 * after the bulk copies it has issued have landed, and bvls_solve returns BVLS_ETIMEOUT with
 * the outputs untouched; the handle stays usable.  A bound far below the time of one
 * iteration makes every solve in the persistent form time out: the hook exists so that tests
 * can drive that path without a GPU fault.  Discards the handle's cached solve graphs.
 */
BVLS_API bvls_status bvls_set_grid_wait(bvls_handle* h, long long cycles);

/* Release the handle and its device memory (NULL is ignored). */
BVLS_API void bvls_destroy(bvls_handle* h);

/* Text of the last error recorded on the calling thread ("" if none). */
BVLS_API const char* bvls_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* BVLS_GB300_H */
