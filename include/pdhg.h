/*
 * pdhg.h -- C ABI of the GB300 PDHG solver for LP relaxations of DC unit
 * commitment (sm_103a CUDA kernels; no host fallback).
 *
 * Method.  The paper solves the relaxed UC LP with the Primal-Dual Hybrid
 * Gradient method (Sec. II.E):  x+ = proj(x + tau A^T y - tau c),
 * y+ = y - sigma A (2x+ - x) + sigma b, with the adaptive step sizes and
 * restarts of Applegate et al. that it cites there.  Its LP statement
 * (min c^T x, Ax <= b, x >= 0, Sec. II.E) is sign-inconsistent with its saddle
 * function and lacks the dual projection; this library uses the PDLP general
 * form the cited method is defined on:
 *
 *     min c^T x  s.t.  K_i x = q_i (i < m_eq),  K_i x >= q_i (i >= m_eq),
 *                      l <= x <= u                 (entries may be +-INFINITY)
 *     L(x, y) = c^T x - y^T (K x - q),  y_i free (i < m_eq),  y_i >= 0 (i >= m_eq)
 *
 * Optimality is measured on the unscaled LP in FP64 (Sec. III.B names the log
 * quantities: primal and dual objective, primal and dual residual, gap):
 *     rel_p   = ||r_p||_2 / (1 + ||q||_2),   r_p = q - Kx (eq), (q - Kx)^+ (>=)
 *     rel_d   = ||r_d||_2 / (1 + ||c||_2),   r_d = lambda - proj(lambda),
 *               lambda = c - K^T y, proj keeps the sign each finite bound allows
 *     rel_gap = |P - D| / (1 + |P| + |D|),   P = c^T x,
 *               D = q^T y + sum_j (l_j lambda_j^+ - u_j lambda_j^-)
 *     rel_kkt = max(rel_p, rel_d, rel_gap)
 *
 * Conventions for every entry point.
 *   - Pointers documented "device" must be device memory of the current CUDA
 *     device; "host" pointers are host memory.  The caller owns every input and
 *     output buffer; the workspace owns its internal buffers.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     All device work of a call is enqueued on it.  Calls that return results
 *     in host structs synchronise that stream before returning.
 *   - Return value: PDHG_OK (0) or a negative PDHG_ERR_* code; the message of
 *     the last failure on the calling thread is in pdhg_last_error().
 *   - A workspace is not thread safe; use one per host thread.
 */
#ifndef PDHG_H
#define PDHG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* error codes (return values) */
#define PDHG_OK 0
#define PDHG_ERR_INVALID_ARG (-1) /* bad pointer, size, or option             */
#define PDHG_ERR_CUDA (-2)        /* a CUDA runtime call failed                */
#define PDHG_ERR_NUMERIC (-3)     /* NaN/Inf in the data or the iterates       */
#define PDHG_ERR_TIMEOUT (-4)     /* a bounded device wait gave up             */
#define PDHG_ERR_UNSUPPORTED (-5) /* size or mode not supported (e.g. > 2^31)  */
#define PDHG_ERR_NOMEM (-6)       /* device or host allocation failed          */

/* solver outcome (pdhg_result.status) */
#define PDHG_STATUS_OPTIMAL 1    /* rel_kkt <= tol                              */
#define PDHG_STATUS_ITER_LIMIT 2 /* max_iters attempts done                     */
#define PDHG_STATUS_TIME_LIMIT 3 /* time_limit_s reached (device clock)         */
#define PDHG_STATUS_CANCELLED 4  /* *cancel_flag became nonzero                 */
#define PDHG_STATUS_NUMERIC 5    /* NaN/Inf met in a KKT evaluation             */
#define PDHG_STATUS_PRIMAL_INFEASIBLE 6 /* a dual ray certifies that no x exists  */
#define PDHG_STATUS_DUAL_INFEASIBLE 7   /* a primal ray certifies an unbounded LP */

/* arithmetic of the iterations (KKT, restart and gap reductions are FP64 always) */
#define PDHG_PREC_FP64 0  /* FP64 matrix, iterates and accumulation            */
#define PDHG_PREC_MIXED 1 /* FP32 matrix/iterates + FP64 iterative refinement   */

/* The LP, as device pointers in the caller's memory (read, never written).
 * CSR of K with ascending column indices in each row, no duplicates.
 * Sizes: n, m >= 1, 0 <= m_eq <= m, nnz < 2^31, n, m < 2^31. */
typedef struct pdhg_problem {
  int64_t n, m, m_eq, nnz;
  const int64_t *row_ptr; /* device [m+1] */
  const int32_t *col;     /* device [nnz] */
  const double *val;      /* device [nnz] */
  const double *c;        /* device [n]   */
  const double *l;        /* device [n]   */
  const double *u;        /* device [n]   */
  const double *q;        /* device [m]   */
} pdhg_problem;

/* Options.  pdhg_opts_default fills the values listed in the comments. */
typedef struct pdhg_opts {
  double tol;               /* target rel_kkt (1e-8)                                  */
  int32_t precision;        /* PDHG_PREC_FP64 / PDHG_PREC_MIXED (FP64)                */
  int32_t check_every;      /* attempts between KKT checks; fixed at 64               */
  int64_t max_iters;        /* cap on step attempts, all refinement rounds (10^7)     */
  double time_limit_s;      /* wall limit on the device clock (600)                   */
  double beta_sufficient;   /* restart if KKT_w(cand) <= 0.2 KKT_w(last restart)      */
  double beta_necessary;    /* ... or <= 0.8 and increased since the last check       */
  double beta_artificial;   /* ... or attempts since restart >= 0.36 of all attempts  */
  double omega_smoothing;   /* primal weight smoothing theta (0.5)                    */
  double step_reduction_exp; /* eta' = min((1-(k+1)^-0.3) eta_max, ...) (0.3)         */
  double step_growth_exp;    /* ... (1+(k+1)^-0.6) eta) (0.6)                         */
  int32_t ruiz_iters;       /* Ruiz l_inf passes (10)                                 */
  int32_t pock_chambolle;   /* 1: one Pock-Chambolle alpha=1 pass (1)                 */
  double ir_reduction;      /* mixed: a refinement round ends at a check (without a
                               restart) whose current iterate has rel_kkt <=
                               ir_reduction x that of the round's start; pdhg_solve
                               folds the iterate into x*, y* in FP64 and continues
                               the same iteration in rescaled coordinates (0.5)      */
  int32_t ir_max_rounds;    /* mixed: refinement rounds after the first (100000)      */
  int32_t trace;            /* 1: record per-attempt/per-check trace (testing) (0)    */
  double fixed_eta;         /* > 0: constant steps eta/omega, no restarts (0)         */
  double fixed_omega;       /* primal weight in fixed-step mode                       */
  int32_t bound_obj_rescale; /* 1: also scale q, l, u by 1/(1+||q~||) and c by
                                1/(1+||c~||) after Ruiz + Pock-Chambolle (0)          */
  int32_t artificial_total; /* 1: the artificial restart compares with the attempts of
                               all refinement rounds, not the current round's (1)     */
  int32_t host_loop;        /* 1: launch each 64-attempt body from the host and read the
                               done flag after every check instead of one CUDA graph
                               with a device-side while loop (for profilers) (0)      */
  int32_t autotune;         /* 1: time the launch variants of the per-attempt kernels
                               at the first solve of each precision and keep the
                               fastest; 0: fixed defaults (1)                         */
  volatile int32_t *cancel_flag; /* host-mapped int polled at every check, or NULL    */
  int32_t kernel_variant;   /* -1: the autotuner decides, variant 1 when autotune is 0;
                               0, 1, 2, 4, 8, 9, 16-21: that variant of both
                               per-attempt kernels, as reported by pdhg_get_tuning,
                               with the default grid; read at the first solve of
                               each precision; batched solves with autotune 0: 1, 2
                               or 4 rows (columns) per warp of both sweeps (4 for
                               any other value); default -1                        */
  int32_t kernel_grid;      /* > 0: blocks of both per-attempt kernels, overriding the
                               autotuner's grid; small grids make each warp sweep
                               many slices; batched solves with autotune 0: blocks
                               of both sweeps; 0: default or autotuned; default 0    */
  double infeas_tol;        /* infeasibility detection (Applegate et al.'s certificates
                               from iterate differences, the detection of the PDLP
                               method cited in Sec. II.E): at every check the
                               differences since the last restart of the current and
                               the average iterate are tested as rays of the unscaled
                               LP.  Dual ray y, lambda = -K^T y: objective
                               q^T y + sum_j (l_j lambda_j^+ - u_j lambda_j^-) over
                               finite bounds, violation = l2 norm of y_i < 0 on >=
                               rows and of lambda_j > 0 (l_j = -inf), < 0 (u_j = inf);
                               primal ray x: objective c^T x, violation = l2 norm of
                               (Kx)_i != 0 on equality rows, < 0 on >= rows, x_j < 0
                               (finite l_j), > 0 (finite u_j).  A ray whose violation
                               is <= infeas_tol x |objective| with the certificate's
                               sign (dual > 0, primal < 0) ends the solve with
                               PDHG_STATUS_PRIMAL_INFEASIBLE / _DUAL_INFEASIBLE.
                               Rays of FP32 iterates (mixed precision, batched
                               solves) carry ~1e-7 relative noise and are tested at
                               max(infeas_tol, 1e-6).  0 disables; default 1e-8     */
  int32_t ir_fold_checks;   /* mixed: a refinement round also ends after this many
                               checks without reaching its target, folding the
                               current iterate into x*, y* all the same, so the FP32
                               iterate stays a small correction and the per-attempt
                               changes keep FP32 resolution (0: only at the target);
                               default 16                                           */
  int32_t launch_overlap;   /* 1: the per-attempt kernels (variants 0-9) are launched
                               with programmatic dependent launch, so each one reads
                               its first matrix entries while the previous kernel
                               finishes; results are identical either way.  If the
                               CUDA graph cannot be built with it, the library builds
                               it without (pdhg_result.launch_overlap reports which).
                               Measured within 1-2% of plain launches on GB300 (the
                               per-kernel floor is the chain of dependent memory
                               round trips inside each kernel, not the launch);
                               default 0                                            */
} pdhg_opts;

/* Outcome of one solve (host struct written by the library). */
typedef struct pdhg_result {
  int32_t status;      /* PDHG_STATUS_*                                     */
  int32_t ir_rounds;   /* refinement rounds done (mixed), 0 for FP64          */
  int64_t iterations;  /* step attempts, all rounds                          */
  int64_t accepted;    /* accepted steps                                     */
  int64_t restarts;
  int64_t checks;
  double rel_p, rel_d, rel_gap, rel_kkt; /* of the returned point, unscaled   */
  double primal_obj, dual_obj;
  double solve_seconds;        /* device time of the whole call                */
  double time_to_tol[3];       /* seconds to rel_kkt <= 1e-4, 1e-6, 1e-8 or -1 */
  int64_t iters_to_tol[3];     /* attempts to the same                         */
  double eta, omega;           /* final step size and primal weight            */
  int64_t kernel_launches;     /* kernels this call ran (graph bodies counted
                                  once per executed body)                      */
  int32_t returned_average;    /* 1: the last round's returned candidate was the
                                  step-weighted average since the last restart,
                                  0: the current iterate                       */
  int32_t launch_overlap;      /* 1: the per-attempt kernels ran with programmatic
                                  dependent launch (opts.launch_overlap and accepted
                                  by the driver), 0: plain launches             */
} pdhg_result;

/* Fill *o with the defaults listed above. */
int pdhg_opts_default(pdhg_opts *o);

/* Create a workspace for `prob`.  Copies the sparsity structure to the host
 * once to build the internal row/column orderings and sliced-ELL layouts,
 * then allocates every device buffer a solve needs.  Values (val, c, l, u, q)
 * are read at each solve, so they may change between solves; the structure
 * and the pointers must stay valid and unchanged for the workspace's life.
 * `opts` may be NULL (defaults).  Synchronises `stream`. */
int pdhg_workspace_create(const pdhg_problem *prob, const pdhg_opts *opts, void **ws, void *stream);

/* Release a workspace (NULL is ignored). */
void pdhg_workspace_destroy(void *ws);

/* Replace the options of an existing workspace (validated; no reallocation
 * except for the trace buffer). */
int pdhg_set_opts(void *ws, const pdhg_opts *opts);

/* Solve the LP (PDHG with Ruiz + Pock-Chambolle rescaling, adaptive steps,
 * primal-weight updates, restarts and KKT termination; mixed precision adds
 * FP64 iterative refinement).  Writes the unscaled solution to x_out [n] and
 * y_out [m] (device, may be NULL) and the outcome to *res (host).  The whole
 * PDHG loop runs as one CUDA graph with a device-side while condition; the
 * host waits once per refinement round. */
int pdhg_solve(void *ws, double *x_out, double *y_out, pdhg_result *res, void *stream);

/* Solve B LPs that share K, c and q and differ only in their bounds
 * (branch-and-bound nodes fixing commitments).  l_b, u_b: device [B][n];
 * x_out: device [B][n], y_out: device [B][m] (may be NULL); res_b: host [B].
 * Per-instance step size, primal weight, restarts and termination. */
int pdhg_solve_batched(void *ws, int32_t B, const double *l_b, const double *u_b, double *x_out,
                       double *y_out, pdhg_result *res_b, void *stream);

/* Vector-Jacobian product of the last pdhg_solve of this workspace:
 *   given the cotangent g_cost of the optimal cost and g_x [n] of the primal
 *   solution (device, may be NULL), writes grad_q [m] and grad_c [n] (device)
 *   = d(g_cost * cost + g_x^T x*)/d(q, c), by implicit differentiation of the
 *   KKT system on the detected active set. */
int pdhg_backward(void *ws, double g_cost, const double *g_x, double *grad_q, double *grad_c,
                  void *stream);

/* Active-set polish of the last pdhg_solve (a crossover-lite: the paper's
 * pipeline passes the PDHG point to a crossover, Sec. III.B).  The active set
 * is read off the solution -- equality rows, >= rows whose dual exceeds their
 * slack, variables whose reduced cost exceeds their distance to a bound (held
 * there) -- and, when it is square (as many active rows as free variables),
 * the basic solution of that set is computed in FP64 on the device:
 *   x_B = the bounds,  K_{A,F} x_F = q_A - K_{A,B} x_B,  K_{A,F}^T y_A = c_F,  y = 0 elsewhere
 * (Jacobi-preconditioned conjugate gradients on the normal equations with the
 * workspace's matrix, aiming at relative residual 1e-13, one CUDA graph per
 * system).  x_out [n], y_out [m]:
 * device, original order, may be NULL; written only when the set is square.
 * *res (host) reports the outcome and the optimality measures of the polished
 * point (same definitions as pdhg_result, plus the l2 norms of its bound
 * violations and of negative duals on >= rows; both vanish at an optimal
 * basis).  A polished point with rel_kkt near 1e-15 is the optimal vertex of
 * that basis; violations flag a wrongly detected set. */
#define PDHG_POLISH_OK 1             /* both systems solved                       */
#define PDHG_POLISH_NOT_SQUARE 2     /* degenerate: active rows != free variables */
#define PDHG_POLISH_NO_CONVERGENCE 3 /* a system stayed above 1e-9 (singular set?)  */
typedef struct pdhg_polish_result {
  int32_t status;                 /* PDHG_POLISH_*                              */
  int32_t cg_iterations_primal;   /* CG iterations of the two systems           */
  int32_t cg_iterations_dual;
  int32_t reserved;
  int64_t active_rows, free_vars;
  double rel_p, rel_d, rel_gap, rel_kkt;
  double primal_obj, dual_obj;
  double bound_violation;         /* ||max(l - x, 0) + max(x - u, 0)||_2         */
  double dual_sign_violation;     /* ||min(y_i, 0) over >= rows||_2              */
  double cg_residual_primal;      /* relative residuals of the two systems; OK  */
  double cg_residual_dual;        /* needs both <= 1e-9                          */
} pdhg_polish_result;

int pdhg_polish(void *ws, double *x_out, double *y_out, pdhg_polish_result *res, void *stream);

/* Message of the last failure on this thread ("" if none). */
const char *pdhg_last_error(void);

/* Ruiz + Pock-Chambolle rescaling factors WITHOUT any device allocation.
 * The paper has no counterpart: this is for callers that cannot call
 * cudaMalloc (a caching allocator of another framework owns the device
 * memory, a fixed memory budget is set up front, or an allocation's implicit
 * synchronisation is not allowed).  Computes the same Dr [m], Dc [n] as
 * pdhg_prepare + pdhg_get_scaling (ruiz_iters l_inf passes, then one alpha = 1
 * Pock-Chambolle pass if pock_chambolle != 0), straight from the CSR of `prob`
 * (row_ptr, col, val, n, m; the other fields are ignored).  Dr, Dc: device,
 * caller-owned, written in original order.
 *   - Scratch: one file-scope device array of 2^21 doubles (16 MiB) that every
 *     GPU loading the library holds until the process exits.  n > 2^21 is
 *     rejected with PDHG_ERR_UNSUPPORTED before any device work.
 *   - No cudaMalloc, cudaFree or allocating library call is made.
 *   - The first call in a CUDA context (the device's primary context, or a
 *     driver-API context the caller made current) looks up the array's device
 *     address in that context (cudaGetSymbolAddress) and caches it by the
 *     context's unique id, so a context created after cudaDeviceReset gets its
 *     own lookup; make that first call before any stream capture.
 *   - Every call shares the array and finds the previous call's contents in
 *     it (it clears what must start at zero); calls that overlap on the GPU,
 *     in different streams or threads, race on it.
 *   - Column statistics use FP64 atomics for the Pock-Chambolle sums, so the
 *     last bits may differ from the workspace path and between calls. */
int pdhg_rescale_noalloc(const pdhg_problem *prob, int32_t ruiz_iters, int32_t pock_chambolle,
                         double *Dr, double *Dc, void *stream);

/* ---- diagnostics (kernel-level tests and measurement) -------------------- */

/* Load the values and run the rescaling of a solve without iterating. */
int pdhg_prepare(void *ws, void *stream);

/* Row and column scaling factors Dr [m], Dc [n] (device, FP64, original
 * order): K~ = diag(Dr) K diag(Dc).  Valid after pdhg_prepare or a solve. */
int pdhg_get_scaling(void *ws, double *Dr, double *Dc, void *stream);

/* out = K~ in (transpose = 0; in [n], out [m]) or K~^T in (transpose = 1;
 * in [m], out [n]) with the rescaled matrix in the workspace's sliced-ELL
 * layout, original index order, device FP64 vectors.  precision selects the
 * FP64 or the FP32 copy of the values (FP32 rounds `in` to float first and
 * accumulates in FP32). */
int pdhg_apply_K(void *ws, int32_t transpose, int32_t precision, const double *in, double *out,
                 void *stream);

/* Copy the trace of the last solve (opts.trace = 1) to host arrays:
 *   attempts [cap_a][5]: eta, omega, accepted, eta_max, eta_next
 *   checks   [cap_c][12]: attempts, restart, to_average, omega_after, KKT_w of the
 *                       current and average iterate, rel_kkt of the current and average,
 *                       rel_p, rel_d, rel_gap of the current iterate, eta after the check
 * *n_a, *n_c receive the counts recorded (may exceed the caps). */
int pdhg_get_trace(void *ws, double *attempts, int64_t cap_a, double *checks, int64_t cap_c,
                   int64_t *n_a, int64_t *n_c);

/* Launch configuration chosen for the per-attempt kernels, host int32 [12]:
 * FP64 {dual unroll, dual grid, adjoint unroll, adjoint grid}, then FP32, then
 * the batched sweeps {dual rows per warp, dual grid, adjoint columns per warp,
 * adjoint grid} (-1 and 0 before the first batched solve).
 * unroll 1, 2, 4: 32-row slices a warp sweeps together; 0: one slice per warp,
 * software pipelined (the next slice's first entries and row operands are
 * loaded while the current slice's gathers are in flight); 8, 9: variants 1
 * and 0 compiled for 8 resident blocks per SM (32 registers); 16, 17: the matrix
 * staged in shared memory by TMA bulk copies, one or two slices per warp at a
 * time; 18, 19: the same with the row (column) operands staged too; 20, 21:
 * a per-warp shared-memory ring filled by cp.async two or three slices ahead.
 * A precision not yet solved reports unroll -1 and grid 0. */
int pdhg_get_tuning(void *ws, int32_t *cfg);

/* Launch the two per-attempt kernels of `precision` `reps` times each on
 * `stream` against the workspace's current state, timing each kernel with CUDA
 * events on that stream; writes the average milliseconds per launch and the
 * algorithmic bytes per launch of the dual (K x) and adjoint (K^T y) kernels. */
int pdhg_time_kernels(void *ws, int32_t precision, int32_t reps, double *ms_dual, double *ms_adj,
                      double *bytes_dual, double *bytes_adj, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* PDHG_H */
