/*
 * uc_lp.h -- synthetic DC unit-commitment LP relaxation (instance generator).
 *
 * The paper solves the LP relaxation of the DC unit-commitment (UC) MILP of its
 * two-stage GO-Challenge-3 pipeline (Sec. II.A, Fig. 1) with PDHG (Sec. II.E).
 * The GO3 formulation and datasets are not public here, so this library builds
 * a seeded synthetic DC-UC relaxation with the bus counts and horizons of the
 * paper's networks (Sec. II.B, Table I) in the PDLP general form
 *
 *     min c^T x   s.t.  K_i. x  = q_i   for rows i <  m_eq   (equalities first)
 *                       K_i. x >= q_i   for rows i >= m_eq
 *                       l <= x <= u     (entries may be +-INFINITY)
 *
 * This file holds no solver arithmetic: it is an input generator shared by the
 * GPU solver and by the CPU checker.
 *
 * Ownership: uc_lp_build allocates every array of the returned uc_lp on the
 * host; the caller releases them with uc_lp_free.  Nothing here touches a GPU.
 * Errors: uc_lp_build returns 0 on success and a negative code on failure
 * (UC_ERR_INVALID_ARG for bad sizes, UC_ERR_NOMEM for allocation failure);
 * *out is then NULL and uc_lp_last_error() holds a message.
 */
#ifndef UC_LP_H
#define UC_LP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define UC_OK 0
#define UC_ERR_INVALID_ARG (-1)
#define UC_ERR_NOMEM (-2)

/* Variable kinds (uc_lp.var_kind). */
enum uc_var_kind {
  UC_VAR_P = 0,     /* real power output p_gt, MW, in [0, Pmax_g]                */
  UC_VAR_U = 1,     /* commitment u_gt in [0, 1] (relaxed binary)               */
  UC_VAR_V = 2,     /* start-up v_gt in [0, 1]; fixed to 0 in the first period  */
  UC_VAR_W = 3,     /* shut-down w_gt in [0, 1]; fixed to 0 in the first period */
  UC_VAR_THETA = 4, /* voltage angle theta_bt, rad, free; 0 at bus 0            */
  UC_VAR_SHED = 5,  /* load shed s+_bt in [0, d_bt] (with_slack only)           */
  UC_VAR_SPILL = 6  /* generation spill s-_bt >= 0 at generator buses (slack)   */
};

/* Row kinds (uc_lp.row_kind).  Rows 0..m_eq-1 are the equalities. */
enum uc_row_kind {
  UC_ROW_BALANCE = 0,  /* = : sum_g p - sum_l (+-)S (th_i - th_j)/x_l (+s+ - s-) = d_bt */
  UC_ROW_LOGIC = 1,    /* = : u_t - u_{t-1} - v_t + w_t = 0                          */
  UC_ROW_FLOW_POS = 2, /* >=:  S(th_i - th_j)/x_l >= -F_l                            */
  UC_ROW_FLOW_NEG = 3, /* >=: -S(th_i - th_j)/x_l >= -F_l                            */
  UC_ROW_PMIN = 4,     /* >=: p - Pmin u >= 0                                        */
  UC_ROW_PMAX = 5,     /* >=: Pmax u - p >= 0                                        */
  UC_ROW_RAMP_UP = 6,  /* >=: p_{t-1} - p_t + R u_{t-1} + SU_R v_t >= 0              */
  UC_ROW_RAMP_DN = 7,  /* >=: p_t - p_{t-1} + R u_t + SD_R w_t >= 0                  */
  UC_ROW_MIN_UP = 8,   /* >=: u_t - sum_{tau in window} v_tau >= 0                   */
  UC_ROW_MIN_DN = 9    /* >=: -u_t - sum_{tau in window} w_tau >= -1                 */
};

/* Generator parameters.  Sizes must be >= 1 (n_line may be 0 only when
 * n_bus == 1).  n_line >= n_bus is required for n_bus >= 3 (ring + chords);
 * n_bus == 2 takes exactly one line. */
typedef struct uc_params {
  int32_t n_bus;      /* N buses                                  */
  int32_t n_line;     /* L lines: ring of N plus L-N random chords */
  int32_t n_gen;      /* G generators at uniformly random buses    */
  int32_t n_periods;  /* T periods of length 24/T hours            */
  uint64_t seed;      /* SplitMix64 seed of every random stream    */
  int32_t with_slack; /* 1: add shed/spill slack variables         */
  int32_t reserved;
  double horizon_hours; /* length of the horizon in hours (24)   */
  double s_base;        /* MVA base of the DC flow (100)         */
  double peak_frac;     /* peak system load / sum Pmax (0.7)     */
} uc_params;

/* One instance.  All arrays are host memory owned by the library. */
typedef struct uc_lp {
  int64_t n, m, m_eq, nnz;
  int64_t *row_ptr; /* [m+1] CSR row pointers of K                 */
  int32_t *col;     /* [nnz] column indices, ascending in each row */
  double *val;      /* [nnz] coefficients                          */
  double *c;        /* [n] cost                                    */
  double *l, *u;    /* [n] bounds, +-INFINITY where absent         */
  double *q;        /* [m] right-hand side                         */
  int32_t *var_kind; /* [n] enum uc_var_kind */
  int32_t *row_kind; /* [m] enum uc_row_kind */
  /* index maps, period-major: entry [t*G + g] or [t*N + b] */
  int32_t n_gen, n_bus, n_line, n_periods;
  int64_t *idx_p, *idx_u, *idx_v, *idx_w; /* [T*G] variable index          */
  int64_t *idx_theta;                     /* [T*N] variable index          */
  int64_t *row_balance;                   /* [T*N] row index of balance bt */
  double *load;                           /* [T*N] d_bt, MW                */
  int32_t *gen_bus;                       /* [G] bus of each generator     */
  int32_t *line_from, *line_to;           /* [L] endpoints                 */
  double *gen_pmax;                       /* [G] Pmax, MW                  */
  double *gen_cost;                       /* [G] linear cost, $/MWh        */
  double *gen_noload;                     /* [G] no-load cost, $/h         */
  int32_t *gen_min_up, *gen_min_dn;       /* [G] windows, periods          */
  double dt_hours;                        /* period length                 */
} uc_lp;

/* Build one instance.  Returns UC_OK and sets *out, or a negative code. */
int uc_lp_build(const uc_params *p, uc_lp **out);
/* Release an instance built by uc_lp_build (NULL is ignored). */
void uc_lp_free(uc_lp *lp);
/* Thread-local message of the last failure ("" if none). */
const char *uc_lp_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* UC_LP_H */
