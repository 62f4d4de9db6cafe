/*
 * hcran_oracle.h -- FP64 CPU oracle of the energy-efficient PD-NOMA H-CRAN
 * resource allocator (arXiv 1803.07772: Dinkelbach loop of Section III around
 * the SCALE + Lagrangian dual solve of Section IV-A, Algorithm 1).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header or constant with the CUDA solver.
 */
#ifndef HCRAN_ORACLE_H
#define HCRAN_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int32_t M, N, K, Ks, l;      /* RRHs (0 = HPN), subcarriers, users, streaming users, NOMA cap */
  const double *pmax;          /* [M] W   (C3 / C12) */
  const double *eta;           /* [M]     power-amplifier factor (Sec. II-A power model) */
  const double *Pc;            /* [M] W   circuit power */
  const double *Pf;            /* [M] W   fronthaul power */
  double Bn_hz;                /* subcarrier bandwidth */
  double N0_w_per_hz;          /* noise PSD; sigma = N0 * Bn */
  const double *T_s;           /* [Ks] delay targets (C7) */
  const double *lambda_pps;    /* [Ks] Poisson arrival rates */
  double zbar_bits;            /* packet size */
  const double *w;             /* [M*K] priority weights w_{m,k}, NULL = all 1 */
  const float *G;              /* [N][M][K] channel power gains Gamma (k fastest) */
} orc_problem;

typedef struct {
  double tol_dinkelbach;       /* stop when F(q)/R <= tol (Sec. III) */
  double tol_scale;            /* varpi_2 of Algorithm 1 */
  double tol_dual;             /* varpi_1 of Algorithm 1 */
  int32_t max_dinkelbach, max_scale, max_dual;
  double q_init;               /* > 0: fixed E^1 (else E^1 = R(p^0)/P(p^0)) */
  double tie_eps;              /* relative margin under which a selection decision counts as a tie */
  /* Perturbation ensemble (parity tests only; 0 = off, the default): each new
   * power of a dual iteration is multiplied by (1 + noise_rel * u), u uniform
   * in [-1, 1) from a splitmix64 stream keyed by noise_seed.  With noise_rel
   * near the FP32 unit roundoff this shows where rounding-level differences
   * can move an instance's end point. */
  double noise_rel;
  uint64_t noise_seed;
} orc_params;

typedef struct {
  /* caller-allocated arrays (any may be NULL) */
  int32_t *A;                  /* [K] serving RRH, -1 = unserved */
  int32_t *S;                  /* [N*M*l] user ids per (n,m) in SIC order, -1 = empty */
  double *p;                   /* [N*M*l] W */
  double *alpha, *beta;        /* [N*M*l] SCALE coefficients */
  double *xi;                  /* [M] */
  double *zeta;                /* [Ks] */
  double *zeta_sic;            /* [N*M*l(l-1)/2] */
  double *q_trace;             /* [max_dinkelbach+1] E^1 = R(p^0)/P(p^0), then E^{i+1} after iteration i */
  double *F_trace;             /* [max_dinkelbach] F_i = R - q_i P */
  double *scale_obj_trace;     /* [max_dinkelbach*max_scale] exact R - E^i P after each SCALE pass */
  int32_t *scale_sel_changed;  /* [max_dinkelbach*max_scale] 1 on the first pass after a selection change */
  /* scalars written by the oracle */
  double ee, R, P;
  int32_t iters[3];            /* Dinkelbach, SCALE (total), dual (total) */
  int32_t status;              /* bit 0 not converged (Dinkelbach cap), bit 1 a streaming rate unmet
                                  (exact rate more than 1e-3 below Psi), bit 2 the output's EE is below
                                  an earlier iterate's (one kept for the streaming rates) */
  double slack_power_min;      /* min_m (pmax - sum p)/pmax */
  double slack_rate_min;       /* min_k (r_k - Psi_k)/Psi_k over streaming users (exact rate) */
  double slack_sic_max;        /* max over selected pairs of Omega_bar / mask (<= 0 is feasible) */
  double min_margin;           /* smallest relative margin of any selection decision */
  int32_t n_ties;              /* decisions with margin < tie_eps */
  int32_t n_scale_traced;      /* entries written to the scale traces */
} orc_result;

int orc_solve(const orc_problem *pr, const orc_params *par, orc_result *out);

/* Global-optimum comparator (stands in for Sec. IV-B's monotonic
 * optimisation on small instances): the best EE over every assignment (RRH
 * choice and per-(n, m) user subsets of at most l), powers by multi-start
 * coordinate golden-section search under C12 and C14 (hcran_oracle.c gives
 * the exact order).  Elastic users only (Ks = 0); M <= 8, K <= 6, l <= 3,
 * N*M*l <= 16.  *n_assign = assignments searched, *best_index = the
 * enumeration index of the best one (-1 if none); returns 1 on a bad problem. */
int orc_bruteforce(const orc_problem *pr, double *best_ee, int64_t *n_assign, int64_t *best_index);

/* Paper-literal penalty form of the selection constraints (C10, C11 kept
 * with multipliers theta, theta' instead of the explicit selection; see
 * hcran_penalty.c for the readings and the index order of the arrays).
 * Elastic users only (Ks = 0), unit weights, M <= 8; rho_rel in (0, 1) sets
 * rho_1 = rho_rel^2 mask_m mask_m' and rho_2 = rho_rel^(l+1) mask_m^(l+1).
 * Returns 1 on a bad problem, 2 when out of memory. */
typedef struct {
  double *p;                   /* [N*M*K] W, every (n, m, k) link (may be NULL) */
  double *alpha;               /* [N*M*K] SCALE coefficient after the last pass (may be NULL) */
  double *xi;                  /* [M] (may be NULL) */
  double *theta;               /* [n_theta] C10 multipliers (may be NULL) */
  double *theta2;              /* [n_theta2] C11 multipliers (may be NULL) */
  double ee, R, P;
  int32_t iters[3];
  int32_t status;              /* bit 0: the Dinkelbach cap was reached */
  double slack_power_min;      /* min_m (pmax - sum p)/pmax */
  double c10_max, c11_max;     /* largest C10 / C11 product relative to rho_1 / rho_2 */
  double slack_sic_max;        /* max Omega_bar / mask over pairs of links above rho_rel mask */
  int32_t n_theta, n_theta2;
} orc_pen_result;

int orc_penalty_solve(const orc_problem *pr, const orc_params *par, double rho_rel, orc_pen_result *out);

/* closed-form pieces, exposed so that tests can pin them on their own */
double orc_psi(double T_s, double lambda_pps, double zbar_bits, double Bn_hz);   /* C9 */
void orc_scale_coeffs(double z0, double *alpha, double *beta);                   /* SCALE bound */

#ifdef __cplusplus
}
#endif
#endif
