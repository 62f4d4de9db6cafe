/*
 * hcran_oracle.c -- plain FP64 CPU oracle of the energy-efficient PD-NOMA
 * H-CRAN resource allocator of arXiv 1803.07772.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the CPU
 * baseline of the benchmark, never by the product path.  It shares no code
 * with the CUDA solver.
 *
 * The method reaches a local optimum through an iteration, so the oracle runs
 * the algorithm step by step in the paper's order, in double precision, with
 * plain loops over dense (n, m, slot) arrays and every sum recomputed from its
 * definition:
 *
 *   Dinkelbach (Sec. III, Theorem 1, Lemma 1, Prop. 1):
 *     p^0 initial feasible point, E^1 = R(p^0)/P(p^0)
 *     for i = 1, 2, ...:
 *       RRH/user selection (the binaries of C1/C5, see readings below)
 *       Algorithm 1 (Sec. IV-A) at fixed E^i:
 *         alpha = 1, beta = 0 (high-SIR start)
 *         repeat over SCALE passes s:
 *           repeat over dual iterations v:
 *             multipliers by projected subgradient, powers by eq. (653)/(683)
 *           until ||p^v - p^{v-1}|| < varpi_1
 *           alpha/beta at the new point (eq. scale_approximation)
 *         until ||p^s - p^{s-1}|| < varpi_2 or s = S
 *       C12 projection; F = R(p^i) - E^i P(p^i); E^{i+1} = R(p^i)/P(p^i)
 *     until F <= tol * R or i = I
 *
 * Readings where the paper is silent or garbled (each is listed in the
 * project's design notes and implemented identically by the CUDA solver):
 *  - SINR/interference of Sec. II-A with a strict SIC order (gain descending,
 *    lower user index first on equal gains); user k hears the stronger users
 *    of its own (m,n) and every selected link of the other RRHs on n.
 *  - Power model: Sec. II-A builds the consumed power from the amplifier
 *    power eta_m sum_{k in K} p of every RRH (all users), while the formula of
 *    P(A, rho, p) that follows sums only the elastic users.  P here counts the
 *    transmit power of every user, as the three-part power model states; with
 *    streaming power left out of P a streaming user whose rate target is met
 *    would have neither an energy price nor a rate price, and its power would
 *    be undetermined (0/0 in eq. (683)).  EE = R(elastic) / P.
 *  - KKT powers: the terms of eq. (653)/(683) are derived from the Lagrangian
 *    of problem (final_Problem_formulation_1) in the log-power variable: a
 *    transmitter pays c*alpha/(ln2 * I) * Gamma for every victim it interferes
 *    with, c = w for elastic users and zeta'_k * w for streaming users; every
 *    link carries the E^i * eta_m term of P.
 *  - The outer iteration (eq. outer_iterative_algorithm) labels E^0 -> p^0 as
 *    its initialisation: p^0 is the initial feasible point, E^1 = R(p^0)/P(p^0),
 *    and iteration i >= 1 solves O5 at E^i starting from p^{i-1}.
 *  - C10/C11 (binary relaxation with rho_1, rho_2 -> 0) are taken as an
 *    explicit selection at the start of every Dinkelbach iteration: candidate
 *    water-filling utility for every (m,k,n), A_k = argmax_m sum_n utility,
 *    then per (m,n) the users of m admitted greedily by utility while the
 *    set stays SIC-feasible (Omega_bar <= 0) and has at most l members.
 *    C9 needs every streaming user served: a streaming user left without a
 *    link is then given one, in user order, on the subcarrier of its RRH
 *    (A_k, or argmax_m sum_n Gamma when A_k = -1) with the largest gain that
 *    has a free slot or an elastic user, whom it displaces (the admitted
 *    elastic user of least utility).  New links start at the water-filling
 *    power, at least the floor.
 *  - C14 is used in the divided form Omega_bar = (sigma+X_k)/Gamma_k -
 *    (sigma+X_k')/Gamma_k', linear in the other RRHs' per-subcarrier powers;
 *    positive coefficients enter the denominator, negative ones the numerator
 *    at the SCALE linearisation point (the DC step of eq. C13e_new).
 *  - Subgradient steps (the paper fixes none), all with the diminishing step
 *    delta_v = 1/sqrt(v+1) of the dual loop: power budget and SIC on scaled
 *    residuals; the rate multiplier in log scale,
 *    zeta' <- zeta' * 2^(delta_v clip((Psi - r_hat)/sum alpha, -1, 1)),
 *    since r_hat is linear in log2 zeta'.  p stays in [1e-9 mask, mask];
 *    alpha is evaluated at gamma >= 1e-12; the norms of the stopping tests
 *    are max |delta p| / mask over the selected links.
 *  - The stop test F <= xi of Sec. III is taken relative (F <= tol * R).
 *    Lemma 1 gives max_p R - E^i P >= 0, attained at least by p^{i-1} itself,
 *    so an inner solve that ends below its start point (F < 0) is inexact:
 *    the Dinkelbach iterate then stays p^{i-1} and the loop ends, provided
 *    p^{i-1} meets the streaming rates (C13 with exact rates, within 1e-3) or
 *    misses them by no more than p^i does; otherwise p^i is kept and the loop
 *    goes on.
 */
#include "hcran_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define LN2 0.69314718055994530942
#define P_FLOOR_REL 1e-9
#define GAMMA_FLOOR 1e-12

#define ZETA_ASUM_MIN 0.05
#define ZETA_MIN 1e-6
#define ZETA_MAX 1e6

#define ST_NOT_CONVERGED 1
#define ST_STREAMING_UNMET 2
#define ST_EE_DECREASED 4

/* ------------------------------------------------------------------ */
/* closed forms                                                         */
/* ------------------------------------------------------------------ */

/* C9, eq. (Eq6d): Psi = Psi_hat / B_n with
 * Psi_hat = 2 lambda zbar / ((2 + 2 lambda T) - sqrt((2 + 2 lambda T)^2 - 8 lambda T)),
 * i.e. the smaller root of the quadratic (Eq6b) in the mean service time. */
double orc_psi(double T_s, double lambda_pps, double zbar_bits, double Bn_hz) {
  double b = 2.0 + 2.0 * lambda_pps * T_s;
  double root = sqrt(b * b - 8.0 * lambda_pps * T_s);
  double psi_hat = 2.0 * lambda_pps * zbar_bits / (b - root);
  return psi_hat / Bn_hz;
}

/* SCALE lower bound (eq. scale_approximation): alpha log2 z + beta <= log2(1+z),
 * tight at z = z0 with alpha = z0/(1+z0), beta = log2(1+z0) - alpha log2 z0. */
void orc_scale_coeffs(double z0, double *alpha, double *beta) {
  double a = z0 / (1.0 + z0);
  *alpha = a;
  *beta = log2(1.0 + z0) - a * log2(z0);
}

/* ------------------------------------------------------------------ */
/* instance and state                                                   */
/* ------------------------------------------------------------------ */

typedef struct {
  int M, N, K, Ks, Ke, l, npair;
  const float *G;
  const double *pmax, *eta;
  double sigma, Pconst;
  double *mask, *pfloor, *Psi, *w;
} inst_t;

typedef struct {
  int32_t *A;                       /* [K] */
  int32_t *S;                       /* [N*M*l] */
  double *p, *alpha, *beta, *plin;  /* [N*M*l] */
  double *xi, *zeta, *zsic;         /* [M], [Ks], [N*M*npair] */
} state_t;

static double gain(const inst_t *I, int n, int m, int k) {
  return (double)I->G[((size_t)n * I->M + m) * I->K + k];
}
static size_t slot(const inst_t *I, int n, int m, int s) {
  return ((size_t)n * I->M + m) * I->l + s;
}
static int pair_index(int l, int a, int b) { /* a < b */
  return a * l - a * (a + 1) / 2 + (b - a - 1);
}
/* SIC order on (m,n): a precedes (is stronger than) b */
static int stronger(const inst_t *I, int n, int m, int a, int b) {
  double ga = gain(I, n, m, a), gb = gain(I, n, m, b);
  return ga > gb || (ga == gb && a < b);
}
/* weight c of a link: w for elastic users, zeta'_k w for streaming users */
static double weight_c(const inst_t *I, const state_t *st, int m, int k) {
  double w = I->w[(size_t)m * I->K + k];
  return k >= I->Ke ? st->zeta[k - I->Ke] * w : w;
}

static int state_alloc(const inst_t *I, state_t *st) {
  size_t L = (size_t)I->N * I->M * I->l;
  size_t NP = (size_t)I->N * I->M * (I->npair > 0 ? I->npair : 1);
  st->A = calloc(I->K, sizeof(int32_t));
  st->S = calloc(L, sizeof(int32_t));
  st->p = calloc(L, sizeof(double));
  st->alpha = calloc(L, sizeof(double));
  st->beta = calloc(L, sizeof(double));
  st->plin = calloc(L, sizeof(double));
  st->xi = calloc(I->M, sizeof(double));
  st->zeta = calloc(I->Ks > 0 ? I->Ks : 1, sizeof(double));
  st->zsic = calloc(NP, sizeof(double));
  return st->A && st->S && st->p && st->alpha && st->beta && st->plin && st->xi &&
         st->zeta && st->zsic;
}
static void state_copy(const inst_t *I, state_t *dst, const state_t *src) {
  size_t L = (size_t)I->N * I->M * I->l;
  size_t NP = (size_t)I->N * I->M * (I->npair > 0 ? I->npair : 1);
  memcpy(dst->A, src->A, sizeof(int32_t) * I->K);
  memcpy(dst->S, src->S, sizeof(int32_t) * L);
  memcpy(dst->p, src->p, sizeof(double) * L);
  memcpy(dst->alpha, src->alpha, sizeof(double) * L);
  memcpy(dst->beta, src->beta, sizeof(double) * L);
  memcpy(dst->plin, src->plin, sizeof(double) * L);
  memcpy(dst->xi, src->xi, sizeof(double) * I->M);
  memcpy(dst->zeta, src->zeta, sizeof(double) * (I->Ks > 0 ? I->Ks : 1));
  memcpy(dst->zsic, src->zsic, sizeof(double) * NP);
}
static void state_free(state_t *st) {
  free(st->A); free(st->S); free(st->p); free(st->alpha); free(st->beta);
  free(st->plin); free(st->xi); free(st->zeta); free(st->zsic);
}
/* ------------------------------------------------------------------ */
/* interference and SINR (Sec. II-A; I_bar of problem eq7)              */
/* ------------------------------------------------------------------ */

/* Ptot[n*M + j] = sum of the powers RRH j puts on subcarrier n */
static void rrh_totals(const inst_t *I, const state_t *st, double *Ptot) {
  for (int n = 0; n < I->N; n++)
    for (int j = 0; j < I->M; j++) {
      double t = 0.0;
      for (int s = 0; s < I->l; s++)
        if (st->S[slot(I, n, j, s)] >= 0) t += st->p[slot(I, n, j, s)];
      Ptot[(size_t)n * I->M + j] = t;
    }
}

/* inter-cell interference X_{m,k}^{(n)} = sum_{j != m} Gamma_{j,k}^{(n)} Ptot_{j}^{(n)} */
static double inter_cell(const inst_t *I, const double *Ptot, int n, int m, int k) {
  double x = 0.0;
  for (int j = 0; j < I->M; j++)
    if (j != m) x += gain(I, n, j, k) * Ptot[(size_t)n * I->M + j];
  return x;
}

/* sigma + I of the selected link in slot s of (m,n): the stronger users of
 * the same (m,n) (slots 0..s-1 in SIC order) plus every other RRH on n */
static double noise_plus_interference(const inst_t *I, const state_t *st, const double *Ptot,
                                      int n, int m, int s) {
  int k = st->S[slot(I, n, m, s)];
  double intra = 0.0;
  for (int b = 0; b < s; b++)
    if (st->S[slot(I, n, m, b)] >= 0) intra += st->p[slot(I, n, m, b)];
  return I->sigma + gain(I, n, m, k) * intra + inter_cell(I, Ptot, n, m, k);
}

/* per selected link: Ie = sigma + I, gamma, victim price pi = c alpha / (ln2 Ie) */
static void link_quantities(const inst_t *I, const state_t *st, const double *Ptot,
                            double *Ie, double *gam, double *pi) {
  for (int n = 0; n < I->N; n++)
    for (int m = 0; m < I->M; m++)
      for (int s = 0; s < I->l; s++) {
        size_t e = slot(I, n, m, s);
        int k = st->S[e];
        if (k < 0) continue;
        double ie = noise_plus_interference(I, st, Ptot, n, m, s);
        Ie[e] = ie;
        gam[e] = st->p[e] * gain(I, n, m, k) / ie;
        pi[e] = weight_c(I, st, m, k) * st->alpha[e] / (LN2 * ie);
      }
}

/* C14 in divided form for the selected pair (a stronger, b weaker) on (m,n):
 * Omega_bar = (sigma + X_a)/Gamma_a - (sigma + X_b)/Gamma_b <= 0 */
static double omega_bar(const inst_t *I, const double *Ptot, int n, int m, int ka, int kb) {
  double xa = inter_cell(I, Ptot, n, m, ka);
  double xb = inter_cell(I, Ptot, n, m, kb);
  return (I->sigma + xa) / gain(I, n, m, ka) - (I->sigma + xb) / gain(I, n, m, kb);
}

/* sum over the SIC pairs of the other RRHs on n of zeta_sic * coefficient of
 * Ptot_j in Omega_bar, split by sign: SICp (>0, priced in the denominator)
 * and SICm (<0, linearised into the numerator) */
static void sic_terms(const inst_t *I, const state_t *st, double *SICp, double *SICm) {
  for (int n = 0; n < I->N; n++)
    for (int j = 0; j < I->M; j++) {
      double sp = 0.0, sm = 0.0;
      for (int m = 0; m < I->M; m++) {
        if (m == j) continue;
        for (int a = 0; a < I->l; a++)
          for (int b = a + 1; b < I->l; b++) {
            int ka = st->S[slot(I, n, m, a)], kb = st->S[slot(I, n, m, b)];
            if (ka < 0 || kb < 0) continue;
            double z = st->zsic[((size_t)n * I->M + m) * I->npair + pair_index(I->l, a, b)];
            if (z == 0.0) continue;
            double c = gain(I, n, j, ka) / gain(I, n, m, ka) - gain(I, n, j, kb) / gain(I, n, m, kb);
            if (c > 0.0) sp += z * c;
            else sm += z * (-c);
          }
      }
      SICp[(size_t)n * I->M + j] = sp;
      SICm[(size_t)n * I->M + j] = sm;
    }
}

/* sum_{victims v of the link (n,m,k)} pi_v * Gamma_{m,v}^{(n)}: the weaker
 * selected users of (m,n) and every selected user of the other RRHs on n,
 * skipping user `skip` (the candidate itself during selection) */
static double victim_price(const inst_t *I, const state_t *st, const double *pi,
                           int n, int m, int k, int skip) {
  double acc = 0.0;
  for (int j = 0; j < I->M; j++)
    for (int b = 0; b < I->l; b++) {
      int v = st->S[slot(I, n, j, b)];
      if (v < 0 || v == skip || v == k) continue;
      if (j == m && !stronger(I, n, m, k, v)) continue;
      acc += pi[slot(I, n, j, b)] * gain(I, n, m, v);
    }
  return acc;
}

/* ------------------------------------------------------------------ */
/* exact objective pieces (problem eq7)                                 */
/* ------------------------------------------------------------------ */

/* R = sum over elastic links of w log2(1+gamma); P = P_const + sum_m eta_m sum p
 * over every selected link (the power model of Sec. II-A) */
static void exact_R_P(const inst_t *I, const state_t *st, double *R, double *P, double *Ptot) {
  rrh_totals(I, st, Ptot);
  double r = 0.0, tx = 0.0;
  for (int n = 0; n < I->N; n++)
    for (int m = 0; m < I->M; m++)
      for (int s = 0; s < I->l; s++) {
        size_t e = slot(I, n, m, s);
        int k = st->S[e];
        if (k < 0) continue;
        tx += I->eta[m] * st->p[e];
        if (k >= I->Ke) continue;
        double ie = noise_plus_interference(I, st, Ptot, n, m, s);
        double g = st->p[e] * gain(I, n, m, k) / ie;
        r += I->w[(size_t)m * I->K + k] * log2(1.0 + g);
      }
  *R = r;
  *P = I->Pconst + tx;
}

/* ------------------------------------------------------------------ */
/* initial feasible point p^0 (Sec. III asks for one without giving it) */
/* ------------------------------------------------------------------ */

/* sort user ids by SIC order on (m,n) (insertion sort, tiny lists) */
static void sort_sic(const inst_t *I, int n, int m, int *ids, int cnt) {
  for (int i = 1; i < cnt; i++) {
    int x = ids[i], j = i - 1;
    while (j >= 0 && stronger(I, n, m, x, ids[j])) { ids[j + 1] = ids[j]; j--; }
    ids[j + 1] = x;
  }
}

/* argmax_m sum_n Gamma_{m,k}^{(n)} (lowest m on equal sums) */
static int strongest_rrh(const inst_t *I, int k) {
  int best = 0;
  double bestv = -1.0;
  for (int m = 0; m < I->M; m++) {
    double t = 0.0;
    for (int n = 0; n < I->N; n++) t += gain(I, n, m, k);
    if (t > bestv) { bestv = t; best = m; }
  }
  return best;
}

static void initial_state(const inst_t *I, state_t *st) {
  for (int k = 0; k < I->K; k++) st->A[k] = strongest_rrh(I, k);
  /* S_{m,n} = the l strongest users served by m; p = mask/l */
  int *ids = malloc(sizeof(int) * I->K);
  for (int n = 0; n < I->N; n++)
    for (int m = 0; m < I->M; m++) {
      int cnt = 0;
      for (int k = 0; k < I->K; k++) if (st->A[k] == m) ids[cnt++] = k;
      sort_sic(I, n, m, ids, cnt);
      for (int s = 0; s < I->l; s++) {
        size_t e = slot(I, n, m, s);
        if (s < cnt) {
          st->S[e] = ids[s];
          st->p[e] = I->mask[m] / I->l;
        } else {
          st->S[e] = -1;
          st->p[e] = 0.0;
        }
        st->alpha[e] = 1.0;
        st->beta[e] = 0.0;
        st->plin[e] = st->p[e];
      }
    }
  free(ids);
  for (int m = 0; m < I->M; m++) st->xi[m] = 0.0;
  for (int k = 0; k < I->Ks; k++) st->zeta[k] = 1.0;
  memset(st->zsic, 0, sizeof(double) * (size_t)I->N * I->M * (I->npair > 0 ? I->npair : 1));
}

/* ------------------------------------------------------------------ */
/* selection (the binaries of C1, C2, C5, C6 via C10/C11 with ϱ -> 0)   */
/* ------------------------------------------------------------------ */

typedef struct {
  double *Ptot, *Ie, *gam, *pi, *SICp, *SICm, *u, *pstar, *Xc;
  int *ids;
  double *keys;
  double noise_rel;                 /* perturbation ensemble (orc_params), 0 = off */
  uint64_t noise_seed, noise_ctr;
} scratch_t;

/* u uniform in [-1, 1) from the splitmix64 output of counter noise_ctr */
static double noise_u(scratch_t *w) {
  uint64_t z = w->noise_seed + 0x9E3779B97F4A7C15ull * (++w->noise_ctr);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

static void track(double margin, double eps, double *min_margin, int *n_ties) {
  if (margin < *min_margin) *min_margin = margin;
  if (margin < eps) (*n_ties)++;
}

/* candidate power that maximises c log2(1+g p) - den p on [0, mask]
 * (water-filling form of the single-link KKT condition) */
static double waterfill(double c, double den, double g, double mask) {
  if (c <= 0.0) return 0.0;
  if (den <= 0.0) return mask;
  double x = c / (LN2 * den) - 1.0 / g;
  if (x <= 0.0) return 0.0;
  return x >= mask ? mask : x;
}

static int select_links(const inst_t *I, state_t *st, double q, scratch_t *w,
                        double tie_eps, double *min_margin, int *n_ties) {
  const int N = I->N, M = I->M, K = I->K, l = I->l;
  rrh_totals(I, st, w->Ptot);
  link_quantities(I, st, w->Ptot, w->Ie, w->gam, w->pi);
  sic_terms(I, st, w->SICp, w->SICm);

  /* candidate utility of every (n, m, k) at the current prices */
  for (int n = 0; n < N; n++)
    for (int m = 0; m < M; m++)
      for (int k = 0; k < K; k++) {
        int a = st->A[k];
        double pk = 0.0; /* k's own current power on n (excluded from its interference) */
        if (a >= 0)
          for (int b = 0; b < l; b++)
            if (st->S[slot(I, n, a, b)] == k) pk = st->p[slot(I, n, a, b)];
        double X = 0.0;
        for (int j = 0; j < M; j++)
          if (j != m) X += gain(I, n, j, k) * (w->Ptot[(size_t)n * M + j] - (j == a ? pk : 0.0));
        double Y = 0.0;
        for (int b = 0; b < l; b++) {
          int i = st->S[slot(I, n, m, b)];
          if (i < 0 || i == k) continue;
          if (stronger(I, n, m, i, k)) Y += st->p[slot(I, n, m, b)];
        }
        double gk = gain(I, n, m, k);
        double Ic = I->sigma + X + gk * Y;
        double g = gk / Ic;
        double den = q * I->eta[m] + st->xi[m] +
                     victim_price(I, st, w->pi, n, m, k, k) + w->SICp[(size_t)n * M + m];
        double c = weight_c(I, st, m, k);
        double ps = waterfill(c, den, g, I->mask[m]);
        size_t t = ((size_t)n * M + m) * K + k;
        w->pstar[t] = ps;
        w->Xc[t] = X;
        w->u[t] = ps > 0.0 ? c * log2(1.0 + g * ps) - den * ps : 0.0;
        /* margin of the "transmit at all" decision c g > ln2 den */
        w->keys[t] = (c > 0.0 && den > 0.0)
                         ? fabs(c * g - LN2 * den) / fmax(c * g, LN2 * den)
                         : 1.0;
      }

  /* A_k = argmax_m sum_n u (lowest m on equal sums; -1 if all zero) */
  int changed = 0;
  int *Anew = malloc(sizeof(int) * K);
  for (int k = 0; k < K; k++) {
    int best = -1;
    double b1 = 0.0, b2 = 0.0;
    for (int m = 0; m < M; m++) {
      double U = 0.0;
      for (int n = 0; n < N; n++) U += w->u[((size_t)n * M + m) * K + k];
      if (U > b1) { b2 = b1; b1 = U; best = m; }
      else if (U > b2) b2 = U;
    }
    if (best >= 0 && b2 > 0.0) track((b1 - b2) / b1, tie_eps, min_margin, n_ties);
    Anew[k] = best;
    if (Anew[k] != st->A[k]) changed = 1;
  }

  /* S_{m,n}: users with A_k = m and positive utility, admitted greedily in
   * utility order while the set stays SIC-feasible and has at most l members */
  size_t L = (size_t)N * M * l;
  int32_t *Snew = malloc(sizeof(int32_t) * L);
  for (int n = 0; n < N; n++)
    for (int m = 0; m < M; m++) {
      const double *um = w->u + ((size_t)n * M + m) * K;
      const double *xm = w->Xc + ((size_t)n * M + m) * K;
      int cnt = 0;
      for (int k = 0; k < K; k++)
        if (Anew[k] == m) w->ids[cnt++] = k;
      /* order candidates by utility descending, lower id first on equal utility */
      for (int i = 1; i < cnt; i++) {
        int x = w->ids[i], j = i - 1;
        while (j >= 0 && (um[x] > um[w->ids[j]] || (um[x] == um[w->ids[j]] && x < w->ids[j]))) {
          w->ids[j + 1] = w->ids[j];
          j--;
        }
        w->ids[j + 1] = x;
      }
      int chosen[64];
      int nc = 0, i = 0;
      for (; i < cnt && nc < l; i++) {
        int k = w->ids[i];
        size_t t = ((size_t)n * M + m) * K + k;
        track(w->keys[t], tie_eps, min_margin, n_ties); /* transmit-at-all decision */
        if (!(um[k] > 0.0)) break;
        int feasible = 1;
        for (int c = 0; c < nc && feasible; c++) {
          int o = chosen[c];
          int a = stronger(I, n, m, k, o) ? k : o, b = a == k ? o : k;
          double ra = (I->sigma + xm[a]) / gain(I, n, m, a);
          double rb = (I->sigma + xm[b]) / gain(I, n, m, b);
          track(fabs(ra - rb) / fmax(ra, rb), tie_eps, min_margin, n_ties);
          if (ra - rb > 0.0) feasible = 0; /* Omega_bar > 0: SIC would fail */
        }
        if (feasible) chosen[nc++] = k;
      }
      if (nc == l && i < cnt && um[w->ids[i]] > 0.0) /* first user left out by the cap */
        track((um[chosen[l - 1]] - um[w->ids[i]]) / um[chosen[l - 1]], tie_eps, min_margin, n_ties);
      sort_sic(I, n, m, chosen, nc);
      for (int s2 = 0; s2 < l; s2++) Snew[slot(I, n, m, s2)] = s2 < nc ? chosen[s2] : -1;
    }

  /* C9 needs every streaming user served: one left without a link gets one, in
   * user order, on the subcarrier of its RRH with the largest gain (lowest n
   * on equal gains) that has a free slot or an admitted elastic user; a full
   * (m,n) gives up its elastic user of least utility (higher id on equal
   * utility) */
  for (int k = I->Ke; k < K; k++) {
    int served = 0;
    for (size_t e = 0; e < L && !served; e++)
      if (Snew[e] == k) served = 1;
    if (served) continue;
    const int m = Anew[k] >= 0 ? Anew[k] : strongest_rrh(I, k);
    Anew[k] = m;
    int nb = -1, sb = -1;
    double gb = -1.0;
    for (int n = 0; n < N; n++) {
      double g = gain(I, n, m, k);
      if (!(g > gb)) continue;
      int cnt = 0, rs = -1;
      for (int s = 0; s < l; s++) {
        int v = Snew[slot(I, n, m, s)];
        if (v < 0) continue;
        cnt++;
        if (v >= I->Ke) continue;
        double uv = w->u[((size_t)n * M + m) * K + v];
        int vr = rs >= 0 ? Snew[slot(I, n, m, rs)] : -1;
        double ur = rs >= 0 ? w->u[((size_t)n * M + m) * K + vr] : 0.0;
        if (rs < 0 || uv < ur || (uv == ur && v > vr)) rs = s;
      }
      if (cnt < l || rs >= 0) { gb = g; nb = n; sb = cnt < l ? -1 : rs; }
    }
    if (nb < 0) continue; /* every (m,n) is full of streaming users */
    int ids[64], cnt = 0;
    for (int s = 0; s < l; s++) {
      int v = Snew[slot(I, nb, m, s)];
      if (v >= 0 && s != sb) ids[cnt++] = v;
    }
    if (sb >= 0) { /* margin of the displaced user against the next elastic one */
      double ur = w->u[((size_t)nb * M + m) * K + Snew[slot(I, nb, m, sb)]];
      for (int c = 0; c < cnt; c++)
        if (ids[c] < I->Ke) {
          double uo = w->u[((size_t)nb * M + m) * K + ids[c]];
          track(fabs(uo - ur) / fmax(fabs(uo), fabs(ur)), tie_eps, min_margin, n_ties);
        }
    }
    ids[cnt++] = k;
    sort_sic(I, nb, m, ids, cnt);
    for (int s = 0; s < l; s++) Snew[slot(I, nb, m, s)] = s < cnt ? ids[s] : -1;
  }

  /* new state: kept links keep p, alpha, beta; new links start at p*, at
   * least the floor */
  for (int n = 0; n < N; n++)
    for (int m = 0; m < M; m++) {
      int same_set = 1;
      for (int s = 0; s < l; s++)
        if (Snew[slot(I, n, m, s)] != st->S[slot(I, n, m, s)]) same_set = 0;
      if (!same_set) changed = 1;
      double np_[64], na[64], nb[64], nl[64];
      for (int s = 0; s < l; s++) {
        int k = Snew[slot(I, n, m, s)];
        np_[s] = na[s] = nb[s] = nl[s] = 0.0;
        if (k < 0) continue;
        int old = -1;
        for (int b = 0; b < l; b++)
          if (st->S[slot(I, n, m, b)] == k) old = b;
        if (old >= 0) {
          size_t e = slot(I, n, m, old);
          np_[s] = st->p[e]; na[s] = st->alpha[e]; nb[s] = st->beta[e]; nl[s] = st->plin[e];
        } else {
          size_t t = ((size_t)n * M + m) * K + k;
          np_[s] = w->pstar[t] > I->pfloor[m] ? w->pstar[t] : I->pfloor[m];
          nl[s] = np_[s];
          na[s] = 1.0;
          nb[s] = 0.0;
        }
      }
      for (int s = 0; s < l; s++) {
        size_t e = slot(I, n, m, s);
        st->S[e] = Snew[e];
        st->p[e] = np_[s]; st->alpha[e] = na[s]; st->beta[e] = nb[s]; st->plin[e] = nl[s];
      }
      if (!same_set)
        for (int pr = 0; pr < I->npair; pr++) st->zsic[((size_t)n * M + m) * I->npair + pr] = 0.0;
    }
  for (int k = 0; k < K; k++) st->A[k] = Anew[k];
  free(Anew);
  free(Snew);
  return changed;
}

/* ------------------------------------------------------------------ */
/* one dual iteration of Algorithm 1 (eq. 653 / 683 + subgradient)     */
/* ------------------------------------------------------------------ */

static double dual_iteration(const inst_t *I, state_t *st, double q, int v, scratch_t *w) {
  const int N = I->N, M = I->M, l = I->l;
  rrh_totals(I, st, w->Ptot);
  link_quantities(I, st, w->Ptot, w->Ie, w->gam, w->pi);

  /* projected subgradient step on the multipliers, residuals at the current p */
  double delta = 1.0 / sqrt((double)v + 1.0);
  for (int m = 0; m < M; m++) { /* C12: sum_{k,n} p <= pmax */
    double tot = 0.0;
    for (int n = 0; n < N; n++) tot += w->Ptot[(size_t)n * M + m];
    double res = (tot - I->pmax[m]) / I->pmax[m];
    double xi = st->xi[m] + delta * res / (LN2 * I->mask[m]);
    st->xi[m] = xi > 0.0 ? xi : 0.0;
  }
  for (int ks = 0; ks < I->Ks; ks++) { /* C13 hat: sum_n w (alpha log2 gamma + beta) >= Psi */
    int k = I->Ke + ks;
    double r = 0.0;
    for (int n = 0; n < N; n++)
      for (int m = 0; m < M; m++)
        for (int s = 0; s < l; s++) {
          size_t e = slot(I, n, m, s);
          if (st->S[e] != k) continue;
          double g = w->gam[e] > GAMMA_FLOOR ? w->gam[e] : GAMMA_FLOOR;
          r += I->w[(size_t)m * I->K + k] * (st->alpha[e] * log2(g) + st->beta[e]);
        }
    double asum = 0.0;
    for (int n = 0; n < N; n++)
      for (int m = 0; m < M; m++)
        for (int s = 0; s < l; s++)
          if (st->S[slot(I, n, m, s)] == k) asum += st->alpha[slot(I, n, m, s)];
    double x = (I->Psi[ks] - r) / (asum > ZETA_ASUM_MIN ? asum : ZETA_ASUM_MIN);
    if (x > 1.0) x = 1.0;
    if (x < -1.0) x = -1.0;
    double z = st->zeta[ks] * exp2(delta * x);
    if (z > ZETA_MAX) z = ZETA_MAX;
    if (z < ZETA_MIN) z = ZETA_MIN;
    st->zeta[ks] = z;
  }
  for (int n = 0; n < N; n++) /* C14: Omega_bar <= 0 per selected pair */
    for (int m = 0; m < M; m++)
      for (int a = 0; a < l; a++)
        for (int b = a + 1; b < l; b++) {
          int ka = st->S[slot(I, n, m, a)], kb = st->S[slot(I, n, m, b)];
          if (ka < 0 || kb < 0) continue;
          double om = omega_bar(I, w->Ptot, n, m, ka, kb);
          size_t ix = ((size_t)n * M + m) * I->npair + pair_index(l, a, b);
          double ref = (I->sigma + inter_cell(I, w->Ptot, n, m, kb)) / gain(I, n, m, kb);
          double z = st->zsic[ix] + delta * (om / ref) / (LN2 * I->mask[m]);
          st->zsic[ix] = z > 0.0 ? z : 0.0;
        }
  sic_terms(I, st, w->SICp, w->SICm);

  /* closed-form KKT power of every selected link (Jacobi: all from the same p) */
  double dmax = 0.0;
  size_t L = (size_t)N * M * l;
  double *pnew = w->u; /* reuse */
  for (int n = 0; n < N; n++)
    for (int m = 0; m < M; m++)
      for (int s = 0; s < l; s++) {
        size_t e = slot(I, n, m, s);
        int k = st->S[e];
        if (k < 0) { pnew[e] = 0.0; continue; }
        double den = q * I->eta[m] + st->xi[m] +
                     victim_price(I, st, w->pi, n, m, k, -1) + w->SICp[(size_t)n * M + m];
        double num = weight_c(I, st, m, k) * st->alpha[e] / LN2 + w->SICm[(size_t)n * M + m] * st->plin[e];
        double pv;
        if (den <= 0.0 || num >= den * I->mask[m]) pv = I->mask[m];
        else pv = num / den;
        if (pv < I->pfloor[m]) pv = I->pfloor[m];
        pnew[e] = pv;
      }
  for (size_t e = 0; e < L; e++) {
    if (st->S[e] < 0) continue;
    double d = fabs(pnew[e] - st->p[e]) / I->mask[(e / l) % M];
    if (d > dmax) dmax = d;
    st->p[e] = w->noise_rel > 0.0 ? pnew[e] * (1.0 + w->noise_rel * noise_u(w)) : pnew[e];
  }
  return dmax;
}

/* alpha/beta update of Algorithm 1 at the current point */
static void scale_update(const inst_t *I, state_t *st, scratch_t *w) {
  rrh_totals(I, st, w->Ptot);
  link_quantities(I, st, w->Ptot, w->Ie, w->gam, w->pi);
  size_t L = (size_t)I->N * I->M * I->l;
  for (size_t e = 0; e < L; e++) {
    if (st->S[e] < 0) continue;
    double z = w->gam[e] > GAMMA_FLOOR ? w->gam[e] : GAMMA_FLOOR;
    orc_scale_coeffs(z, &st->alpha[e], &st->beta[e]);
  }
}

/* min over streaming users of (r_k - Psi_k) / Psi_k with exact rates (C13); 0 without streaming users */
static double rate_slack_min(const inst_t *I, const state_t *st, double *Ptot) {
  rrh_totals(I, st, Ptot);
  double rmin = 1e300;
  for (int ks = 0; ks < I->Ks; ks++) {
    int k = I->Ke + ks;
    double r = 0.0;
    for (int n = 0; n < I->N; n++)
      for (int m = 0; m < I->M; m++)
        for (int s = 0; s < I->l; s++) {
          size_t e = slot(I, n, m, s);
          if (st->S[e] != k) continue;
          double ie = noise_plus_interference(I, st, Ptot, n, m, s);
          r += I->w[(size_t)m * I->K + k] * log2(1.0 + st->p[e] * gain(I, n, m, k) / ie);
        }
    double sl = (r - I->Psi[ks]) / I->Psi[ks];
    if (sl < rmin) rmin = sl;
  }
  return I->Ks > 0 ? rmin : 0.0;
}

/* exact C12: scale an RRH's powers down when its total exceeds pmax */
static void project_power(const inst_t *I, state_t *st) {
  for (int m = 0; m < I->M; m++) {
    double tot = 0.0;
    for (int n = 0; n < I->N; n++)
      for (int s = 0; s < I->l; s++)
        if (st->S[slot(I, n, m, s)] >= 0) tot += st->p[slot(I, n, m, s)];
    if (tot > I->pmax[m]) {
      double f = I->pmax[m] / tot;
      for (int n = 0; n < I->N; n++)
        for (int s = 0; s < I->l; s++)
          if (st->S[slot(I, n, m, s)] >= 0) st->p[slot(I, n, m, s)] *= f;
    }
  }
}

/* ------------------------------------------------------------------ */
/* driver                                                               */
/* ------------------------------------------------------------------ */

int orc_solve(const orc_problem *pr, const orc_params *par, orc_result *out) {
  if (!pr || !par || !out || !pr->G || !pr->pmax || !pr->eta || !pr->Pc || !pr->Pf) return 1;
  if (pr->M < 1 || pr->N < 1 || pr->K < 1 || pr->Ks < 0 || pr->Ks > pr->K || pr->l < 1 ||
      pr->l > 64 || pr->Bn_hz <= 0 || pr->N0_w_per_hz <= 0)
    return 1;
  if (pr->Ks > 0 && (!pr->T_s || !pr->lambda_pps)) return 1;

  inst_t I;
  memset(&I, 0, sizeof(I));
  I.M = pr->M; I.N = pr->N; I.K = pr->K; I.Ks = pr->Ks; I.Ke = pr->K - pr->Ks; I.l = pr->l;
  I.npair = pr->l * (pr->l - 1) / 2;
  I.G = pr->G; I.pmax = pr->pmax; I.eta = pr->eta;
  I.sigma = pr->N0_w_per_hz * pr->Bn_hz;
  I.mask = malloc(sizeof(double) * I.M);
  I.pfloor = malloc(sizeof(double) * I.M);
  I.Psi = malloc(sizeof(double) * (I.Ks > 0 ? I.Ks : 1));
  I.w = malloc(sizeof(double) * (size_t)I.M * I.K);
  I.Pconst = 0.0;
  for (int m = 0; m < I.M; m++) {
    I.mask[m] = pr->pmax[m] / I.N;          /* spectral mask p^mask = pmax / N (Sec. VI) */
    I.pfloor[m] = P_FLOOR_REL * I.mask[m];
    I.Pconst += pr->Pc[m] + pr->Pf[m];      /* P_f^H + M_f P_f^L + M_f P_c^L + P_c^H */
  }
  for (int k = 0; k < I.Ks; k++) I.Psi[k] = orc_psi(pr->T_s[k], pr->lambda_pps[k], pr->zbar_bits, pr->Bn_hz);
  for (size_t t = 0; t < (size_t)I.M * I.K; t++) I.w[t] = pr->w ? pr->w[t] : 1.0;

  size_t L = (size_t)I.N * I.M * I.l;
  size_t NMK = (size_t)I.N * I.M * I.K;
  scratch_t w;
  w.Ptot = malloc(sizeof(double) * I.N * I.M);
  w.SICp = malloc(sizeof(double) * I.N * I.M);
  w.SICm = malloc(sizeof(double) * I.N * I.M);
  w.Ie = calloc(L, sizeof(double));
  w.gam = calloc(L, sizeof(double));
  w.pi = calloc(L, sizeof(double));
  w.u = calloc(NMK > L ? NMK : L, sizeof(double));
  w.pstar = calloc(NMK, sizeof(double));
  w.keys = calloc(NMK, sizeof(double));
  w.Xc = calloc(NMK, sizeof(double));
  w.ids = malloc(sizeof(int) * I.K);
  w.noise_rel = par->noise_rel;
  w.noise_seed = par->noise_seed;
  w.noise_ctr = 0;
  double *pstart = malloc(sizeof(double) * L);
  state_t st, prev;
  int ok = state_alloc(&I, &st) && state_alloc(&I, &prev) && w.Ptot && w.Ie && w.u && w.pstar &&
           w.keys && w.Xc && w.ids && pstart && I.mask && I.pfloor && I.Psi && I.w;
  int rc = 0;
  if (!ok) { rc = 2; goto done; }

  initial_state(&I, &st);
  double R = 0.0, P = 1.0;
  /* E^1 = R(p^0)/P(p^0) unless the caller fixes the starting E */
  exact_R_P(&I, &st, &R, &P, w.Ptot);
  double q = par->q_init > 0.0 ? par->q_init : R / P;
  if (out->q_trace) out->q_trace[0] = q;
  double slack_prev = rate_slack_min(&I, &st, w.Ptot), ee_best = R / P;
  double min_margin = 1.0;
  int n_ties = 0, it_d = 0, it_s = 0, it_v = 0, ntr = 0;
  const int Imax = par->max_dinkelbach > 0 ? par->max_dinkelbach : 1;
  const int Smax = par->max_scale > 0 ? par->max_scale : 1;
  const int Vmax = par->max_dual > 0 ? par->max_dual : 1;
  int status = ST_NOT_CONVERGED;

  for (int i = 0; i < Imax; i++) {
    state_copy(&I, &prev, &st); /* p^{i-1}, kept if Algorithm 1 ends below it */
    const double q_prev = q;
    int changed = select_links(&I, &st, q, &w, par->tie_eps, &min_margin, &n_ties);
    /* ---- Algorithm 1 at E^i = q ---- */
    for (size_t e = 0; e < L; e++) { st.alpha[e] = 1.0; st.beta[e] = 0.0; }
    for (int s = 0; s < Smax; s++) {
      for (size_t e = 0; e < L; e++) { pstart[e] = st.p[e]; st.plin[e] = st.p[e]; }
      for (int v = 0; v < Vmax; v++) {
        double d = dual_iteration(&I, &st, q, v, &w);
        it_v++;
        if (d < par->tol_dual) break;
      }
      scale_update(&I, &st, &w);
      it_s++;
      double dmax = 0.0;
      for (size_t e = 0; e < L; e++)
        if (st.S[e] >= 0) {
          double d = fabs(st.p[e] - pstart[e]) / I.mask[(e / I.l) % I.M];
          if (d > dmax) dmax = d;
        }
      if (out->scale_obj_trace && ntr < Imax * Smax) {
        double r_, p_;
        exact_R_P(&I, &st, &r_, &p_, w.Ptot);
        out->scale_obj_trace[ntr] = r_ - q * p_;
        if (out->scale_sel_changed) out->scale_sel_changed[ntr] = s == 0 ? changed : 0;
        ntr++;
      }
      if (dmax < par->tol_scale) break;
    }
    project_power(&I, &st);
    /* ---- Dinkelbach update ---- */
    exact_R_P(&I, &st, &R, &P, w.Ptot);
    double F = R - q * P;
    double qn = R / P;
    if (out->q_trace) out->q_trace[i + 1] = qn;
    if (out->F_trace) out->F_trace[i] = F;
    it_d++;
    const double slack = rate_slack_min(&I, &st, w.Ptot);
    if (F < 0.0) {
      /* the inner solve ended below p^{i-1}, which attains F = 0 (Lemma 1):
       * keep p^{i-1} and stop, unless p^{i-1} misses the streaming rates
       * that p^i meets better */
      if (slack_prev >= -1e-3 || slack_prev >= slack) {
        state_copy(&I, &st, &prev);
        q = q_prev;
        status = 0;
        break;
      }
      q = qn;
      slack_prev = slack;
      continue;
    }
    q = qn;
    slack_prev = slack;
    if (qn > ee_best) ee_best = qn;
    /* stop test of Sec. III (F <= xi, relative here) */
    if (F <= par->tol_dinkelbach * R) {
      status = 0;
      break;
    }
  }

  /* ---- report ---- */
  {
    double Rf, Pf;
    exact_R_P(&I, &st, &Rf, &Pf, w.Ptot);
    out->R = Rf; out->P = Pf; out->ee = Rf / Pf;
    /* slacks with exact rates */
    double smin = 1e300;
    for (int m = 0; m < I.M; m++) {
      double tot = 0.0;
      for (int n = 0; n < I.N; n++) tot += w.Ptot[(size_t)n * I.M + m];
      double sl = (I.pmax[m] - tot) / I.pmax[m];
      if (sl < smin) smin = sl;
    }
    out->slack_power_min = smin;
    double rmin = 1e300;
    for (int ks = 0; ks < I.Ks; ks++) {
      int k = I.Ke + ks;
      double r = 0.0;
      for (int n = 0; n < I.N; n++)
        for (int m = 0; m < I.M; m++)
          for (int s = 0; s < I.l; s++) {
            size_t e = slot(&I, n, m, s);
            if (st.S[e] != k) continue;
            double ie = noise_plus_interference(&I, &st, w.Ptot, n, m, s);
            r += I.w[(size_t)m * I.K + k] * log2(1.0 + st.p[e] * gain(&I, n, m, k) / ie);
          }
      double sl = (r - I.Psi[ks]) / I.Psi[ks];
      if (sl < rmin) rmin = sl;
    }
    out->slack_rate_min = I.Ks > 0 ? rmin : 0.0;
    if (I.Ks > 0 && rmin < -1e-3) status |= ST_STREAMING_UNMET;
    if (out->ee < ee_best * (1.0 - 1e-9)) status |= ST_EE_DECREASED;
    double smax = -1e300;
    int npairs = 0;
    for (int n = 0; n < I.N; n++)
      for (int m = 0; m < I.M; m++)
        for (int a = 0; a < I.l; a++)
          for (int b = a + 1; b < I.l; b++) {
            int ka = st.S[slot(&I, n, m, a)], kb = st.S[slot(&I, n, m, b)];
            if (ka < 0 || kb < 0) continue;
            double om = omega_bar(&I, w.Ptot, n, m, ka, kb) / I.mask[m];
            if (om > smax) smax = om;
            npairs++;
          }
    out->slack_sic_max = npairs ? smax : 0.0;
    out->iters[0] = it_d; out->iters[1] = it_s; out->iters[2] = it_v;
    out->status = status;
    out->min_margin = min_margin;
    out->n_ties = n_ties;
    out->n_scale_traced = ntr;
    if (out->A) memcpy(out->A, st.A, sizeof(int32_t) * I.K);
    if (out->S) memcpy(out->S, st.S, sizeof(int32_t) * L);
    if (out->p) memcpy(out->p, st.p, sizeof(double) * L);
    if (out->alpha) memcpy(out->alpha, st.alpha, sizeof(double) * L);
    if (out->beta) memcpy(out->beta, st.beta, sizeof(double) * L);
    if (out->xi) memcpy(out->xi, st.xi, sizeof(double) * I.M);
    if (out->zeta && I.Ks > 0) memcpy(out->zeta, st.zeta, sizeof(double) * I.Ks);
    if (out->zeta_sic && I.npair > 0)
      memcpy(out->zeta_sic, st.zsic, sizeof(double) * (size_t)I.N * I.M * I.npair);
  }

done:
  state_free(&st);
  state_free(&prev);
  free(w.Ptot); free(w.SICp); free(w.SICm); free(w.Ie); free(w.gam); free(w.pi);
  free(w.u); free(w.pstar); free(w.keys); free(w.Xc); free(w.ids);
  free(pstart);
  free(I.mask); free(I.pfloor); free(I.Psi); free(I.w);
  return rc;
}

/* ------------------------------------------------------------------ */
/* global-optimum comparator: brute force over assignments              */
/* ------------------------------------------------------------------ */
/*
 * Stands in for the paper's monotonic-optimisation optimum (Sec. IV-B) on
 * small instances with elastic users only.  Every RRH choice A_k in
 * {-1, .., M-1} and, on every (n, m), every subset of the users of m of at
 * most l members (every user with A_k >= 0 on at least one link) is an
 * assignment.  Enumeration order: A as a number in base M+1 (user 0 the
 * fastest digit, digit d meaning A_k = d - 1), then the subsets of (n, m) in
 * (n, m) order, n slowest, each (n, m) a digit over its subsets listed by size
 * then lexicographically (user ids ascending).  For each assignment the EE
 * (R over every link / P of the Sec. II-A power model) is maximised over the
 * powers by coordinate golden-section search in [1e-6 mask, mask] from three
 * starts p = f mask, f = 0.1, 0.4, 1: BF_SWEEPS sweeps over the links in
 * assignment order, BF_GOLDEN golden-section steps per link (the upper point
 * moves when the lower is at least as good), the midpoint kept when it
 * improves.  A point that breaks C12 (sum over m's links > pmax_m) or C14
 * (Omega_bar > 0 for a pair of the same (m, n) in SIC order) has value -1.
 */
#define BF_SWEEPS 8
#define BF_GOLDEN 40
#define BF_MAXL 16

typedef struct {
  int n, m, k;
} bf_link;

typedef struct {
  const inst_t *I;
  const bf_link *L;
  int nl;
} bf_ctx;

static double bf_value(const bf_ctx *c, const double *p) {
  const inst_t *I = c->I;
  double tot[64];
  for (int m = 0; m < I->M; m++) tot[m] = 0.0;
  for (int j = 0; j < c->nl; j++) tot[c->L[j].m] += p[j];
  for (int m = 0; m < I->M; m++)
    if (tot[m] > I->pmax[m] * (1.0 + 1e-12)) return -1.0;
  double R = 0.0, P = I->Pconst;
  for (int j = 0; j < c->nl; j++) {
    const bf_link a = c->L[j];
    double intra = 0.0, inter = 0.0;
    for (int i = 0; i < c->nl; i++) {
      const bf_link b = c->L[i];
      if (b.n != a.n) continue;
      if (b.m == a.m) {
        if (i != j && stronger(I, a.n, a.m, b.k, a.k)) intra += p[i];
        /* C14 for the pair (stronger a, weaker b) */
        if (i != j && stronger(I, a.n, a.m, a.k, b.k)) {
          double xa = 0.0, xb = 0.0;
          for (int q = 0; q < c->nl; q++) {
            const bf_link t = c->L[q];
            if (t.n != a.n || t.m == a.m) continue;
            xa += gain(I, a.n, t.m, a.k) * p[q];
            xb += gain(I, a.n, t.m, b.k) * p[q];
          }
          if ((I->sigma + xa) / gain(I, a.n, a.m, a.k) - (I->sigma + xb) / gain(I, a.n, a.m, b.k) > 0.0)
            return -1.0;
        }
      } else {
        inter += gain(I, a.n, b.m, a.k) * p[i];
      }
    }
    const double g = gain(I, a.n, a.m, a.k);
    R += I->w[(size_t)a.m * I->K + a.k] * log2(1.0 + p[j] * g / (I->sigma + g * intra + inter));
    P += I->eta[a.m] * p[j];
  }
  return R / P;
}

static double bf_search(const bf_ctx *c) {
  const inst_t *I = c->I;
  const double gr = (sqrt(5.0) - 1.0) / 2.0;
  const double starts[3] = {0.1, 0.4, 1.0};
  double best = -1.0, p[BF_MAXL], q[BF_MAXL];
  for (int st = 0; st < 3; st++) {
    for (int j = 0; j < c->nl; j++) p[j] = starts[st] * I->mask[c->L[j].m];
    double cur = bf_value(c, p);
    if (cur < 0.0) continue;
    for (int sw = 0; sw < BF_SWEEPS; sw++)
      for (int j = 0; j < c->nl; j++) {
        const double mk = I->mask[c->L[j].m];
        double lo = 1e-6 * mk, hi = mk;
        for (int i = 0; i < c->nl; i++) q[i] = p[i];
        for (int it = 0; it < BF_GOLDEN; it++) {
          const double a = hi - gr * (hi - lo), b = lo + gr * (hi - lo);
          q[j] = a;
          const double va = bf_value(c, q);
          q[j] = b;
          const double vb = bf_value(c, q);
          if (va >= vb) hi = b;
          else lo = a;
        }
        q[j] = 0.5 * (lo + hi);
        const double vn = bf_value(c, q);
        if (vn > cur) {
          p[j] = q[j];
          cur = vn;
        }
      }
    if (cur > best) best = cur;
  }
  return best;
}

int orc_bruteforce(const orc_problem *pr, double *best_ee, int64_t *n_assign, int64_t *best_index) {
  if (!pr || !best_ee || !pr->G || pr->Ks != 0 || pr->M < 1 || pr->M > 8 || pr->N < 1 || pr->K < 1 ||
      pr->K > 6 || pr->l < 1 || pr->l > 3 || (int64_t)pr->N * pr->M * pr->l > BF_MAXL)
    return 1;
  inst_t I;
  memset(&I, 0, sizeof(I));
  I.M = pr->M; I.N = pr->N; I.K = pr->K; I.Ks = 0; I.Ke = pr->K; I.l = pr->l;
  I.G = pr->G; I.pmax = pr->pmax; I.eta = pr->eta;
  I.sigma = pr->N0_w_per_hz * pr->Bn_hz;
  double mask[8], w[64];
  I.mask = mask;
  I.w = w;
  I.Pconst = 0.0;
  for (int m = 0; m < I.M; m++) {
    mask[m] = pr->pmax[m] / I.N;
    I.Pconst += pr->Pc[m] + pr->Pf[m];
  }
  for (int t = 0; t < I.M * I.K; t++) w[t] = pr->w ? pr->w[t] : 1.0;
  const int M = I.M, N = I.N, K = I.K, l = I.l, NM = N * M;
  int64_t nA = 1;
  for (int k = 0; k < K; k++) nA *= (M + 1);
  double best = 0.0;
  int64_t idx = 0, bidx = -1;
  int A[8];
  /* subsets of a user list of size <= l, by size then lexicographic */
  int subs[64][64][4], nsub[64], ssz[64][64];
  for (int64_t a = 0; a < nA; a++) {
    int64_t r = a;
    for (int k = 0; k < K; k++) { A[k] = (int)(r % (M + 1)) - 1; r /= (M + 1); }
    int64_t nch = 1;
    for (int nm = 0; nm < NM; nm++) {
      const int m = nm % M;
      int users[8], cnt = 0;
      for (int k = 0; k < K; k++) if (A[k] == m) users[cnt++] = k;
      int ns = 0;
      for (int sz = 0; sz <= (cnt < l ? cnt : l); sz++) {
        int comb[4];
        for (int i = 0; i < sz; i++) comb[i] = i;
        for (;;) {
          for (int i = 0; i < sz; i++) subs[nm][ns][i] = users[comb[i]];
          ssz[nm][ns] = sz;
          ns++;
          int i = sz - 1;
          while (i >= 0 && comb[i] == cnt - sz + i) i--;
          if (i < 0) break;
          comb[i]++;
          for (int j2 = i + 1; j2 < sz; j2++) comb[j2] = comb[j2 - 1] + 1;
        }
      }
      nsub[nm] = ns;
      nch *= ns;
    }
    for (int64_t ch = 0; ch < nch; ch++) {
      bf_link L[BF_MAXL];
      int nl = 0, served[8] = {0};
      int64_t rr = ch;
      /* digits: (n, m) in (n, m) order with n slowest, so the last (n, m) varies fastest */
      int digit[64];
      for (int nm = NM - 1; nm >= 0; nm--) { digit[nm] = (int)(rr % nsub[nm]); rr /= nsub[nm]; }
      for (int nm = 0; nm < NM; nm++)
        for (int i = 0; i < ssz[nm][digit[nm]]; i++) {
          L[nl].n = nm / M; L[nl].m = nm % M; L[nl].k = subs[nm][digit[nm]][i];
          served[L[nl].k] = 1;
          nl++;
        }
      int ok = nl > 0;
      for (int k = 0; k < K && ok; k++) if (A[k] >= 0 && !served[k]) ok = 0;
      if (!ok) continue;
      bf_ctx c = {&I, L, nl};
      const double v = bf_search(&c);
      if (v > best) { best = v; bidx = idx; }
      idx++;
    }
  }
  *best_ee = best;
  if (n_assign) *n_assign = idx;
  if (best_index) *best_index = bidx;
  return 0;
}
