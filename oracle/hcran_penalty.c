/*
 * hcran_penalty.c -- plain FP64 CPU oracle of the paper-literal penalty form
 * of the selection constraints (arXiv 1803.07772, Sec. IV-A: C10, C11 and
 * their multipliers theta, theta' in eq. (653)).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests and the benchmark's
 * comparison leg, never by the product path.  It shares no code with the
 * CUDA solver (nor with hcran_oracle.c, whose readings it restates where the
 * two forms agree).
 *
 * The main method takes the rho -> 0 limit of C10/C11 as an explicit
 * selection.  This form keeps them as the paper writes them: every
 * (RRH m, user k, subcarrier n) carries a power, and
 *   C10  p_{m,k}^{(n)} p_{m',k}^{(n')} <= rho_1   for m != m' (a user is
 *        served by one RRH),
 *   C11  the product of the powers of any l + 1 distinct users on (m, n)
 *        <= rho_2   (at most l users per subcarrier of an RRH; the paper
 *        writes l = 3, four factors)
 * are priced by the multipliers theta, theta' inside Algorithm 1.  In the
 * closed-form power of eq. (653) they add, for the link (m, k, n),
 *   sum over its C10 partners (m', n')   theta * p_{m',k}^{(n')}
 *   sum over its C11 sets S              theta'_S * prod_{u in S, u != k} p_u
 * to the denominator: the derivative of theta (p p' - rho_1) with respect to
 * log p, divided by p (each unordered pair and each set is one constraint
 * with one multiplier; the paper's factors 2 and 4 count its ordered copies).
 *
 * Everything else is the main method's iteration (hcran_oracle.c): the
 * Dinkelbach loop of Sec. III around Algorithm 1 (SCALE passes of dual
 * loops, alpha = 1 / beta = 0 at the start of each call), SINR of Sec. II-A
 * with the strict SIC order over all K users of (m, n), victim prices paid
 * for every user interfered with, E eta_m on every link, xi' for C12 with the
 * same step, Jacobi updates clipped to [1e-9 mask, mask], the same stopping
 * norms and the same keep rule for an inner solve that ends below its start.
 *
 * Readings of this form (the paper gives none of these values):
 *  - Scope: elastic users only (the comparison instances of the optimum have
 *    no streaming users).  C14 is not enforced: in its product form it is a
 *    three-factor term whose DC split the paper gives only garbled, and the
 *    divided form of the main method would bind pairs that C11 has switched
 *    off.  Its slack is reported on the result.
 *  - Initial point: p = mask_m / K on every link (C12 tight); multipliers 0.
 *  - rho_1 = rho_rel^2 mask_m mask_m', rho_2 = rho_rel^(l+1) mask_m^(l+1).
 *  - Steps, with the dual loop's delta_v = 1/sqrt(v+1):
 *      theta   <- [theta  + delta_v clip((p p'  - rho_1)/rho_1, -1, 1) / (ln2 mask_m mask_m')]+
 *      theta'  <- [theta' + delta_v clip((prod  - rho_2)/rho_2, -1, 1) / (ln2 mask_m^(l+1))]+
 *    so that one step changes a link's price by about that of a link at its
 *    mask (1 / (ln2 mask)), as the main method's steps do.
 *
 * Index conventions (shared with the result arrays):
 *  - links e = (n*M + m)*K + k (the gain array's order);
 *  - C10 pairs, per user k: every (m, n), (m', n') with m < m', listed
 *    k slowest, then m, m', n, n' (n' fastest);
 *  - C11 sets, per (n, m): the (l+1)-subsets of the K users in
 *    lexicographic order, n slowest, then m.
 */
#include "hcran_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define LN2 0.69314718055994530942
#define P_FLOOR_REL 1e-9
#define GAMMA_FLOOR 1e-12

typedef struct {
  int M, N, K, l;
  const float *G;
  double sigma, Pconst;
  double pmax[8], eta[8], mask[8];
  double rho_rel;
  int n10, n11, nsub;     /* C10 pairs, C11 sets, sets per (n, m) */
  int *sub;               /* [nsub][l+1] user ids of each set */
} pen_t;

static double gain(const pen_t *I, int n, int m, int k) { return (double)I->G[((size_t)n * I->M + m) * I->K + k]; }

/* user i is decoded after (is stronger than) user k on (m, n) */
static int stronger(const pen_t *I, int n, int m, int i, int k) {
  double gi = gain(I, n, m, i), gk = gain(I, n, m, k);
  return gi > gk || (gi == gk && i < k);
}

static int choose(int a, int b) {
  if (b < 0 || b > a) return 0;
  long r = 1;
  for (int i = 1; i <= b; i++) r = r * (a - b + i) / i;
  return (int)r;
}

/* index of the C10 pair of user k between (m, n) and (m2, n2), m < m2 */
static int pair10(const pen_t *I, int k, int m, int n, int m2, int n2) {
  int mm = 0; /* ordinal of (m, m2) among m < m2 */
  for (int a = 0; a < I->M; a++)
    for (int b = a + 1; b < I->M; b++) {
      if (a == m && b == m2) goto found;
      mm++;
    }
found:;
  int npm = I->M * (I->M - 1) / 2;
  return ((k * npm + mm) * I->N + n) * I->N + n2;
}

/* R (elastic, unit weights), P (every link) and the link quantities at p */
static void link(const pen_t *I, const double *p, double *Ptot, double *Ie, double *gam) {
  const int M = I->M, N = I->N, K = I->K;
  for (int n = 0; n < N; n++)
    for (int m = 0; m < M; m++) {
      double t = 0.0;
      for (int k = 0; k < K; k++) t += p[((size_t)n * M + m) * K + k];
      Ptot[n * M + m] = t;
    }
  for (int n = 0; n < N; n++)
    for (int m = 0; m < M; m++)
      for (int k = 0; k < K; k++) {
        size_t e = ((size_t)n * M + m) * K + k;
        double intra = 0.0, inter = 0.0;
        for (int i = 0; i < K; i++)
          if (i != k && stronger(I, n, m, i, k)) intra += p[((size_t)n * M + m) * K + i];
        for (int j = 0; j < M; j++)
          if (j != m) inter += gain(I, n, j, k) * Ptot[n * M + j];
        Ie[e] = I->sigma + gain(I, n, m, k) * intra + inter;
        gam[e] = p[e] * gain(I, n, m, k) / Ie[e];
      }
}

static void exact_R_P(const pen_t *I, const double *p, double *R, double *P, double *Ptot, double *Ie,
                      double *gam) {
  link(I, p, Ptot, Ie, gam);
  size_t L = (size_t)I->N * I->M * I->K;
  double r = 0.0, tx = 0.0;
  for (size_t e = 0; e < L; e++) {
    int m = (int)((e / I->K) % I->M);
    r += log2(1.0 + gam[e]);
    tx += I->eta[m] * p[e];
  }
  *R = r;
  *P = I->Pconst + tx;
}

typedef struct {
  double *p, *pnew, *alpha, *xi, *th10, *th11;
  double *Ptot, *Ie, *gam, *pi;
} pstate_t;

/* one dual iteration at p (Jacobi); returns max |p_new - p| / mask */
static double pen_dual_iteration(const pen_t *I, pstate_t *s, double q, int v) {
  const int M = I->M, N = I->N, K = I->K, l = I->l;
  link(I, s->p, s->Ptot, s->Ie, s->gam);
  size_t L = (size_t)N * M * K;
  for (size_t e = 0; e < L; e++) s->pi[e] = s->alpha[e] / (LN2 * s->Ie[e]);
  double delta = 1.0 / sqrt((double)v + 1.0);
  /* C12 */
  for (int m = 0; m < M; m++) {
    double tot = 0.0;
    for (int n = 0; n < N; n++) tot += s->Ptot[n * M + m];
    double x = s->xi[m] + delta * ((tot - I->pmax[m]) / I->pmax[m]) / (LN2 * I->mask[m]);
    s->xi[m] = x > 0.0 ? x : 0.0;
  }
  /* C10 */
  for (int k = 0; k < K; k++)
    for (int m = 0; m < M; m++)
      for (int m2 = m + 1; m2 < M; m2++)
        for (int n = 0; n < N; n++)
          for (int n2 = 0; n2 < N; n2++) {
            int t = pair10(I, k, m, n, m2, n2);
            double rho = I->rho_rel * I->rho_rel * I->mask[m] * I->mask[m2];
            double prod = s->p[((size_t)n * M + m) * K + k] * s->p[((size_t)n2 * M + m2) * K + k];
            double r = (prod - rho) / rho;
            if (r > 1.0) r = 1.0;
            if (r < -1.0) r = -1.0;
            double x = s->th10[t] + delta * r / (LN2 * I->mask[m] * I->mask[m2]);
            s->th10[t] = x > 0.0 ? x : 0.0;
          }
  /* C11 */
  for (int n = 0; n < N; n++)
    for (int m = 0; m < M; m++) {
      double rho = pow(I->rho_rel * I->mask[m], l + 1);
      for (int c = 0; c < I->nsub; c++) {
        double prod = 1.0;
        for (int u = 0; u <= l; u++) prod *= s->p[((size_t)n * M + m) * K + I->sub[c * (l + 1) + u]];
        double r = (prod - rho) / rho;
        if (r > 1.0) r = 1.0;
        if (r < -1.0) r = -1.0;
        size_t t = ((size_t)n * M + m) * I->nsub + c;
        double x = s->th11[t] + delta * r / (LN2 * pow(I->mask[m], l + 1));
        s->th11[t] = x > 0.0 ? x : 0.0;
      }
    }
  /* closed-form power of every link */
  double dmax = 0.0;
  for (int n = 0; n < N; n++)
    for (int m = 0; m < M; m++)
      for (int k = 0; k < K; k++) {
        size_t e = ((size_t)n * M + m) * K + k;
        double den = q * I->eta[m] + s->xi[m];
        /* victims: weaker users of (m, n), every user of the other RRHs on n */
        for (int i = 0; i < K; i++)
          if (i != k && stronger(I, n, m, k, i)) den += s->pi[((size_t)n * M + m) * K + i] * gain(I, n, m, i);
        for (int j = 0; j < M; j++)
          if (j != m)
            for (int i = 0; i < K; i++) den += s->pi[((size_t)n * M + j) * K + i] * gain(I, n, m, i);
        /* C10 partners of (m, k, n) */
        for (int m2 = 0; m2 < M; m2++) {
          if (m2 == m) continue;
          for (int n2 = 0; n2 < N; n2++) {
            int t = m < m2 ? pair10(I, k, m, n, m2, n2) : pair10(I, k, m2, n2, m, n);
            den += s->th10[t] * s->p[((size_t)n2 * M + m2) * K + k];
          }
        }
        /* C11 sets of (m, n) that contain k */
        for (int c = 0; c < I->nsub; c++) {
          int in = 0;
          double prod = 1.0;
          for (int u = 0; u <= l; u++) {
            int uk = I->sub[c * (l + 1) + u];
            if (uk == k) in = 1;
            else prod *= s->p[((size_t)n * M + m) * K + uk];
          }
          if (in) den += s->th11[((size_t)n * M + m) * I->nsub + c] * prod;
        }
        double num = s->alpha[e] / LN2;
        double mk = I->mask[m];
        double pv = (den <= 0.0 || num >= den * mk) ? mk : num / den;
        if (pv < P_FLOOR_REL * mk) pv = P_FLOOR_REL * mk;
        double d = fabs(pv - s->p[e]) / mk;
        if (d > dmax) dmax = d;
        s->pnew[e] = pv;
      }
  memcpy(s->p, s->pnew, sizeof(double) * L);
  return dmax;
}

int orc_penalty_solve(const orc_problem *pr, const orc_params *par, double rho_rel, orc_pen_result *out) {
  if (!pr || !par || !out || pr->Ks != 0 || pr->M < 1 || pr->M > 8 || pr->N < 1 || pr->K < 1 || pr->l < 1 ||
      !(rho_rel > 0.0 && rho_rel < 1.0))
    return 1;
  pen_t I;
  memset(&I, 0, sizeof(I));
  I.M = pr->M; I.N = pr->N; I.K = pr->K; I.l = pr->l; I.G = pr->G;
  I.sigma = pr->N0_w_per_hz * pr->Bn_hz;
  I.rho_rel = rho_rel;
  I.Pconst = 0.0;
  for (int m = 0; m < I.M; m++) {
    I.pmax[m] = pr->pmax[m];
    I.eta[m] = pr->eta[m];
    I.mask[m] = pr->pmax[m] / I.N;
    I.Pconst += pr->Pc[m] + pr->Pf[m];
  }
  if (pr->w)
    for (int t = 0; t < I.M * I.K; t++)
      if (pr->w[t] != 1.0) return 1;  /* unit weights only */
  I.n10 = I.K * (I.M * (I.M - 1) / 2) * I.N * I.N;
  I.nsub = choose(I.K, I.l + 1);
  I.n11 = I.N * I.M * I.nsub;
  I.sub = malloc(sizeof(int) * (size_t)(I.nsub > 0 ? I.nsub : 1) * (I.l + 1));
  if (!I.sub) return 2;
  { /* (l+1)-subsets in lexicographic order */
    int c = 0, idx[16];
    for (int u = 0; u <= I.l; u++) idx[u] = u;
    while (I.nsub > 0 && c < I.nsub) {
      for (int u = 0; u <= I.l; u++) I.sub[c * (I.l + 1) + u] = idx[u];
      c++;
      int u = I.l;
      while (u >= 0 && idx[u] == I.K - (I.l + 1) + u) u--;
      if (u < 0) break;
      idx[u]++;
      for (int w = u + 1; w <= I.l; w++) idx[w] = idx[w - 1] + 1;
    }
  }
  const size_t L = (size_t)I.N * I.M * I.K;
  pstate_t s;
  s.p = calloc(L, sizeof(double));
  s.pnew = calloc(L, sizeof(double));
  s.alpha = calloc(L, sizeof(double));
  s.xi = calloc(I.M, sizeof(double));
  s.th10 = calloc(I.n10 > 0 ? I.n10 : 1, sizeof(double));
  s.th11 = calloc(I.n11 > 0 ? I.n11 : 1, sizeof(double));
  s.Ptot = calloc((size_t)I.N * I.M, sizeof(double));
  s.Ie = calloc(L, sizeof(double));
  s.gam = calloc(L, sizeof(double));
  s.pi = calloc(L, sizeof(double));
  double *pstart = calloc(L, sizeof(double)), *pprev = calloc(L, sizeof(double));
  int rc = 0;
  if (!s.p || !s.pnew || !s.alpha || !s.xi || !s.th10 || !s.th11 || !s.Ptot || !s.Ie || !s.gam || !s.pi ||
      !pstart || !pprev) {
    rc = 2;
    goto done;
  }
  for (size_t e = 0; e < L; e++) s.p[e] = I.mask[(e / I.K) % I.M] / I.K;
  double R, P;
  exact_R_P(&I, s.p, &R, &P, s.Ptot, s.Ie, s.gam);
  double q = par->q_init > 0.0 ? par->q_init : R / P;
  const int Imax = par->max_dinkelbach > 0 ? par->max_dinkelbach : 1;
  const int Smax = par->max_scale > 0 ? par->max_scale : 1;
  const int Vmax = par->max_dual > 0 ? par->max_dual : 1;
  int it_d = 0, it_s = 0, it_v = 0, status = 1;
  for (int i = 0; i < Imax; i++) {
    memcpy(pprev, s.p, sizeof(double) * L);
    const double q_prev = q;
    for (size_t e = 0; e < L; e++) s.alpha[e] = 1.0;
    for (int sp = 0; sp < Smax; sp++) {
      memcpy(pstart, s.p, sizeof(double) * L);
      for (int v = 0; v < Vmax; v++) {
        double d = pen_dual_iteration(&I, &s, q, v);
        it_v++;
        if (d < par->tol_dual) break;
      }
      /* alpha at the new point */
      link(&I, s.p, s.Ptot, s.Ie, s.gam);
      for (size_t e = 0; e < L; e++) {
        double z = s.gam[e] > GAMMA_FLOOR ? s.gam[e] : GAMMA_FLOOR;
        s.alpha[e] = z / (1.0 + z);
      }
      it_s++;
      double dmax = 0.0;
      for (size_t e = 0; e < L; e++) {
        double d = fabs(s.p[e] - pstart[e]) / I.mask[(e / I.K) % I.M];
        if (d > dmax) dmax = d;
      }
      if (dmax < par->tol_scale) break;
    }
    /* exact C12 */
    for (int m = 0; m < I.M; m++) {
      double tot = 0.0;
      for (int n = 0; n < I.N; n++)
        for (int k = 0; k < I.K; k++) tot += s.p[((size_t)n * I.M + m) * I.K + k];
      if (tot > I.pmax[m]) {
        double f = I.pmax[m] / tot;
        for (int n = 0; n < I.N; n++)
          for (int k = 0; k < I.K; k++) s.p[((size_t)n * I.M + m) * I.K + k] *= f;
      }
    }
    exact_R_P(&I, s.p, &R, &P, s.Ptot, s.Ie, s.gam);
    it_d++;
    double F = R - q * P;
    if (F < 0.0) { /* the inner solve ended below p^{i-1}: keep it */
      memcpy(s.p, pprev, sizeof(double) * L);
      q = q_prev;
      status = 0;
      break;
    }
    q = R / P;
    if (F <= par->tol_dinkelbach * R) {
      status = 0;
      break;
    }
  }
  exact_R_P(&I, s.p, &R, &P, s.Ptot, s.Ie, s.gam);
  out->ee = R / P;
  out->R = R;
  out->P = P;
  out->iters[0] = it_d;
  out->iters[1] = it_s;
  out->iters[2] = it_v;
  out->status = status;
  { /* slacks: C12, the largest C10 / C11 products relative to rho, C14 */
    double smin = 1e300, c10 = 0.0, c11 = 0.0, c14 = -1e300;
    for (int m = 0; m < I.M; m++) {
      double tot = 0.0;
      for (int n = 0; n < I.N; n++) tot += s.Ptot[n * I.M + m];
      double sl = (I.pmax[m] - tot) / I.pmax[m];
      if (sl < smin) smin = sl;
    }
    for (int k = 0; k < I.K; k++)
      for (int m = 0; m < I.M; m++)
        for (int m2 = m + 1; m2 < I.M; m2++)
          for (int n = 0; n < I.N; n++)
            for (int n2 = 0; n2 < I.N; n2++) {
              double r = s.p[((size_t)n * I.M + m) * I.K + k] * s.p[((size_t)n2 * I.M + m2) * I.K + k] /
                         (I.rho_rel * I.rho_rel * I.mask[m] * I.mask[m2]);
              if (r > c10) c10 = r;
            }
    for (int n = 0; n < I.N; n++)
      for (int m = 0; m < I.M; m++)
        for (int c = 0; c < I.nsub; c++) {
          double prod = 1.0;
          for (int u = 0; u <= I.l; u++) prod *= s.p[((size_t)n * I.M + m) * I.K + I.sub[c * (I.l + 1) + u]];
          double r = prod / pow(I.rho_rel * I.mask[m], I.l + 1);
          if (r > c11) c11 = r;
        }
    /* C14 (divided form) over pairs of links both above rho_rel mask */
    for (int n = 0; n < I.N; n++)
      for (int m = 0; m < I.M; m++)
        for (int a = 0; a < I.K; a++)
          for (int b = 0; b < I.K; b++) {
            if (a == b || !stronger(&I, n, m, a, b)) continue;
            double pa = s.p[((size_t)n * I.M + m) * I.K + a], pb = s.p[((size_t)n * I.M + m) * I.K + b];
            if (pa <= I.rho_rel * I.mask[m] || pb <= I.rho_rel * I.mask[m]) continue;
            double xa = 0.0, xb = 0.0;
            for (int j = 0; j < I.M; j++)
              if (j != m) {
                xa += gain(&I, n, j, a) * s.Ptot[n * I.M + j];
                xb += gain(&I, n, j, b) * s.Ptot[n * I.M + j];
              }
            double om = (I.sigma + xa) / gain(&I, n, m, a) - (I.sigma + xb) / gain(&I, n, m, b);
            if (om / I.mask[m] > c14) c14 = om / I.mask[m];
          }
    out->slack_power_min = smin;
    out->c10_max = c10;
    out->c11_max = c11;
    out->slack_sic_max = c14 > -1e300 ? c14 : 0.0;
  }
  if (out->p) memcpy(out->p, s.p, sizeof(double) * L);
  if (out->alpha) memcpy(out->alpha, s.alpha, sizeof(double) * L);
  if (out->xi) memcpy(out->xi, s.xi, sizeof(double) * I.M);
  if (out->theta) memcpy(out->theta, s.th10, sizeof(double) * (size_t)I.n10);
  if (out->theta2) memcpy(out->theta2, s.th11, sizeof(double) * (size_t)I.n11);
  out->n_theta = I.n10;
  out->n_theta2 = I.n11;
done:
  free(I.sub);
  free(s.p); free(s.pnew); free(s.alpha); free(s.xi); free(s.th10); free(s.th11);
  free(s.Ptot); free(s.Ie); free(s.gam); free(s.pi); free(pstart); free(pprev);
  return rc;
}
