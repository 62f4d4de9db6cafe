// hcran_pen.cu -- the paper-literal penalty form of the selection
// constraints on the GPU: a cross-check of the explicit selection.
//
// Sec. IV-A relaxes the binary RRH and subcarrier assignment into
//   C10  p_{m,k}^{(n)} p_{m',k}^{(n')} <= rho_1        (m != m'),
//   C11  product of the powers of l + 1 users on (m, n) <= rho_2,
// priced by the multipliers theta, theta' of eq. (653).  The main solver takes
// the rho -> 0 limit as an explicit selection; this kernel solves the penalty
// form itself for small instances (elastic users only), so that the two can be
// compared on the same inputs.  Every (m, k, n) link carries a power; the
// closed-form power of eq. (653) gets, besides the victim prices, E eta_m and
// xi'_m, the terms theta * p_{m',k}^{(n')} of the link's C10 partners and
// theta'_S * (product of the other powers of S) of the C11 sets S holding it.
// The iteration is the main method's (Dinkelbach loop of Sec. III around
// Algorithm 1: SCALE passes of dual loops, Jacobi power updates clipped to
// [1e-9 mask, mask], delta_v = 1/sqrt(v+1), the same stop norms and keep rule);
// the steps of the penalty multipliers are
//   theta  <- [theta  + delta_v clip((p p' - rho_1)/rho_1, -1, 1) / (ln2 mask_m mask_m')]+
//   theta' <- [theta' + delta_v clip((prod - rho_2)/rho_2, -1, 1) / (ln2 mask_m^(l+1))]+
// with rho_1 = rho_rel^2 mask_m mask_m', rho_2 = (rho_rel mask_m)^(l+1).
//
// One CTA solves one instance with one thread per link (at most 128 links):
// the state and every multiplier live in shared memory, and each dual
// iteration is four block-wide steps (RRH totals; interference, SINR and
// prices; multiplier steps; powers).  The arithmetic is FP64 throughout and
// every sum runs in the order the definitions list (this file is compiled
// without FMA contraction): the tool is a cross-check on small instances,
// where exact agreement with the CPU statement of the same form is worth more
// than speed.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <vector>

#include "../../include/hcran.h"

namespace {

constexpr int kPenThreads = 128;
constexpr int kPenMaxM = 4, kPenMaxN = 4, kPenMaxK = 8, kPenMaxL = 3;
constexpr double kLn2 = 0.69314718055994530942;

struct PenShape {
  int M, N, K, l, T;    // T = N M K links
  int npm, n10, nsub, n11;
  int64_t g_stride;     // gain elements per instance (T rounded up to 4)
};

// per-instance constants (host -> device)
struct PenConst {
  double pmax[kPenMaxM], eta[kPenMaxM], mask[kPenMaxM];
  double Pconst, sigma;
};

// per-instance results (device -> host)
struct PenOut {
  double ee, R, P, slack_power_min, c10_max, c11_max;
  int32_t iters[3];
  int32_t status;
};

struct PenTol {
  double tol_dinkelbach, tol_scale, tol_dual, q_init, rho_rel;
  int max_dinkelbach, max_scale, max_dual;
};

__device__ __forceinline__ int pen_pair10(const PenShape &s, int k, int m, int n, int m2, int n2) {
  const int mm = m * (2 * s.M - m - 1) / 2 + (m2 - m - 1);  // ordinal of (m, m2), m < m2
  return ((k * s.npm + mm) * s.N + n) * s.N + n2;
}

__device__ double pen_block_max(double v, double *red) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (lane == 0) red[w] = v;
  __syncthreads();
  double t = red[0];
  for (int i = 1; i < kPenThreads / 32; i++) t = fmax(t, red[i]);
  __syncthreads();
  return t;
}

struct PenSmem {
  double *p, *pnew, *alpha, *Ie, *gam, *pi, *pstart, *pprev, *G, *Ptot, *xi, *th10, *th11;
  unsigned char *rank, *sub;  // SIC rank of every link on its (n, m); the users of every C11 set
};

__device__ PenSmem pen_smem(const PenShape &s, double *base) {
  PenSmem m;
  double *b = base;
  m.p = b; b += s.T;
  m.pnew = b; b += s.T;
  m.alpha = b; b += s.T;
  m.Ie = b; b += s.T;
  m.gam = b; b += s.T;
  m.pi = b; b += s.T;
  m.pstart = b; b += s.T;
  m.pprev = b; b += s.T;
  m.G = b; b += s.T;
  m.Ptot = b; b += s.N * s.M;
  m.xi = b; b += s.M;
  m.th10 = b; b += s.n10 > 0 ? s.n10 : 1;
  m.th11 = b; b += s.n11 > 0 ? s.n11 : 1;
  m.rank = reinterpret_cast<unsigned char *>(b);
  m.sub = m.rank + s.T;
  return m;
}

// RRH totals, then interference and SINR of every link at sm.p
__device__ void pen_link(const PenShape &s, const PenConst &c, const PenSmem &sm) {
  const int M = s.M, K = s.K;
  for (int h = threadIdx.x; h < s.N * M; h += kPenThreads) {
    double t = 0.0;
    for (int k = 0; k < K; k++) t += sm.p[h * K + k];
    sm.Ptot[h] = t;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < s.T; e += kPenThreads) {
    const int k = e % K, m = (e / K) % M, n = e / (K * M);
    double intra = 0.0, inter = 0.0;
    for (int i = 0; i < K; i++)
      if (i != k && sm.rank[(n * M + m) * K + i] < sm.rank[e]) intra += sm.p[(n * M + m) * K + i];
    for (int j = 0; j < M; j++)
      if (j != m) inter += sm.G[(n * M + j) * K + k] * sm.Ptot[n * M + j];
    sm.Ie[e] = c.sigma + sm.G[e] * intra + inter;
    sm.gam[e] = sm.p[e] * sm.G[e] / sm.Ie[e];
  }
  __syncthreads();
}

// one dual iteration at sm.p; returns max |p_new - p| / mask
__device__ double pen_dual_iteration(const PenShape &s, const PenConst &c, const PenSmem &sm, const PenTol &tol,
                                     double q, int v, double *red) {
  const int M = s.M, N = s.N, K = s.K, l = s.l;
  pen_link(s, c, sm);
  for (int e = threadIdx.x; e < s.T; e += kPenThreads) sm.pi[e] = sm.alpha[e] / (kLn2 * sm.Ie[e]);
  const double delta = 1.0 / sqrt((double)v + 1.0);
  // multiplier steps: xi' (C12), then theta (C10), then theta' (C11), one per thread
  const int nstep = M + s.n10 + s.n11;
  for (int t = threadIdx.x; t < nstep; t += kPenThreads) {
    if (t < M) {
      const int m = t;
      double tot = 0.0;
      for (int n = 0; n < N; n++) tot += sm.Ptot[n * M + m];
      const double x = sm.xi[m] + delta * ((tot - c.pmax[m]) / c.pmax[m]) / (kLn2 * c.mask[m]);
      sm.xi[m] = x > 0.0 ? x : 0.0;
    } else if (t < M + s.n10) {
      const int i = t - M;  // ((k npm + mm) N + n) N + n2
      const int n2 = i % N, n = (i / N) % N, mm = (i / (N * N)) % s.npm, k = i / (N * N * s.npm);
      int m = 0, r = mm;
      while (r >= M - 1 - m) {
        r -= M - 1 - m;
        m++;
      }
      const int m2 = m + 1 + r;
      const double rho = tol.rho_rel * tol.rho_rel * c.mask[m] * c.mask[m2];
      const double prod = sm.p[(n * M + m) * K + k] * sm.p[(n2 * M + m2) * K + k];
      double rr = (prod - rho) / rho;
      rr = rr > 1.0 ? 1.0 : (rr < -1.0 ? -1.0 : rr);
      const double x = sm.th10[i] + delta * rr / (kLn2 * c.mask[m] * c.mask[m2]);
      sm.th10[i] = x > 0.0 ? x : 0.0;
    } else {
      const int i = t - M - s.n10;  // (n M + m) nsub + set
      const int cset = i % s.nsub, nm = i / s.nsub, m = nm % M;
      const double rho = pow(tol.rho_rel * c.mask[m], (double)(l + 1));
      double prod = 1.0;
      for (int u = 0; u <= l; u++) prod *= sm.p[nm * K + sm.sub[cset * (l + 1) + u]];
      double rr = (prod - rho) / rho;
      rr = rr > 1.0 ? 1.0 : (rr < -1.0 ? -1.0 : rr);
      const double x = sm.th11[i] + delta * rr / (kLn2 * pow(c.mask[m], (double)(l + 1)));
      sm.th11[i] = x > 0.0 ? x : 0.0;
    }
  }
  __syncthreads();
  double dmax = 0.0;
  for (int e = threadIdx.x; e < s.T; e += kPenThreads) {
    const int k = e % K, m = (e / K) % M, n = e / (K * M);
    double den = q * c.eta[m] + sm.xi[m];
    for (int i = 0; i < K; i++)  // weaker users of (m, n) hear this link
      if (i != k && sm.rank[e] < sm.rank[(n * M + m) * K + i]) den += sm.pi[(n * M + m) * K + i] * sm.G[(n * M + m) * K + i];
    for (int j = 0; j < M; j++)  // every user of the other RRHs on n
      if (j != m)
        for (int i = 0; i < K; i++) den += sm.pi[(n * M + j) * K + i] * sm.G[(n * M + m) * K + i];
    for (int m2 = 0; m2 < M; m2++) {  // C10 partners
      if (m2 == m) continue;
      for (int n2 = 0; n2 < N; n2++) {
        const int t = m < m2 ? pen_pair10(s, k, m, n, m2, n2) : pen_pair10(s, k, m2, n2, m, n);
        den += sm.th10[t] * sm.p[(n2 * M + m2) * K + k];
      }
    }
    for (int cs = 0; cs < s.nsub; cs++) {  // C11 sets of (m, n) holding k
      bool in = false;
      double prod = 1.0;
      for (int u = 0; u <= l; u++) {
        const int uk = sm.sub[cs * (l + 1) + u];
        if (uk == k) in = true;
        else prod *= sm.p[(n * M + m) * K + uk];
      }
      if (in) den += sm.th11[(n * M + m) * s.nsub + cs] * prod;
    }
    const double num = sm.alpha[e] / kLn2;
    const double mk = c.mask[m];
    double pv = (den <= 0.0 || num >= den * mk) ? mk : num / den;
    if (pv < 1e-9 * mk) pv = 1e-9 * mk;
    dmax = fmax(dmax, fabs(pv - sm.p[e]) / mk);
    sm.pnew[e] = pv;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < s.T; e += kPenThreads) sm.p[e] = sm.pnew[e];
  return pen_block_max(dmax, red);  // synchronises
}

// exact R (unit weights, every link) and P of the Sec. II-A power model, in link order
__device__ void pen_exact_R_P(const PenShape &s, const PenConst &c, const PenSmem &sm, double *rp) {
  pen_link(s, c, sm);
  if (threadIdx.x == 0) {
    double r = 0.0, tx = 0.0;
    for (int e = 0; e < s.T; e++) {
      r += log2(1.0 + sm.gam[e]);
      tx += c.eta[(e / s.K) % s.M] * sm.p[e];
    }
    rp[0] = r;
    rp[1] = c.Pconst + tx;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kPenThreads) pen_kernel(PenShape s, PenTol tol, const float *gains,
                                                          const PenConst *consts, PenOut *outs, double *p_out) {
  extern __shared__ __align__(16) double pen_dyn[];
  __shared__ double red[kPenThreads / 32];
  __shared__ double rp[2];
  const int b = blockIdx.x;
  const PenConst c = consts[b];
  const PenSmem sm = pen_smem(s, pen_dyn);
  const float *G = gains + (size_t)b * s.g_stride;
  const int M = s.M, N = s.N, K = s.K, l = s.l;
  for (int e = threadIdx.x; e < s.T; e += kPenThreads) {
    sm.G[e] = (double)G[e];
    sm.p[e] = c.mask[(e / K) % M] / K;
    sm.alpha[e] = 1.0;
  }
  for (int i = threadIdx.x; i < s.n10; i += kPenThreads) sm.th10[i] = 0.0;
  for (int i = threadIdx.x; i < s.n11; i += kPenThreads) sm.th11[i] = 0.0;
  for (int m = threadIdx.x; m < M; m += kPenThreads) sm.xi[m] = 0.0;
  if (threadIdx.x == 0) {
    // (l+1)-subsets of the users in lexicographic order
    int idx[kPenMaxL + 1];
    for (int u = 0; u <= l; u++) idx[u] = u;
    for (int cs = 0; cs < s.nsub; cs++) {
      for (int u = 0; u <= l; u++) sm.sub[cs * (l + 1) + u] = (unsigned char)idx[u];
      int u = l;
      while (u >= 0 && idx[u] == K - (l + 1) + u) u--;
      if (u < 0) break;
      idx[u]++;
      for (int w = u + 1; w <= l; w++) idx[w] = idx[w - 1] + 1;
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < s.T; e += kPenThreads) {  // SIC rank: gain descending, lower index first
    const int k = e % K, nm = e / K;
    int r = 0;
    for (int i = 0; i < K; i++) {
      const double gi = sm.G[nm * K + i], gk = sm.G[e];
      if (i != k && (gi > gk || (gi == gk && i < k))) r++;
    }
    sm.rank[e] = (unsigned char)r;
  }
  __syncthreads();
  pen_exact_R_P(s, c, sm, rp);
  double q = tol.q_init > 0.0 ? tol.q_init : rp[0] / rp[1];
  const int Imax = tol.max_dinkelbach > 0 ? tol.max_dinkelbach : 1;
  const int Smax = tol.max_scale > 0 ? tol.max_scale : 1;
  const int Vmax = tol.max_dual > 0 ? tol.max_dual : 1;
  int it_d = 0, it_s = 0, it_v = 0, status = 1;
  for (int i = 0; i < Imax; i++) {
    for (int e = threadIdx.x; e < s.T; e += kPenThreads) {
      sm.pprev[e] = sm.p[e];
      sm.alpha[e] = 1.0;
    }
    const double q_prev = q;
    __syncthreads();
    for (int sp = 0; sp < Smax; sp++) {
      for (int e = threadIdx.x; e < s.T; e += kPenThreads) sm.pstart[e] = sm.p[e];
      __syncthreads();
      for (int v = 0; v < Vmax; v++) {
        const double d = pen_dual_iteration(s, c, sm, tol, q, v, red);
        it_v++;
        if (d < tol.tol_dual) break;
      }
      pen_link(s, c, sm);
      double dm = 0.0;
      for (int e = threadIdx.x; e < s.T; e += kPenThreads) {
        const double z = sm.gam[e] > 1e-12 ? sm.gam[e] : 1e-12;
        sm.alpha[e] = z / (1.0 + z);
        dm = fmax(dm, fabs(sm.p[e] - sm.pstart[e]) / c.mask[(e / K) % M]);
      }
      it_s++;
      dm = pen_block_max(dm, red);
      if (dm < tol.tol_scale) break;
    }
    // exact C12
    if (threadIdx.x < M) {
      const int m = threadIdx.x;
      double tot = 0.0;
      for (int n = 0; n < N; n++)
        for (int k = 0; k < K; k++) tot += sm.p[(n * M + m) * K + k];
      red[m] = tot > c.pmax[m] ? c.pmax[m] / tot : 1.0;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < s.T; e += kPenThreads) {
      const double f = red[(e / K) % M];
      if (f < 1.0) sm.p[e] *= f;
    }
    __syncthreads();
    pen_exact_R_P(s, c, sm, rp);
    it_d++;
    const double F = rp[0] - q * rp[1];
    if (F < 0.0) {  // the inner solve ended below p^{i-1}: keep it
      for (int e = threadIdx.x; e < s.T; e += kPenThreads) sm.p[e] = sm.pprev[e];
      q = q_prev;
      status = 0;
      __syncthreads();
      break;
    }
    q = rp[0] / rp[1];
    if (F <= tol.tol_dinkelbach * rp[0]) {
      status = 0;
      break;
    }
  }
  pen_exact_R_P(s, c, sm, rp);
  if (threadIdx.x == 0) {
    PenOut o;
    o.ee = rp[0] / rp[1];
    o.R = rp[0];
    o.P = rp[1];
    o.iters[0] = it_d;
    o.iters[1] = it_s;
    o.iters[2] = it_v;
    o.status = status;
    double smin = 1e300, c10 = 0.0, c11 = 0.0;
    for (int m = 0; m < M; m++) {
      double tot = 0.0;
      for (int n = 0; n < N; n++) tot += sm.Ptot[n * M + m];
      const double sl = (c.pmax[m] - tot) / c.pmax[m];
      if (sl < smin) smin = sl;
    }
    for (int k = 0; k < K; k++)
      for (int m = 0; m < M; m++)
        for (int m2 = m + 1; m2 < M; m2++)
          for (int n = 0; n < N; n++)
            for (int n2 = 0; n2 < N; n2++) {
              const double r = sm.p[(n * M + m) * K + k] * sm.p[(n2 * M + m2) * K + k] /
                               (tol.rho_rel * tol.rho_rel * c.mask[m] * c.mask[m2]);
              if (r > c10) c10 = r;
            }
    for (int nm = 0; nm < N * M; nm++)
      for (int cs = 0; cs < s.nsub; cs++) {
        double prod = 1.0;
        for (int u = 0; u <= l; u++) prod *= sm.p[nm * K + sm.sub[cs * (l + 1) + u]];
        const double r = prod / pow(tol.rho_rel * c.mask[nm % M], (double)(l + 1));
        if (r > c11) c11 = r;
      }
    o.slack_power_min = smin;
    o.c10_max = c10;
    o.c11_max = c11;
    outs[b] = o;
  }
  for (int e = threadIdx.x; e < s.T; e += kPenThreads) p_out[(size_t)b * s.T + e] = sm.p[e];
}

int choose(int a, int b) {
  if (b < 0 || b > a) return 0;
  long r = 1;
  for (int i = 1; i <= b; i++) r = r * (a - b + i) / i;
  return (int)r;
}

bool pos(double x) { return isfinite(x) && x > 0.0; }

int pen_shape(const hcran_config *cfgs, int32_t n, PenShape &s) {
  if (!cfgs || n < 1) return HCRAN_EINVAL;
  const hcran_config &c0 = cfgs[0];
  s.M = c0.M; s.N = c0.N; s.K = c0.K; s.l = c0.l;
  if (s.M < 1 || s.M > kPenMaxM || s.N < 1 || s.N > kPenMaxN || s.K < 1 || s.K > kPenMaxK || s.l < 1 ||
      s.l > kPenMaxL)
    return HCRAN_EINVAL;
  s.T = s.N * s.M * s.K;
  if (s.T > kPenThreads) return HCRAN_EINVAL;
  s.npm = s.M * (s.M - 1) / 2;
  s.n10 = s.K * s.npm * s.N * s.N;
  s.nsub = choose(s.K, s.l + 1);
  s.n11 = s.N * s.M * s.nsub;
  s.g_stride = (s.T + 3) / 4 * 4;
  for (int32_t b = 0; b < n; b++) {
    const hcran_config &c = cfgs[b];
    if (c.M != s.M || c.N != s.N || c.K != s.K || c.l != s.l || c.Ks != 0) return HCRAN_EINVAL;
    if (!c.pmax || !c.eta || !c.Pc || !c.Pf || !pos(c.Bn_hz) || !pos(c.N0_w_per_hz)) return HCRAN_EINVAL;
    for (int m = 0; m < s.M; m++)
      if (!pos(c.pmax[m]) || !pos(c.eta[m]) || !(c.Pc[m] >= 0.0) || !(c.Pf[m] >= 0.0)) return HCRAN_EINVAL;
    if (c.w)
      for (int t = 0; t < s.M * s.K; t++)
        if (c.w[t] != 1.0) return HCRAN_EINVAL;
  }
  return HCRAN_OK;
}

size_t pen_smem_bytes(const PenShape &s) {
  return sizeof(double) * (9 * (size_t)s.T + (size_t)s.N * s.M + s.M + (s.n10 > 0 ? s.n10 : 1) +
                           (s.n11 > 0 ? s.n11 : 1)) +
         (size_t)s.T + (size_t)(s.nsub > 0 ? s.nsub : 1) * (s.l + 1);
}

uint64_t al256(uint64_t x) { return (x + 255) & ~uint64_t(255); }

struct PenLayout {
  uint64_t consts, outs, p, total;
};
PenLayout pen_layout(const PenShape &s, int32_t n) {
  PenLayout L;
  uint64_t o = 0;
  L.consts = o; o = al256(o + sizeof(PenConst) * (uint64_t)n);
  L.outs = o; o = al256(o + sizeof(PenOut) * (uint64_t)n);
  L.p = o; o = al256(o + sizeof(double) * (uint64_t)n * s.T);
  L.total = o;
  return L;
}

}  // namespace

extern "C" int hcran_penalty_workspace_size(const hcran_config *cfgs, int32_t n, uint64_t *bytes) {
  PenShape s;
  if (!bytes || pen_shape(cfgs, n, s) != HCRAN_OK) return HCRAN_EINVAL;
  *bytes = pen_layout(s, n).total;
  return HCRAN_OK;
}

extern "C" int hcran_penalty_solve(const hcran_config *cfgs, int32_t n, const float *gains_dev,
                                   const hcran_tol *tol, double rho_rel, void *workspace_dev, void *stream,
                                   double *ee, double *p, int32_t *iters, double *c10_max, double *c11_max) {
  PenShape s;
  if (!gains_dev || !tol || !workspace_dev || !ee || !(rho_rel > 0.0 && rho_rel < 1.0) ||
      (reinterpret_cast<uintptr_t>(gains_dev) & 15) || (reinterpret_cast<uintptr_t>(workspace_dev) & 255) ||
      pen_shape(cfgs, n, s) != HCRAN_OK)
    return HCRAN_EINVAL;
  if (!(tol->tol_dinkelbach >= 0.0) || !(tol->tol_scale >= 0.0) || !(tol->tol_dual >= 0.0) ||
      !(tol->q_init >= 0.0))
    return HCRAN_EINVAL;
  const PenLayout L = pen_layout(s, n);
  std::vector<PenConst> consts(n);
  for (int32_t b = 0; b < n; b++) {
    const hcran_config &c = cfgs[b];
    PenConst &d = consts[b];
    memset(&d, 0, sizeof(d));
    d.Pconst = 0.0;
    for (int m = 0; m < s.M; m++) {
      d.pmax[m] = c.pmax[m];
      d.eta[m] = c.eta[m];
      d.mask[m] = c.pmax[m] / s.N;
      d.Pconst += c.Pc[m] + c.Pf[m];
    }
    d.sigma = c.N0_w_per_hz * c.Bn_hz;
  }
  PenTol t;
  t.tol_dinkelbach = tol->tol_dinkelbach;
  t.tol_scale = tol->tol_scale;
  t.tol_dual = tol->tol_dual;
  t.q_init = tol->q_init;
  t.rho_rel = rho_rel;
  t.max_dinkelbach = tol->max_dinkelbach;
  t.max_scale = tol->max_scale;
  t.max_dual = tol->max_dual;
  char *ws = static_cast<char *>(workspace_dev);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // pageable source: staged before the call returns
  if (cudaMemcpyAsync(ws + L.consts, consts.data(), sizeof(PenConst) * n, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return HCRAN_ECUDA;
  const size_t smem = pen_smem_bytes(s);
  if (smem > 48 * 1024 && cudaFuncSetAttribute(pen_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem) != cudaSuccess)
    return HCRAN_ECUDA;
  pen_kernel<<<n, kPenThreads, smem, st>>>(s, t, gains_dev, reinterpret_cast<const PenConst *>(ws + L.consts),
                                           reinterpret_cast<PenOut *>(ws + L.outs),
                                           reinterpret_cast<double *>(ws + L.p));
  if (cudaGetLastError() != cudaSuccess) return HCRAN_ECUDA;
  std::vector<PenOut> outs(n);
  if (cudaMemcpyAsync(outs.data(), ws + L.outs, sizeof(PenOut) * n, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      (p && cudaMemcpyAsync(p, ws + L.p, sizeof(double) * (size_t)n * s.T, cudaMemcpyDeviceToHost, st) !=
                cudaSuccess) ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return HCRAN_ECUDA;
  for (int32_t b = 0; b < n; b++) {
    ee[b] = outs[b].ee;
    if (iters)
      for (int i = 0; i < 3; i++) iters[3 * b + i] = outs[b].iters[i];
    if (c10_max) c10_max[b] = outs[b].c10_max;
    if (c11_max) c11_max[b] = outs[b].c11_max;
  }
  return HCRAN_OK;
}
