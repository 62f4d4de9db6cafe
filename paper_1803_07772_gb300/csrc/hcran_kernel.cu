// hcran_kernel.cu -- persistent batched solver for sm_103a.
//
// One CTA (512 threads) solves one instance at a time and pulls the next one
// from an LPT-ordered queue (instances sorted by M*N*K, largest first).  The
// whole method runs inside the CTA, so no inter-CTA wait exists:
//
//   p^0 (gain-based RRH choice, l strongest users, p = mask/l); E^1 = R/P
//   Dinkelbach i (Sec. III):  selection  ->  Algorithm 1  ->  E^{i+1} = R/P
//     selection (C1/C5 via C10/C11 with rho -> 0): water-filling utility of
//       every (m,k,n) at the current prices, A_k = argmax_m sum_n, then per
//       (m,n) greedy admission by utility under SIC feasibility (C14)
//     Algorithm 1 (Sec. IV-A): alpha = 1, beta = 0; SCALE passes, each a
//       dual loop of [interference/SINR/prices -> projected subgradient on
//       xi', zeta', zeta_sic' -> closed-form KKT power of eq. (653)/(683)],
//       then alpha/beta at the new point (eq. scale_approximation)
//
// Work mapping: subcarriers map to warps (interference, SIC order and prices
// of one subcarrier stay inside a warp); per-RRH and per-user sums are warp
// reductions in a fixed order, so results are bit-reproducible run to run.
// The gains of the selected users are repacked once per selection into a
// compact slab slab[n][j][u] = Gamma_{j, user(u)}^{(n)} (u = m*l + s), which is
// all the dual loop reads.  Precision: FP32 for SINR, prices, powers and
// residuals; FP64 for q = R/P, the F(q) test, R and P sums and the multiplier
// values that accumulate the subgradient steps.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "hcran_layout.h"

namespace hcran {

#define LN2F 0.69314718f
#define LN2D 0.69314718055994530942

constexpr float kPFloorRel = 1e-9f;
constexpr float kGammaFloor = 1e-12f;
constexpr double kZetaAsumMin = 0.05;
constexpr double kZetaMin = 1e-6, kZetaMax = 1e6;

struct Ctx {
  int M, N, K, Ks, Ke, l, U, L, npair, nchunk;
  const float *G;  // Gamma[n][m][k]
  const double *pmax, *eta, *mask, *Psi, *w;
  double *xi, *zeta, *zsic;
  float *p, *plin, *pstart, *alpha, *beta, *pi, *gam, *X, *slab, *SICp, *SICm, *Ptot, *cu, *cp,
      *cX, *ckey, *Upart;
  int *A, *Anew, *S, *uslot;
  float sigma;
  double Pconst;
};

struct Shared {
  float maskf[kMaxM], floorf[kMaxM], etaf[kMaxM], xif[kMaxM], fac[kMaxM];
  float pio[kWarps][kMaxM];
  double redd[kWarps];
  float redf[kWarps];
  int redi[kWarps];
  int inst;
  int changed;
  float min_margin;
  int n_ties;
};

// ------------------------------------------------------------------ helpers

__device__ __forceinline__ float warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_max(float v) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float warp_min(float v) {
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ int warp_isum(int v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block reductions: fixed tree, result broadcast to every thread
__device__ double block_sum(double v, Shared &sh) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  v = warp_sum(v);
  if (lane == 0) sh.redd[warp] = v;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < kWarps; i++) t += sh.redd[i];
  __syncthreads();
  return t;
}
__device__ float block_max(float v, Shared &sh) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  v = warp_max(v);
  if (lane == 0) sh.redf[warp] = v;
  __syncthreads();
  float t = sh.redf[0];
  for (int i = 1; i < kWarps; i++) t = fmaxf(t, sh.redf[i]);
  __syncthreads();
  return t;
}
__device__ float block_min(float v, Shared &sh) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  v = warp_min(v);
  if (lane == 0) sh.redf[warp] = v;
  __syncthreads();
  float t = sh.redf[0];
  for (int i = 1; i < kWarps; i++) t = fminf(t, sh.redf[i]);
  __syncthreads();
  return t;
}
__device__ int block_isum(int v, Shared &sh) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  v = warp_isum(v);
  if (lane == 0) sh.redi[warp] = v;
  __syncthreads();
  int t = 0;
  for (int i = 0; i < kWarps; i++) t += sh.redi[i];
  __syncthreads();
  return t;
}

__device__ __forceinline__ float gain(const Ctx &c, int n, int m, int k) {
  return __ldg(c.G + ((size_t)n * c.M + m) * c.K + k);
}
// slab[n][j][u] = Gamma_{j, user in slot u}^{(n)}
__device__ __forceinline__ float sgain(const Ctx &c, int n, int j, int u) {
  return c.slab[((size_t)n * c.M + j) * c.U + u];
}
// SIC order on (m,n): user a decoded after (is stronger than) user b
__device__ __forceinline__ bool stronger(float ga, int a, float gb, int b) {
  return ga > gb || (ga == gb && a < b);
}
__device__ __forceinline__ float weight_c(const Ctx &c, int m, int k) {
  float w = (float)c.w[(size_t)m * c.K + k];
  return k >= c.Ke ? (float)c.zeta[k - c.Ke] * w : w;
}
__device__ __forceinline__ int pair_index(int l, int a, int b) {
  return a * l - a * (a + 1) / 2 + (b - a - 1);
}
__device__ __forceinline__ void track(float margin, float eps, float &mm, int &nt) {
  mm = fminf(mm, margin);
  if (margin < eps) nt++;
}

// ------------------------------------------------------------------ model pieces

// Per subcarrier (one warp): RRH totals Ptot[n][j], then for every selected
// slot the inter-cell interference X, SINR gamma and victim price
// pi = c alpha / (ln2 (sigma + I)).  Sec. II-A SINR with the SIC order.
__device__ void link_pass(const Ctx &c) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int n = warp; n < c.N; n += kWarps) {
    const int base = n * c.U;
    for (int j = lane; j < c.M; j += 32) {
      float t = 0.f;
      for (int s = 0; s < c.l; s++) {
        const int e = base + j * c.l + s;
        if (c.S[e] >= 0) t += c.p[e];
      }
      c.Ptot[n * c.M + j] = t;
    }
    __syncwarp();
    for (int u = lane; u < c.U; u += 32) {
      const int e = base + u;
      const int k = c.S[e];
      if (k < 0) {
        c.gam[e] = 0.f;
        c.pi[e] = 0.f;
        c.X[e] = 0.f;
        continue;
      }
      const int m = u / c.l, s = u - m * c.l;
      float inter = 0.f;
      for (int j = 0; j < c.M; j++)
        if (j != m) inter += sgain(c, n, j, u) * c.Ptot[n * c.M + j];
      float intra = 0.f;
      for (int b = 0; b < s; b++) {
        const int eb = base + m * c.l + b;
        if (c.S[eb] >= 0) intra += c.p[eb];
      }
      const float g = sgain(c, n, m, u);
      const float ie = c.sigma + g * intra + inter;
      c.X[e] = inter;
      c.gam[e] = c.p[e] * g / ie;
      c.pi[e] = weight_c(c, m, k) * c.alpha[e] / (LN2F * ie);
    }
    __syncwarp();
  }
  __syncthreads();
}

// SIC multiplier sums per (n, j) from the pairs of the other RRHs on n:
// Omega_bar of a pair (a stronger, b weaker) on (m,n) has coefficient
// Gamma_{j,a}/Gamma_{m,a} - Gamma_{j,b}/Gamma_{m,b} on Ptot_j.
__device__ void sic_terms(const Ctx &c) {
  for (int nj = threadIdx.x; nj < c.N * c.M; nj += kThreads) {
    const int n = nj / c.M, j = nj - n * c.M;
    float sp = 0.f, sm = 0.f;
    if (c.npair > 0)
      for (int m = 0; m < c.M; m++) {
        if (m == j) continue;
        const int base = n * c.U + m * c.l;
        const double *z = c.zsic + ((size_t)n * c.M + m) * c.npair;
        for (int a = 0; a < c.l; a++) {
          if (c.S[base + a] < 0) break;
          for (int b = a + 1; b < c.l; b++) {
            if (c.S[base + b] < 0) break;
            const double zz = z[pair_index(c.l, a, b)];
            if (zz == 0.0) continue;
            const int ua = m * c.l + a, ub = m * c.l + b;
            const float cc = sgain(c, n, j, ua) / sgain(c, n, m, ua) - sgain(c, n, j, ub) / sgain(c, n, m, ub);
            if (cc > 0.f) sp += (float)zz * cc;
            else sm += (float)zz * (-cc);
          }
        }
      }
    c.SICp[nj] = sp;
    c.SICm[nj] = sm;
  }
  __syncthreads();
}

// Projected subgradient step on every multiplier from the residuals at the
// current point (computed by link_pass).
__device__ void multipliers(const Ctx &c, int v) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const double delta = 1.0 / sqrt((double)v + 1.0);
  for (int it = warp; it < c.M + c.Ks; it += kWarps) {
    if (it < c.M) {  // C12
      const int m = it;
      double t = 0.0;
      for (int n = lane; n < c.N; n += 32) t += (double)c.Ptot[n * c.M + m];
      t = warp_sum(t);
      if (lane == 0) {
        const double res = (t - c.pmax[m]) / c.pmax[m];
        const double x = c.xi[m] + delta * res / (LN2D * c.mask[m]);
        c.xi[m] = x > 0.0 ? x : 0.0;
      }
    } else {  // C13 hat, log-scale step
      const int ks = it - c.M, k = c.Ke + ks;
      float r = 0.f, as = 0.f;
      const int a = c.A[k];
      if (a >= 0) {
        const float wk = (float)c.w[(size_t)a * c.K + k];
        for (int n = lane; n < c.N; n += 32) {
          const int u = c.uslot[(size_t)k * c.N + n];
          if (u < 0) continue;
          const int e = n * c.U + u;
          const float g = fmaxf(c.gam[e], kGammaFloor);
          r += wk * (c.alpha[e] * log2f(g) + c.beta[e]);
          as += c.alpha[e];
        }
      }
      r = warp_sum(r);
      as = warp_sum(as);
      if (lane == 0) {
        double x = (c.Psi[ks] - (double)r) / fmax((double)as, kZetaAsumMin);
        x = fmin(fmax(x, -1.0), 1.0);
        double z = c.zeta[ks] * exp2(x);
        c.zeta[ks] = fmin(fmax(z, kZetaMin), kZetaMax);
      }
    }
  }
  if (c.npair > 0)  // C14 per selected pair
    for (int nm = threadIdx.x; nm < c.N * c.M; nm += kThreads) {
      const int n = nm / c.M, m = nm - n * c.M;
      const int base = n * c.U + m * c.l;
      for (int a = 0; a < c.l; a++) {
        if (c.S[base + a] < 0) break;
        for (int b = a + 1; b < c.l; b++) {
          if (c.S[base + b] < 0) break;
          const float ga = sgain(c, n, m, m * c.l + a), gb = sgain(c, n, m, m * c.l + b);
          const float ra = (c.sigma + c.X[base + a]) / ga;
          const float rb = (c.sigma + c.X[base + b]) / gb;
          const size_t ix = (size_t)nm * c.npair + pair_index(c.l, a, b);
          const double z = c.zsic[ix] + delta * ((double)(ra - rb) / (double)rb) / (LN2D * c.mask[m]);
          c.zsic[ix] = z > 0.0 ? z : 0.0;
        }
      }
    }
  __syncthreads();
  sic_terms(c);
}

// Closed-form KKT power of every selected slot (eq. 653 / 683 in the
// log-power variable, Jacobi: all slots from the same point).  Returns the
// block-wide max |p_new - p| / mask.
__device__ float power_update(const Ctx &c, double q, Shared &sh) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float dmax = 0.f;
  for (int m = threadIdx.x; m < c.M; m += kThreads) sh.xif[m] = (float)c.xi[m];
  __syncthreads();
  for (int n = warp; n < c.N; n += kWarps) {
    float *pio = sh.pio[warp];
    const float *pin = c.pi + n * c.U;
    // price paid on n by a transmitter of RRH j towards the other RRHs' users
    for (int j = lane; j < c.M; j += 32) {
      const float *row = c.slab + ((size_t)n * c.M + j) * c.U;
      float acc = 0.f;
      for (int jj = 0; jj < c.M; jj++) {
        if (jj == j) continue;
        for (int s = 0; s < c.l; s++) acc += row[jj * c.l + s] * pin[jj * c.l + s];
      }
      pio[j] = acc;
    }
    __syncwarp();
    for (int u = lane; u < c.U; u += 32) {
      const int e = n * c.U + u;
      const int k = c.S[e];
      if (k < 0) continue;
      const int m = u / c.l, s = u - m * c.l;
      const float *row = c.slab + ((size_t)n * c.M + m) * c.U;
      float own = 0.f;  // weaker users of the same (m,n) hear this slot
      for (int b = s + 1; b < c.l; b++) {
        const int ub = m * c.l + b;
        if (c.S[n * c.U + ub] >= 0) own += pin[ub] * row[ub];
      }
      const float den = (k < c.Ke ? (float)(q * c.eta[m]) : 0.f) + sh.xif[m] + pio[m] + own +
                        c.SICp[n * c.M + m];
      const float num = weight_c(c, m, k) * c.alpha[e] / LN2F + c.SICm[n * c.M + m] * c.plin[e];
      const float mk = sh.maskf[m];
      float pv = (den <= 0.f || num >= den * mk) ? mk : num / den;
      pv = fmaxf(pv, sh.floorf[m]);
      dmax = fmaxf(dmax, fabsf(pv - c.p[e]) / mk);
      c.p[e] = pv;
    }
    __syncwarp();
  }
  return block_max(dmax, sh);
}

// alpha/beta of the SCALE bound at the current point
__device__ void scale_update(const Ctx &c) {
  link_pass(c);
  for (int e = threadIdx.x; e < c.L; e += kThreads) {
    if (c.S[e] < 0) continue;
    const float z = fmaxf(c.gam[e], kGammaFloor);
    const float a = z / (1.f + z);
    c.alpha[e] = a;
    c.beta[e] = log1pf(z) / LN2F - a * log2f(z);
  }
  __syncthreads();
}

// exact R (elastic, weighted) and P of problem (eq7); FP64 accumulation
__device__ void exact_R_P(const Ctx &c, Shared &sh, double &R, double &P) {
  link_pass(c);
  double r = 0.0, tx = 0.0;
  for (int e = threadIdx.x; e < c.L; e += kThreads) {
    const int k = c.S[e];
    if (k < 0 || k >= c.Ke) continue;
    const int m = (e % c.U) / c.l;
    r += (double)c.w[(size_t)m * c.K + k] * (double)(log1pf(c.gam[e]) / LN2F);
    tx += c.eta[m] * (double)c.p[e];
  }
  R = block_sum(r, sh);
  P = c.Pconst + block_sum(tx, sh);
}

// exact C12: scale an RRH's powers down when its total exceeds pmax
__device__ void project_power(const Ctx &c, Shared &sh) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int m = warp; m < c.M; m += kWarps) {
    double t = 0.0;
    for (int n = lane; n < c.N; n += 32)
      for (int s = 0; s < c.l; s++) {
        const int e = n * c.U + m * c.l + s;
        if (c.S[e] >= 0) t += (double)c.p[e];
      }
    t = warp_sum(t);
    if (lane == 0) sh.fac[m] = t > c.pmax[m] ? (float)(c.pmax[m] / t) : 1.f;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < c.L; e += kThreads) {
    if (c.S[e] < 0) continue;
    const int m = (e % c.U) / c.l;
    const float f = sh.fac[m];
    if (f < 1.f) c.p[e] *= f;
  }
  __syncthreads();
}

// ------------------------------------------------------------------ selection

// Water-filling candidate of user k on (m, n) at the current prices:
// maximise c log2(1 + g p) - den p on [0, mask].
__device__ float cand_utility(const Ctx &c, const Shared &sh, double q, int n, int m, int k,
                              float *ps_out, float *X_out, float *key_out) {
  const int a = c.A[k];
  float pk = 0.f;
  if (a >= 0) {
    const int u = c.uslot[(size_t)k * c.N + n];
    if (u >= 0) pk = c.p[n * c.U + u];
  }
  float X = 0.f;
  for (int j = 0; j < c.M; j++)
    if (j != m) X += gain(c, n, j, k) * (c.Ptot[n * c.M + j] - (j == a ? pk : 0.f));
  const float gk = gain(c, n, m, k);
  float Y = 0.f, Pi = 0.f;
  for (int j = 0; j < c.M; j++)
    for (int b = 0; b < c.l; b++) {
      const int ub = j * c.l + b;
      const int v = c.S[n * c.U + ub];
      if (v < 0) break;
      if (v == k) continue;
      if (j != m) {
        Pi += c.pi[n * c.U + ub] * sgain(c, n, m, ub);
      } else {
        const float gv = sgain(c, n, m, ub);
        if (stronger(gv, v, gk, k)) Y += c.p[n * c.U + ub];
        else Pi += c.pi[n * c.U + ub] * gv;
      }
    }
  const float g = gk / (c.sigma + X + gk * Y);
  const float den = (k < c.Ke ? (float)(q * c.eta[m]) : 0.f) + (float)c.xi[m] + Pi + c.SICp[n * c.M + m];
  const float cw = weight_c(c, m, k);
  const float mk = sh.maskf[m];
  float ps;
  if (cw <= 0.f) ps = 0.f;
  else if (den <= 0.f) ps = mk;
  else {
    const float x = cw / (LN2F * den) - 1.f / g;
    ps = x <= 0.f ? 0.f : (x >= mk ? mk : x);
  }
  const float u = ps > 0.f ? cw * (log1pf(g * ps) / LN2F) - den * ps : 0.f;
  if (ps_out) {
    *ps_out = ps;
    *X_out = X;
    *key_out = (cw > 0.f && den > 0.f) ? fabsf(cw * g - LN2F * den) / fmaxf(cw * g, LN2F * den) : 1.f;
  }
  return u;
}

__device__ void build_slab(const Ctx &c) {
  for (int t = threadIdx.x; t < c.K * c.N; t += kThreads) c.uslot[t] = -1;
  __syncthreads();
  for (int e = threadIdx.x; e < c.L; e += kThreads) {
    const int k = c.S[e];
    if (k >= 0) c.uslot[(size_t)k * c.N + e / c.U] = e % c.U;
  }
  const int MU = c.M * c.U;
  for (int t = threadIdx.x; t < c.N * MU; t += kThreads) {
    const int n = t / MU, r = t - n * MU, j = r / c.U, u = r - j * c.U;
    const int k = c.S[n * c.U + u];
    c.slab[t] = k >= 0 ? gain(c, n, j, k) : 0.f;
  }
  __syncthreads();
}

// next candidate of (m, n) in (utility desc, user asc) order after (lu, lk)
__device__ int next_candidate(const Ctx &c, int n, int m, float lu, int lk, float &bu) {
  int bk = -1;
  bu = 0.f;
  const float *un = c.cu + (size_t)n * c.K;
  for (int k = 0; k < c.K; k++) {
    if (c.Anew[k] != m) continue;
    const float u = un[k];
    if (!(u < lu || (u == lu && k > lk))) continue;
    if (bk < 0 || u > bu || (u == bu && k < bk)) {
      bu = u;
      bk = k;
    }
  }
  return bk;
}

// Returns 1 when the selection changed.
__device__ int selection(const Ctx &c, Shared &sh, double q, float tie_eps) {
  link_pass(c);
  sic_terms(c);
  float mm = 1.f;
  int nt = 0;
  if (threadIdx.x == 0) sh.changed = 0;
  // (A) per-chunk sums over n of the candidate utilities
  const int nch = c.nchunk;
  for (int t = threadIdx.x; t < nch * c.K; t += kThreads) {
    const int ch = t / c.K, k = t - ch * c.K;
    const int n0 = (int)((int64_t)c.N * ch / nch), n1 = (int)((int64_t)c.N * (ch + 1) / nch);
    float *up = c.Upart + (size_t)ch * c.M * c.K + k;
    for (int m = 0; m < c.M; m++) {
      float acc = 0.f;
      for (int n = n0; n < n1; n++) acc += cand_utility(c, sh, q, n, m, k, nullptr, nullptr, nullptr);
      up[(size_t)m * c.K] = acc;
    }
  }
  __syncthreads();
  // (B) A_k = argmax_m sum_n u, lowest m on equal sums, -1 when all zero
  int ch_local = 0;
  for (int k = threadIdx.x; k < c.K; k += kThreads) {
    int best = -1;
    float b1 = 0.f, b2 = 0.f;
    for (int m = 0; m < c.M; m++) {
      float U = 0.f;
      for (int ch = 0; ch < nch; ch++) U += c.Upart[((size_t)ch * c.M + m) * c.K + k];
      if (U > b1) {
        b2 = b1;
        b1 = U;
        best = m;
      } else if (U > b2) {
        b2 = U;
      }
    }
    if (best >= 0 && b2 > 0.f) track((b1 - b2) / b1, tie_eps, mm, nt);
    c.Anew[k] = best;
    if (best != c.A[k]) ch_local = 1;
  }
  __syncthreads();
  // (C) the candidate of every (n, k) on its chosen RRH
  for (int t = threadIdx.x; t < c.N * c.K; t += kThreads) {
    const int n = t / c.K, k = t - n * c.K;
    const int m = c.Anew[k];
    if (m < 0) {
      c.cu[t] = 0.f;
      c.cp[t] = 0.f;
      c.cX[t] = 0.f;
      c.ckey[t] = 1.f;
      continue;
    }
    float ps, X, key;
    c.cu[t] = cand_utility(c, sh, q, n, m, k, &ps, &X, &key);
    c.cp[t] = ps;
    c.cX[t] = X;
    c.ckey[t] = key;
  }
  __syncthreads();
  // (D) greedy SIC-feasible admission per (n, m); new state written in place
  for (int nm = threadIdx.x; nm < c.N * c.M; nm += kThreads) {
    const int n = nm / c.M, m = nm - n * c.M;
    int chosen[kMaxL];
    int nc = 0;
    float lu = INFINITY, bu;
    int lk = -1;
    while (nc < c.l) {
      const int bk = next_candidate(c, n, m, lu, lk, bu);
      if (bk < 0) break;
      lu = bu;
      lk = bk;
      track(c.ckey[(size_t)n * c.K + bk], tie_eps, mm, nt);
      if (!(bu > 0.f)) break;
      bool feasible = true;
      const float gk = gain(c, n, m, bk);
      for (int i = 0; i < nc && feasible; i++) {
        const int o = chosen[i];
        const float go = gain(c, n, m, o);
        const bool kfirst = stronger(gk, bk, go, o);
        const int a = kfirst ? bk : o, b = kfirst ? o : bk;
        const float ga = kfirst ? gk : go, gb = kfirst ? go : gk;
        const float ra = (c.sigma + c.cX[(size_t)n * c.K + a]) / ga;
        const float rb = (c.sigma + c.cX[(size_t)n * c.K + b]) / gb;
        track(fabsf(ra - rb) / fmaxf(ra, rb), tie_eps, mm, nt);
        if (ra - rb > 0.f) feasible = false;
      }
      if (feasible) chosen[nc++] = bk;
    }
    if (nc == c.l) {
      float bu2;
      const int k2 = next_candidate(c, n, m, lu, lk, bu2);
      const float ul = c.cu[(size_t)n * c.K + chosen[c.l - 1]];
      if (k2 >= 0 && bu2 > 0.f) track((ul - bu2) / ul, tie_eps, mm, nt);
    }
    // SIC order: gain descending, lower id first
    float cg[kMaxL];
    for (int i = 0; i < nc; i++) cg[i] = gain(c, n, m, chosen[i]);
    for (int i = 1; i < nc; i++) {
      const int x = chosen[i];
      const float gx = cg[i];
      int j = i - 1;
      while (j >= 0 && stronger(gx, x, cg[j], chosen[j])) {
        chosen[j + 1] = chosen[j];
        cg[j + 1] = cg[j];
        j--;
      }
      chosen[j + 1] = x;
      cg[j + 1] = gx;
    }
    const int base = n * c.U + m * c.l;
    int oldk[kMaxL];
    float oldp[kMaxL], oldl[kMaxL];
    bool same = true;
    for (int s = 0; s < c.l; s++) {
      oldk[s] = c.S[base + s];
      oldp[s] = c.p[base + s];
      oldl[s] = c.plin[base + s];
      if (oldk[s] != (s < nc ? chosen[s] : -1)) same = false;
    }
    for (int s = 0; s < c.l; s++) {
      const int e = base + s;
      if (s >= nc) {
        c.S[e] = -1;
        c.p[e] = 0.f;
        c.plin[e] = 0.f;
      } else {
        const int k = chosen[s];
        int old = -1;
        for (int b = 0; b < c.l; b++)
          if (oldk[b] == k) old = b;
        c.S[e] = k;
        if (old >= 0) {
          c.p[e] = oldp[old];
          c.plin[e] = oldl[old];
        } else {
          c.p[e] = c.cp[(size_t)n * c.K + k];
          c.plin[e] = c.p[e];
        }
      }
      c.alpha[e] = 1.f;
      c.beta[e] = 0.f;
    }
    if (!same) {
      ch_local = 1;
      for (int pr = 0; pr < c.npair; pr++) c.zsic[(size_t)nm * c.npair + pr] = 0.0;
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < c.K; k += kThreads) c.A[k] = c.Anew[k];
  __syncthreads();
  build_slab(c);
  // fold decision margins and the change flag
  const float bm = block_min(mm, sh);
  const int bt = block_isum(nt, sh);
  const int anych = block_isum(ch_local, sh);
  if (threadIdx.x == 0) {
    sh.min_margin = fminf(sh.min_margin, bm);
    sh.n_ties += bt;
  }
  __syncthreads();
  return anych > 0;
}

// ------------------------------------------------------------------ initial point

__device__ void initial_state(const Ctx &c) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // A_k = argmax_m sum_n Gamma_{m,k}^{(n)}
  for (int k = threadIdx.x; k < c.K; k += kThreads) {
    int best = 0;
    float bv = -1.f;
    for (int m = 0; m < c.M; m++) {
      float t = 0.f;
      for (int n = 0; n < c.N; n++) t += gain(c, n, m, k);
      if (t > bv) {
        bv = t;
        best = m;
      }
    }
    c.A[k] = best;
  }
  __syncthreads();
  // S_{m,n}: the l strongest users of m (already in SIC order); p = mask / l
  for (int nm = warp; nm < c.N * c.M; nm += kWarps) {
    const int n = nm / c.M, m = nm - n * c.M;
    float pg = INFINITY;
    int pk = -1;
    const float p0 = (float)(c.mask[m] / c.l);
    for (int s = 0; s < c.l; s++) {
      float bg = -1.f;
      int bk = -1;
      for (int k = lane; k < c.K; k += 32) {
        if (c.A[k] != m) continue;
        const float g = gain(c, n, m, k);
        if (!(g < pg || (g == pg && k > pk))) continue;
        if (bk < 0 || stronger(g, k, bg, bk)) {
          bg = g;
          bk = k;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const float og = __shfl_xor_sync(0xffffffffu, bg, o);
        const int ok = __shfl_xor_sync(0xffffffffu, bk, o);
        if (ok >= 0 && (bk < 0 || stronger(og, ok, bg, bk))) {
          bg = og;
          bk = ok;
        }
      }
      if (lane == 0) {
        const int e = n * c.U + m * c.l + s;
        c.S[e] = bk;
        c.p[e] = bk >= 0 ? p0 : 0.f;
        c.plin[e] = c.p[e];
        c.alpha[e] = 1.f;
        c.beta[e] = 0.f;
      }
      if (bk < 0) {
        for (int s2 = s + 1 + lane; s2 < c.l; s2 += 32) {
          const int e = n * c.U + m * c.l + s2;
          c.S[e] = -1;
          c.p[e] = 0.f;
          c.plin[e] = 0.f;
          c.alpha[e] = 1.f;
          c.beta[e] = 0.f;
        }
        break;
      }
      pg = bg;
      pk = bk;
    }
  }
  for (int m = threadIdx.x; m < c.M; m += kThreads) c.xi[m] = 0.0;
  for (int k = threadIdx.x; k < c.Ks; k += kThreads) c.zeta[k] = 1.0;
  for (int t = threadIdx.x; t < c.N * c.M * c.npair; t += kThreads) c.zsic[t] = 0.0;
  __syncthreads();
  build_slab(c);
}

// ------------------------------------------------------------------ driver

__device__ void solve_instance(const Ctx &c, Shared &sh, const Tol &tol, InstOut *out) {
  for (int m = threadIdx.x; m < c.M; m += kThreads) {
    sh.maskf[m] = (float)c.mask[m];
    sh.floorf[m] = (float)c.mask[m] * kPFloorRel;
    sh.etaf[m] = (float)c.eta[m];
  }
  if (threadIdx.x == 0) {
    sh.min_margin = 1.f;
    sh.n_ties = 0;
  }
  __syncthreads();
  initial_state(c);
  double R, P;
  exact_R_P(c, sh, R, P);
  double q = tol.q_init > 0.0 ? tol.q_init : R / P;
  int it_d = 0, it_s = 0, it_v = 0, status = 1;  // not converged until the stop test fires
  const int Imax = tol.max_dinkelbach > 0 ? tol.max_dinkelbach : 1;
  const int Smax = tol.max_scale > 0 ? tol.max_scale : 1;
  const int Vmax = tol.max_dual > 0 ? tol.max_dual : 1;
  for (int i = 0; i < Imax; i++) {
    selection(c, sh, q, tol.tie_eps);
    // Algorithm 1 at E^i = q (alpha = 1, beta = 0 written by the selection)
    for (int s = 0; s < Smax; s++) {
      for (int e = threadIdx.x; e < c.L; e += kThreads) {
        c.pstart[e] = c.p[e];
        c.plin[e] = c.p[e];
      }
      __syncthreads();
      for (int v = 0; v < Vmax; v++) {
        link_pass(c);
        multipliers(c, v);
        const float d = power_update(c, q, sh);
        it_v++;
        if (d < (float)tol.tol_dual) break;
      }
      scale_update(c);
      it_s++;
      float dm = 0.f;
      for (int e = threadIdx.x; e < c.L; e += kThreads)
        if (c.S[e] >= 0) dm = fmaxf(dm, fabsf(c.p[e] - c.pstart[e]) / sh.maskf[(e % c.U) / c.l]);
      dm = block_max(dm, sh);
      if (dm < (float)tol.tol_scale) break;
    }
    project_power(c, sh);
    exact_R_P(c, sh, R, P);
    it_d++;
    if (!isfinite(R) || !isfinite(P) || P <= 0.0) {
      status = 8;
      break;
    }
    const double F = R - q * P;
    q = R / P;
    if (F <= tol.tol_dinkelbach * R) {
      status = F < 0.0 ? 4 : 0;
      break;
    }
  }
  // slacks (exact rates from the last link_pass inside exact_R_P)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float smin = INFINITY;
  for (int m = warp; m < c.M; m += kWarps) {
    double t = 0.0;
    for (int n = lane; n < c.N; n += 32) t += (double)c.Ptot[n * c.M + m];
    t = warp_sum(t);
    smin = fminf(smin, (float)((c.pmax[m] - t) / c.pmax[m]));
  }
  const float slack_power = block_min(smin, sh);
  float rmin = INFINITY;
  for (int ks = warp; ks < c.Ks; ks += kWarps) {
    const int k = c.Ke + ks;
    const int a = c.A[k];
    float r = 0.f;
    if (a >= 0) {
      const float wk = (float)c.w[(size_t)a * c.K + k];
      for (int n = lane; n < c.N; n += 32) {
        const int u = c.uslot[(size_t)k * c.N + n];
        if (u >= 0) r += wk * log1pf(c.gam[n * c.U + u]) / LN2F;
      }
    }
    r = warp_sum(r);
    rmin = fminf(rmin, (float)((r - c.Psi[ks]) / c.Psi[ks]));
  }
  const float slack_rate = block_min(rmin, sh);
  float smax = -INFINITY;
  for (int nm = threadIdx.x; nm < c.N * c.M; nm += kThreads) {
    const int n = nm / c.M, m = nm - n * c.M;
    const int base = n * c.U + m * c.l;
    for (int a = 0; a < c.l; a++) {
      if (c.S[base + a] < 0) break;
      for (int b = a + 1; b < c.l; b++) {
        if (c.S[base + b] < 0) break;
        const float ra = (c.sigma + c.X[base + a]) / sgain(c, n, m, m * c.l + a);
        const float rb = (c.sigma + c.X[base + b]) / sgain(c, n, m, m * c.l + b);
        smax = fmaxf(smax, (ra - rb) / sh.maskf[m]);
      }
    }
  }
  const float slack_sic = block_max(smax, sh);
  if (threadIdx.x == 0) {
    if (c.Ks > 0 && slack_rate < -1e-3f) status |= 2;
    out->ee = R / P;
    out->R = R;
    out->P = P;
    out->iters[0] = it_d;
    out->iters[1] = it_s;
    out->iters[2] = it_v;
    out->status = status;
    out->slack_power_min = slack_power;
    out->slack_rate_min = c.Ks > 0 ? slack_rate : 0.0;
    out->slack_sic_max = isfinite(slack_sic) ? slack_sic : 0.0;
    out->min_margin = sh.min_margin;
    out->n_ties = sh.n_ties;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kThreads, 1)
    solve_kernel(const InstDesc *__restrict__ descs, const int *__restrict__ order, int n_inst,
                 const float *__restrict__ gains, double *darena, float *farena, int *iarena,
                 InstOut *outs, Tol tol, int *counter) {
  __shared__ Shared sh;
  for (;;) {
    if (threadIdx.x == 0) sh.inst = atomicAdd(counter, 1);
    __syncthreads();
    const int w = sh.inst;
    __syncthreads();
    if (w >= n_inst) break;
    const int b = order[w];
    const InstDesc d = descs[b];
    Ctx c;
    c.M = d.M; c.N = d.N; c.K = d.K; c.Ks = d.Ks; c.Ke = d.K - d.Ks; c.l = d.l;
    c.U = d.U; c.L = d.L; c.npair = d.npair; c.nchunk = d.nchunk;
    c.G = gains + d.g_off;
    c.sigma = (float)d.sigma;
    c.Pconst = d.Pconst;
    const DLayout dl = dlayout(d.M, d.N, d.K, d.Ks, d.l);
    double *db = darena + d.d_off;
    c.pmax = db + dl.pmax; c.eta = db + dl.eta; c.mask = db + dl.mask; c.Psi = db + dl.Psi;
    c.w = db + dl.w; c.xi = db + dl.xi; c.zeta = db + dl.zeta; c.zsic = db + dl.zsic;
    const FLayout fl = flayout(d.M, d.N, d.K, d.l, d.nchunk);
    float *fb = farena + d.f_off;
    c.p = fb + fl.p; c.plin = fb + fl.plin; c.pstart = fb + fl.pstart; c.alpha = fb + fl.alpha;
    c.beta = fb + fl.beta; c.pi = fb + fl.pi; c.gam = fb + fl.gam; c.X = fb + fl.X;
    c.slab = fb + fl.slab; c.SICp = fb + fl.SICp; c.SICm = fb + fl.SICm; c.Ptot = fb + fl.Ptot;
    c.cu = fb + fl.cu; c.cp = fb + fl.cp; c.cX = fb + fl.cX; c.ckey = fb + fl.ckey;
    c.Upart = fb + fl.Upart;
    const ILayout il = ilayout(d.M, d.N, d.K, d.l);
    int *ib = iarena + d.i_off;
    c.A = ib + il.A; c.Anew = ib + il.Anew; c.S = ib + il.S; c.uslot = ib + il.uslot;
    solve_instance(c, sh, tol, outs + b);
  }
}

cudaError_t launch_solve(const InstDesc *descs, const int *order, int n_inst, const float *gains,
                         double *darena, float *farena, int *iarena, InstOut *outs, const Tol &tol,
                         int *counter, cudaStream_t stream, int *launches) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (err != cudaSuccess) return err;
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, solve_kernel, kThreads, 0);
  if (err != cudaSuccess) return err;
  if (per_sm < 1) per_sm = 1;
  int grid = sms * per_sm;
  if (grid > n_inst) grid = n_inst;
  if (grid < 1) grid = 1;
  err = cudaMemsetAsync(counter, 0, sizeof(int), stream);
  if (err != cudaSuccess) return err;
  solve_kernel<<<grid, kThreads, 0, stream>>>(descs, order, n_inst, gains, darena, farena, iarena,
                                               outs, tol, counter);
  *launches = 1;
  return cudaGetLastError();
}

}  // namespace hcran
