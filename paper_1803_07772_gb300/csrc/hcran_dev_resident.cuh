// hcran_dev_resident.cuh -- the dual loop of Algorithm 1 on shared-memory
// resident state (internal).
//
// At the start of a dual loop the CTA copies, for its subcarriers, the compact
// slab, the slot arrays and the SIC multipliers into shared memory (structure
// of arrays, sized by res_floats); every dual iteration then works on shared
// memory only, and the powers, the committed multipliers and xi', zeta' go
// back to global memory at the end.
//
// One iteration is three block-wide stages, each over a flat index space so
// that every thread has work and long independent loops:
//   sums    per (n, j): the prices a transmitter of RRH j pays towards the
//           other RRHs' users (row j of the slab against pi) and the SIC+ /
//           SIC- sums of row j over the nonzero SIC multipliers of n; beside
//           them, on the last warps, the residual sums over n (RRH totals,
//           streaming rates) and the projected subgradient steps of xi'
//           (C12) and zeta' (C13-hat) they give
//   power   per (n, m): closed-form KKT power of the l slots of RRH m on n
//           (eq. 653 / 683, log-power variable, Jacobi) and the RRH total
//   link    per (n, m): interference, SINR and victim prices of the l slots,
//           the streaming-rate contributions, and the step of the SIC
//           multipliers of (n, m) (C14 in divided form)
// The SIC multipliers are unevaluated float pairs (hi + lo): about 48
// significant bits through the accumulated steps, with no FP64 arithmetic in
// the stages.  Every sum runs in a fixed order, so results are reproducible.
#pragma once
#include "hcran_dev_dual.cuh"

namespace hcran {

struct RView {
  int Nc, Rs, Mi, NW;
  float *slab;                                      // [Nc][M][Rs], own-RRH entries zeroed
  int *k;                                           // [Nc][Up] user per slot, -1 = empty
  float *p, *pi, *g, *gi, *wa, *al, *wb, *pl, *X;   // [Nc][Up]
  float *Pt, *pio, *Sp, *Sm;                        // [Nc][M]
  float *zh0, *zl0, *zh1, *zl1;                     // [Nc][M*npair], two generations
  unsigned *nz;                                     // [Nc][NW] nonzero SIC multipliers
  float *sr, *sa;                                   // [Nc][Ks] streaming rate / alpha contributions
};

struct RScratch {
  float *xch0, *xch1;  // the CTA's residual vector, by iteration parity
  float *xih, *xil;    // xi' as (hi, lo) float pairs
  float *lzh, *lzl;    // log2 zeta' as (hi, lo) float pairs
  float *pmf, *xsp, *psi;  // pmax_m, 1 / (ln2 mask_m pmax_m), Psi_k
};

__device__ __forceinline__ RScratch res_scratch(const KDims &kd) {
  float *b = hcran_dyn + al4(kd.KSmax > 0 ? kd.KSmax : 1);
  const int xf = res_xch_floats(kd);
  RScratch s;
  s.xch0 = b;
  s.xch1 = b + xf;
  b += 2 * xf;
  const int m4 = (int)al4(kd.Mmax), s4 = (int)al4(kd.KSmax > 0 ? kd.KSmax : 1);
  s.xih = b;
  s.xil = b + m4;
  b += 2 * m4;
  s.lzh = b;
  s.lzl = b + s4;
  b += 2 * s4;
  s.pmf = b;
  b += m4;
  s.xsp = b;
  b += m4;
  s.psi = b;
  return s;
}

// geometry of the resident region: offset in the dynamic shared memory and
// the sizes the array offsets follow from
struct RGeom {
  int base, Nc, Rs, Mi, NW;
};
__device__ __forceinline__ RGeom res_geom(const Ctx &c, const KDims &kd) {
  RGeom g;
  g.base = (int)dyn_head_floats(kd);
  g.Nc = c.n1 - c.n0;
  g.Rs = res_row_stride(c.M, c.l);
  g.Mi = c.M * c.npair;
  g.NW = (g.Mi + 31) / 32;
  return g;
}

// The views are rebuilt inside every (inlined) stage from the geometry, so a
// stage keeps only the pointers it uses and they stay shared-memory pointers.
// Offsets are 32-bit (the region is at most 216 KB).
__device__ __forceinline__ RView res_view(const Ctx &c, const RGeom &gm) {
  RView r;
  float *b = hcran_dyn + gm.base;
  const int M = c.M, Up = c.Up, Nc = gm.Nc;
  r.Nc = Nc;
  r.Rs = gm.Rs;
  r.Mi = gm.Mi;
  r.NW = gm.NW;
  r.slab = b; b += Nc * M * r.Rs;
  const int su = Nc * Up;
  r.k = reinterpret_cast<int *>(b); b += su;
  r.p = b; b += su;
  r.pi = b; b += su;
  r.g = b; b += su;
  r.gi = b; b += su;
  r.wa = b; b += su;
  r.al = b; b += su;
  r.wb = b; b += su;
  r.pl = b; b += su;
  r.X = b; b += su;
  const int sm = (Nc * M + 3) & ~3, si = (Nc * r.Mi + 3) & ~3, sw = (Nc * r.NW + 3) & ~3,
            ss = (Nc * c.Ks + 3) & ~3;
  r.Pt = b; b += sm;
  r.pio = b; b += sm;
  r.Sp = b; b += sm;
  r.Sm = b; b += sm;
  r.zh0 = b; b += si;
  r.zl0 = b; b += si;
  r.zh1 = b; b += si;
  r.zl1 = b; b += si;
  r.nz = reinterpret_cast<unsigned *>(b); b += sw;
  r.sr = b; b += ss;
  r.sa = b;
  return r;
}

// hi + lo += s: exact two-sum, then renormalisation (round-to-nearest adds only)
__device__ __forceinline__ void ff_add(float &hi, float &lo, float s) {
  const float t = __fadd_rn(hi, s);
  const float bb = __fsub_rn(t, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bb)), __fsub_rn(s, bb));
  const float l2 = __fadd_rn(lo, err);
  const float h2 = __fadd_rn(t, l2);
  lo = __fsub_rn(l2, __fsub_rn(h2, t));
  hi = h2;
}

// global -> shared at the start of a dual loop (subcarriers n0 .. n0+Nc-1)
__device__ __forceinline__ void load_res(const Ctx &c, const RGeom &gm, int n0) {
  const RView r = res_view(c, gm);
  const int M = c.M, Up = c.Up, Rs = r.Rs, Nc = r.Nc;
  const int q = Up / 4, rows = Nc * M;
  const float4 *src = reinterpret_cast<const float4 *>(c.slab + (size_t)n0 * M * Up);
  for (int i = threadIdx.x; i < rows * q; i += kThreads) {
    const int row = i / q, col = i - row * q;
    *reinterpret_cast<float4 *>(r.slab + row * Rs + 4 * col) = src[i];
  }
  for (int e = threadIdx.x; e < Nc * Up; e += kThreads) {
    const size_t gI = (size_t)n0 * Up + e;
    const int k = c.S[gI];
    const float w = c.wslot[gI], a = c.alpha[gI];
    r.k[e] = k;
    r.p[e] = k >= 0 ? c.p[gI] : 0.f;
    r.pi[e] = 0.f;
    r.g[e] = c.gown[gI];
    r.gi[e] = k >= 0 ? c.ginv[gI] : 0.f;
    r.wa[e] = w * a;
    r.al[e] = a;
    r.wb[e] = w * c.beta[gI];
    r.pl[e] = c.plin[gI];
    r.X[e] = 0.f;
  }
  for (int e = threadIdx.x; e < Nc * r.Mi; e += kThreads) {
    const int t = e / r.Mi, i = e - t * r.Mi;
    const double z = c.zsic[(size_t)(n0 + t) * c.NPp + i];
    const float hi = (float)z;
    r.zh0[e] = hi;
    r.zl0[e] = (float)(z - (double)hi);
  }
}

// shared -> global at the end: powers and the committed SIC multipliers
__device__ __forceinline__ void store_res(const Ctx &c, const RGeom &gm, int n0, int zc) {
  const RView r = res_view(c, gm);
  const int Up = c.Up, Mi = r.Mi;
  const float *zh = zc ? r.zh1 : r.zh0, *zl = zc ? r.zl1 : r.zl0;
  for (int e = threadIdx.x; e < r.Nc * Up; e += kThreads)
    if (r.k[e] >= 0) c.p[(size_t)n0 * Up + e] = r.p[e];
  for (int e = threadIdx.x; e < r.Nc * Mi; e += kThreads) {
    const int t = e / Mi, i = e - t * Mi;
    c.zsic[(size_t)(n0 + t) * c.NPp + i] = (double)zh[e] + (double)zl[e];
  }
}

// The (n, m) groups of a stage are visited as h = tid, tid + kThreads, ...;
// t = h / M and m = h % M advance by a fixed step, so no stage divides.
struct GIt {
  int t0, m0, dt, dm;
};
__device__ __forceinline__ GIt group_iter(int M) {
  GIt g;
  g.t0 = (int)threadIdx.x / M;
  g.m0 = (int)threadIdx.x - g.t0 * M;
  g.dt = kThreads / M;
  g.dm = kThreads - g.dt * M;
  return g;
}
__device__ __forceinline__ void group_next(const GIt &g, int M, int &t, int &m) {
  t += g.dt;
  m += g.dm;
  if (m >= M) {
    m -= M;
    t++;
  }
}

// per (n, m): clear the nonzero masks and the streaming contributions of n
__device__ __forceinline__ void clear_sub(const Ctx &c, const RView &r, int t, int m) {
  for (int w = m; w < r.NW; w += c.M) r.nz[t * r.NW + w] = 0u;
  for (int ks = m; ks < c.Ks; ks += c.M) {
    r.sr[t * c.Ks + ks] = 0.f;
    r.sa[t * c.Ks + ks] = 0.f;
  }
}

// entry: RRH totals at p^0
__device__ __forceinline__ void stage_totals(const Ctx &c, const RGeom &gm, const GIt &gi) {
  const RView r = res_view(c, gm);
  const int M = c.M, l = c.l, Up = c.Up;
  int t = gi.t0, m = gi.m0;
  for (int h = threadIdx.x; h < r.Nc * M; h += kThreads, group_next(gi, M, t, m)) {
    const int base = t * Up + m * l;
    float tot = 0.f;
    for (int s = 0; s < l; s++) tot += r.p[base + s];
    r.Pt[h] = tot;
    clear_sub(c, r, t, m);
  }
}

// Projected subgradient steps from the residual sums of the last point:
//   xi'_m        += delta (sum_n P_{m,n} - pmax_m) / (ln2 mask_m pmax_m), then [.]+
//   log2 zeta'_k += delta clip((Psi_k - r_k) / max(sum_n alpha, 0.05), -1, 1), clipped
// (C12 and C13-hat; the zeta' step is multiplicative, a sum in log2 scale),
// accumulated in (hi, lo) float pairs.  The new xi'_m goes to sh.xif, the
// new zeta'_k to szeta.
__device__ __forceinline__ void xi_update(const RScratch &x, Shared &sh, int m, float tot, float delta) {
  const float step = delta * (tot - x.pmf[m]) * x.xsp[m];
  float hi = x.xih[m], lo = x.xil[m];
  if (hi != 0.f || step > 0.f) {  // stays exactly 0 while the constraint is slack
    ff_add(hi, lo, step);
    if (!(hi > 0.f)) {
      hi = 0.f;
      lo = 0.f;
    }
    x.xih[m] = hi;
    x.xil[m] = lo;
  }
  sh.xif[m] = hi;
}
__device__ __forceinline__ void zeta_update(const RScratch &x, float *szeta, int ks, float rr, float as,
                                            float delta) {
  const float e = delta * fminf(fmaxf((x.psi[ks] - rr) / fmaxf(as, (float)kZetaAsumMin), -1.f), 1.f);
  float hi = x.lzh[ks], lo = x.lzl[ks];
  ff_add(hi, lo, e);
  if (hi < kLog2ZetaMin) {
    hi = kLog2ZetaMin;
    lo = 0.f;
  } else if (hi > kLog2ZetaMax) {
    hi = kLog2ZetaMax;
    lo = 0.f;
  }
  x.lzh[ks] = hi;
  x.lzl[ks] = lo;
  szeta[ks] = exp2f(hi) * (1.f + lo * LN2F);
}

// KKT power of one slot (eq. 653 / 683): den = q eta_m + xi'_m +
// prices paid towards other RRHs' users + weaker users of (m, n) + SIC+;
// num = c w alpha / ln2 + SIC- p_lin with c = 1 (elastic) or zeta'_k;
// p = clip(num / den, p_floor, mask)
struct PowerCtx {
  float PIO, SP, SM, qe, xf, mk, fl, im;
  int Ke;
};
__device__ __forceinline__ float kkt_power(const PowerCtx &q, const float *szeta, int k, float own, float wa,
                                           float pl) {
  const float den = q.qe + q.xf + (q.PIO + own + q.SP);
  const float cw = k < q.Ke ? 1.f : szeta[k - q.Ke];
  const float num = cw * (wa * kInvLn2) + q.SM * pl;
  const float pv = (den <= 0.f || num >= den * q.mk) ? q.mk : num * fast_rcp(den);
  return fmaxf(pv, q.fl);
}

// KKT power of the L slots of one group, all values in registers (L <= 4 at
// compile time); writes the new powers, returns the group total
template <int L>
__device__ __forceinline__ float power_group(const RView &r, const PowerCtx &q, const float *szeta, int base,
                                             float &dmax) {
  int k[L];
  float pi[L], g[L], p[L], wa[L], pl[L];
#pragma unroll
  for (int s = 0; s < L; s++) {
    const int e = base + s;
    k[s] = r.k[e];
    pi[s] = r.pi[e];
    g[s] = r.g[e];
    p[s] = r.p[e];
    wa[s] = r.wa[e];
    pl[s] = r.pl[e];
  }
  float own[L];  // weaker users of the same (m, n) that hear slot s
  own[L - 1] = 0.f;
#pragma unroll
  for (int s = L - 2; s >= 0; s--) own[s] = own[s + 1] + pi[s + 1] * g[s + 1];
  float tot = 0.f;
#pragma unroll
  for (int s = L - 1; s >= 0; s--) {
    if (k[s] < 0) continue;
    const float pv = kkt_power(q, szeta, k[s], own[s], wa[s], pl[s]);
    dmax = fmaxf(dmax, fabsf(pv - p[s]) * q.im);
    r.p[base + s] = pv;
    tot += pv;
  }
  return tot;
}

__device__ __forceinline__ void power_ctx(PowerCtx &q, const Shared &sh, const RView &r, int h, int m) {
  q.PIO = r.pio[h];
  q.SP = r.Sp[h];
  q.SM = r.Sm[h];
  q.qe = sh.qeta[m];
  q.xf = sh.xif[m];
  q.mk = sh.maskf[m];
  q.fl = sh.floorf[m];
  q.im = sh.invmask[m];
}

template <int L>
__device__ __forceinline__ float power_stage_l(const Ctx &c, const Shared &sh, const RView &r, const float *szeta,
                                               const GIt &gi) {
  const int M = c.M, Up = c.Up, G = r.Nc * M;
  PowerCtx q;
  q.Ke = c.Ke;
  float dmax = 0.f;
  int t = gi.t0, m = gi.m0;
  for (int h = threadIdx.x; h < G; h += kThreads, group_next(gi, M, t, m)) {
    power_ctx(q, sh, r, h, m);
    r.Pt[h] = power_group<L>(r, q, szeta, t * Up + m * L, dmax);
    clear_sub(c, r, t, m);
  }
  return dmax;
}

// power stage: KKT power of the l slots of (n, m) from the sums of the last
// link / sums stages and the current multipliers; RRH total at the new point.
// L = l (1 .. 4) or 0 for any l.  Returns the thread's max |p_new - p| / mask.
template <int L>
__device__ __forceinline__ float stage_power(const Ctx &c, const Shared &sh, const RGeom &gm, const float *szeta,
                                             const GIt &gi) {
  const RView r = res_view(c, gm);
  if (L > 0) return power_stage_l<(L > 0 ? L : 1)>(c, sh, r, szeta, gi);
  const int M = c.M, l = c.l, Up = c.Up, G = r.Nc * M;
  PowerCtx q;
  q.Ke = c.Ke;
  float dmax = 0.f;
  int t = gi.t0, m = gi.m0;
  for (int h = threadIdx.x; h < G; h += kThreads, group_next(gi, M, t, m)) {
    const int base = t * Up + m * l;
    power_ctx(q, sh, r, h, m);
    float tot = 0.f, own = 0.f;
    for (int s = l - 1; s >= 0; s--) {
      const int e = base + s;
      const int k = r.k[e];
      const float pis = r.pi[e], gs = r.g[e];
      if (k >= 0) {
        const float pv = kkt_power(q, szeta, k, own, r.wa[e], r.pl[e]);
        dmax = fmaxf(dmax, fabsf(pv - r.p[e]) * q.im);
        r.p[e] = pv;
        tot += pv;
      }
      own += pis * gs;
    }
    r.Pt[h] = tot;
    clear_sub(c, r, t, m);
  }
  return dmax;
}

// SINR, price and streaming contribution of one slot at interference X
__device__ __forceinline__ float slot_price(const RView &r, const float *szeta, int t, int Ks, int Ke, float sigma,
                                            int e, int k, float ps, float g, float wa, float intra, float X) {
  const float inv = fast_rcp(sigma + g * intra + X);
  if (k < Ke) return wa * kInvLn2 * inv;
  const int ks = k - Ke;  // a streaming user appears at most once per subcarrier
  const float gam = ps * g * inv;
  // hardware log2 (at most 2^-22 absolute error on [0.5, 2], 2 ulp elsewhere):
  // the streaming-rate term enters only the zeta' step
  r.sr[t * Ks + ks] = wa * __log2f(fmaxf(gam, kGammaFloor)) + r.wb[e];
  r.sa[t * Ks + ks] = r.al[e];
  return szeta[ks] * wa * kInvLn2 * inv;
}

// SIC step of one pair (a stronger than b) of (n, m); returns whether the
// multiplier is nonzero afterwards
__device__ __forceinline__ bool sic_step(float sigma, float scale, float delta, float Xa, float gia, float Xb,
                                         float gib, float &hi, float &lo) {
  const float ra = (sigma + Xa) * gia;
  const float rb = (sigma + Xb) * gib;
  const float step = delta * (ra - rb) * fast_rcp(rb) * scale;
  if (hi != 0.f || step > 0.f) {  // stays exactly 0 while the constraint is slack
    ff_add(hi, lo, step);
    if (!(hi > 0.f)) {
      hi = 0.f;
      lo = 0.f;
    }
  }
  return hi != 0.f;
}

// set bits i0 + pr of subcarrier t's nonzero-multiplier mask (at most 28 bits,
// possibly straddling two words)
__device__ __forceinline__ void mark_nonzero(const RView &r, int t, int i0, unsigned bits) {
  if (!bits) return;
  const unsigned long long wide = (unsigned long long)bits << (i0 & 31);
  unsigned *wd = r.nz + t * r.NW + (i0 >> 5);
  if ((unsigned)wide) atomicOr(wd, (unsigned)wide);
  if ((unsigned)(wide >> 32)) atomicOr(wd + 1, (unsigned)(wide >> 32));
}

// link of one group with L <= 4 slots, every slot value in registers
template <int L>
__device__ __forceinline__ void link_group(const RView &r, const float *szeta, int t, int m, int M, int Rs,
                                           int base, int Ks, int Ke, float sigma, float scale, float delta,
                                           const float *zh, const float *zl, float *nh, float *nl) {
  constexpr int NP = L * (L - 1) / 2;
  int k[L];
  float p[L], g[L], gi[L], wa[L];
#pragma unroll
  for (int s = 0; s < L; s++) {
    const int e = base + s;
    k[s] = r.k[e];
    p[s] = r.p[e];
    g[s] = r.g[e];
    gi[s] = r.gi[e];
    wa[s] = r.wa[e];
  }
  float zhv[NP > 0 ? NP : 1], zlv[NP > 0 ? NP : 1];
#pragma unroll
  for (int pr = 0; pr < NP; pr++) {
    zhv[pr] = zh[pr];
    zlv[pr] = zl[pr];
  }
  // interference of the L slots in one pass over the slab rows (own entry is
  // zero), two partial sums per slot
  const float *Pt = r.Pt + t * M;
  const float *SL = r.slab + (t * M * Rs + m * L);
  float xa[L], xb[L];
#pragma unroll
  for (int s = 0; s < L; s++) xa[s] = xb[s] = 0.f;
  int j = 0;
  for (; j + 1 < M; j += 2) {
    const float pa = Pt[j], pb = Pt[j + 1];
    const float *ra = SL + j * Rs, *rb = ra + Rs;
#pragma unroll
    for (int s = 0; s < L; s++) {
      xa[s] += ra[s] * pa;
      xb[s] += rb[s] * pb;
    }
  }
  if (j < M) {
    const float pa = Pt[j];
    const float *ra = SL + j * Rs;
#pragma unroll
    for (int s = 0; s < L; s++) xa[s] += ra[s] * pa;
  }
  float X[L];
#pragma unroll
  for (int s = 0; s < L; s++) X[s] = xa[s] + xb[s];
  float intra = 0.f;
#pragma unroll
  for (int s = 0; s < L; s++) {
    const int e = base + s;
    const float pi = k[s] >= 0 ? slot_price(r, szeta, t, Ks, Ke, sigma, e, k[s], p[s], g[s], wa[s], intra, X[s])
                               : 0.f;
    r.pi[e] = pi;
    intra += p[s];  // empty slots hold p = 0
  }
  unsigned bits = 0u;
  int pr = 0;
#pragma unroll
  for (int a = 0; a < L; a++)
#pragma unroll
    for (int b = a + 1; b < L; b++, pr++) {
      float hi = zhv[pr], lo = zlv[pr];
      if (k[a] >= 0 && k[b] >= 0 && sic_step(sigma, scale, delta, X[a], gi[a], X[b], gi[b], hi, lo))
        bits |= 1u << pr;
      nh[pr] = hi;
      nl[pr] = lo;
    }
  mark_nonzero(r, t, m * NP, bits);
}

template <int L>
__device__ __forceinline__ void link_stage_l(const Ctx &c, const Shared &sh, const RView &r, const float *szeta,
                                             float delta, int zc, const GIt &gi) {
  const int M = c.M, Up = c.Up, Rs = r.Rs, Ks = c.Ks, Ke = c.Ke, G = r.Nc * M;
  constexpr int NP = L * (L - 1) / 2;
  const float sigma = c.sigma;
  const float *zh0 = zc ? r.zh1 : r.zh0, *zl0 = zc ? r.zl1 : r.zl0;
  float *nh0 = zc ? r.zh0 : r.zh1, *nl0 = zc ? r.zl0 : r.zl1;
  int t = gi.t0, m = gi.m0;
  for (int h = threadIdx.x; h < G; h += kThreads, group_next(gi, M, t, m)) {
    const int o = t * r.Mi + m * NP;
    link_group<L>(r, szeta, t, m, M, Rs, t * Up + m * L, Ks, Ke, sigma, sh.sicscale[m], delta, zh0 + o, zl0 + o,
                  nh0 + o, nl0 + o);
  }
}

// link stage at the point in r.p (Sec. II-A SINR with the SIC order), then the
// SIC step of (n, m): generation zc -> zc ^ 1 with step delta.  L = l (1 .. 4)
// or 0 for any l.
template <int L>
__device__ __forceinline__ void stage_link(const Ctx &c, const Shared &sh, const RGeom &gm, const float *szeta,
                                           float delta, int zc, const GIt &gi) {
  const RView r = res_view(c, gm);
  if (L > 0) {
    link_stage_l<(L > 0 ? L : 1)>(c, sh, r, szeta, delta, zc, gi);
    return;
  }
  const int M = c.M, l = c.l, Up = c.Up, Rs = r.Rs, np = c.npair, Ks = c.Ks, Ke = c.Ke, G = r.Nc * M;
  const float sigma = c.sigma;
  const float *zh0 = zc ? r.zh1 : r.zh0, *zl0 = zc ? r.zl1 : r.zl0;
  float *nh0 = zc ? r.zh0 : r.zh1, *nl0 = zc ? r.zl0 : r.zl1;
  int t = gi.t0, m = gi.m0;
  for (int h = threadIdx.x; h < G; h += kThreads, group_next(gi, M, t, m)) {
    const int base = t * Up + m * l;
    const float *Pt = r.Pt + t * M;
    const float *SL = r.slab + (t * M * Rs + m * l);
    const int o = t * r.Mi + m * np;
    const float *zh = zh0 + o, *zl = zl0 + o;
    float *nh = nh0 + o, *nl = nl0 + o;
    const float scale = sh.sicscale[m];
    float intra = 0.f;
    for (int s = 0; s < l; s++) {
      const int e = base + s;
      const int k = r.k[e];
      const float ps = r.p[e];
      float X = 0.f, pi = 0.f;
      for (int j = 0; j < M; j++) X += SL[j * Rs + s] * Pt[j];
      if (k >= 0) pi = slot_price(r, szeta, t, Ks, Ke, sigma, e, k, ps, r.g[e], r.wa[e], intra, X);
      r.pi[e] = pi;
      r.X[e] = X;
      intra += ps;
    }
    unsigned bits = 0u;
    int pr = 0;
    for (int a = 0; a < l; a++)
      for (int b = a + 1; b < l; b++, pr++) {
        const int ea = base + a, eb = base + b;
        float hi = zh[pr], lo = zl[pr];
        if (r.k[ea] >= 0 && r.k[eb] >= 0 &&
            sic_step(sigma, scale, delta, r.X[ea], r.gi[ea], r.X[eb], r.gi[eb], hi, lo))
          bits |= 1u << pr;
        nh[pr] = hi;
        nl[pr] = lo;
      }
    mark_nonzero(r, t, m * np, bits);
  }
}

// rows stage per (n, j): pio = row j of the slab . pi, and the SIC+ / SIC-
// sums of row j over the nonzero multipliers of n (generation zn)
__device__ __forceinline__ void stage_rows(const Ctx &c, const Shared &sh, const RGeom &gm, int zn, const GIt &gi) {
  const RView r = res_view(c, gm);
  const int M = c.M, Up = c.Up, Rs = r.Rs, q4 = Up / 4;
  int t = gi.t0, j = gi.m0;
  for (int h = threadIdx.x; h < r.Nc * M; h += kThreads, group_next(gi, M, t, j)) {
    const float *row = r.slab + h * Rs;
    const float4 *r4 = reinterpret_cast<const float4 *>(row);
    const float4 *p4 = reinterpret_cast<const float4 *>(r.pi + t * Up);
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    for (int i = 0; i < q4; i++) {
      const float4 x = r4[i], y = p4[i];
      a0 += x.x * y.x;
      a1 += x.y * y.y;
      a2 += x.z * y.z;
      a3 += x.w * y.w;
    }
    float sp = 0.f, sm = 0.f;
    const float *zh = (zn ? r.zh1 : r.zh0) + t * r.Mi;
    const float *ginv = r.gi + t * Up;
    for (int w = 0; w < r.NW; w++) {
      unsigned bits = r.nz[t * r.NW + w];
      while (bits) {  // two nonzero multipliers per pass, in bit order
        const int i1 = w * 32 + __ffs(bits) - 1;
        bits &= bits - 1u;
        const bool two = bits != 0u;
        const int i2 = two ? w * 32 + __ffs(bits) - 1 : i1;
        if (two) bits &= bits - 1u;
        const int ua1 = sh.item_a[i1], ub1 = sh.item_b[i1], ua2 = sh.item_a[i2], ub2 = sh.item_b[i2];
        const float z1 = zh[i1], z2 = zh[i2];
        const float t1 = row[ua1] * (z1 * ginv[ua1]) - row[ub1] * (z1 * ginv[ub1]);
        const float t2 = row[ua2] * (z2 * ginv[ua2]) - row[ub2] * (z2 * ginv[ub2]);
        if (t1 > 0.f) sp += t1;
        else sm -= t1;
        if (two) {
          if (t2 > 0.f) sp += t2;
          else sm -= t2;
        }
      }
    }
    r.pio[h] = (a0 + a1) + (a2 + a3);
    r.Sp[h] = sp;
    r.Sm[h] = sm;
  }
}

// this CTA's residual sums over its subcarriers into xv: RRH totals [M],
// streaming rates [Ks], streaming alphas [Ks].  Teams of 8 lanes, one sum per
// team, lanes over the subcarriers and a 3-step shuffle tree (fixed order).
// Warps take the sums from the last warp down (the sums stage hands its (n, j)
// rows out from the first thread up): the last res_warps(nq) warps hold work.
__device__ __forceinline__ int res_warps(int nq) { return nq >= 4 * kWarps ? kWarps : (nq + 3) / 4; }
__device__ __forceinline__ void res_partials(const Ctx &c, const RGeom &gm, float *xv) {
  const RView r = res_view(c, gm);
  const int warp = kWarps - 1 - (int)(threadIdx.x >> 5), lane = threadIdx.x & 31, sub = lane & 7;
  const int M = c.M, Ks = c.Ks, nq = M + 2 * Ks, Nc = r.Nc;
  for (int q0 = warp * 4; q0 < nq; q0 += kThreads / 8) {  // warp-uniform trip count
    const int q = q0 + (lane >> 3);
    float a = 0.f;
    if (q < nq) {
      const float *src;
      int stride;
      if (q < M) {
        src = r.Pt + q;
        stride = M;
      } else if (q < M + Ks) {
        src = r.sr + (q - M);
        stride = Ks;
      } else {
        src = r.sa + (q - M - Ks);
        stride = Ks;
      }
      float a0 = 0.f, a1 = 0.f;
      int t = sub;
      for (; t + 8 < Nc; t += 16) {
        a0 += src[t * stride];
        a1 += src[(t + 8) * stride];
      }
      if (t < Nc) a0 += src[t * stride];
      a = a0 + a1;
    }
    a += __shfl_xor_sync(0xffffffffu, a, 4);
    a += __shfl_xor_sync(0xffffffffu, a, 2);
    a += __shfl_xor_sync(0xffffffffu, a, 1);
    if (sub == 0 && q < nq) xv[q] = a;
  }
}

// One dual loop of Algorithm 1 (one SCALE pass) on resident state.  Same
// iteration as dual_loop: link at p^0 (SIC step delta_0 = 1); then per
// iteration the stop test on max |p^v - p^{v-1}| / mask, the residual sums at
// p^v with the steps of xi' and zeta' they give (beside the price and SIC
// sums), the KKT power p^{v+1} and the link stage at p^{v+1}.  Returns the
// iterations run.  Instantiated per l (L = 1 .. 4, 0 for any other l) and per
// CL (a cluster of more than one CTA or not): the loop is bound by the latency
// of short stages, and the code of one instantiation stays compact in the
// instruction caches.
template <int L, bool CL>
__device__ __forceinline__ int dual_loop_res_l(const Ctx &c, Shared &sh, float *dyn, const KDims &kd, float *szeta,
                                               const Tol &tol, long long *cyc, unsigned &phase, unsigned &pending) {
  const int Vmax = tol.max_dual > 0 ? tol.max_dual : 1;
  const int M = c.M, Ks = c.Ks, nq = M + 2 * Ks;
  const RGeom r = res_geom(c, kd);
  const RScratch x = res_scratch(kd);
  const long long t0 = clock64();
  const GIt gi = group_iter(M);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // the residual sums run on the last P warps; their thread u (counted from
  // the first of them) takes the step of xi'_u (u < M) or zeta'_{u-M}
  const int P = res_warps(nq);
  const int u = (int)threadIdx.x - (kWarps - P) * 32;
  load_res(c, r, c.n0);
  for (int m = threadIdx.x; m < M; m += kThreads) {
    const float hi = (float)c.xi[m];
    x.xih[m] = hi;
    x.xil[m] = (float)(c.xi[m] - (double)hi);
    x.pmf[m] = (float)c.pmax[m];
    x.xsp[m] = (float)(1.0 / (LN2D * c.mask[m] * c.pmax[m]));
  }
  for (int k = threadIdx.x; k < Ks; k += kThreads) {
    const double lz = log2(c.zeta[k]);
    const float hi = (float)lz;
    x.lzh[k] = hi;
    x.lzl[k] = (float)(lz - (double)hi);
    x.psi[k] = sh_psi(c, k);
  }
  if (threadIdx.x < kWarps) sh.redf[threadIdx.x] = 0.f;
  __syncthreads();
  stage_totals(c, r, gi);
  __syncthreads();
  int zc = 0;  // generation of the committed SIC multipliers
  stage_link<L>(c, sh, r, szeta, 1.f, zc, gi);
  __syncthreads();
  if (threadIdx.x == 0) cyc[1] += clock64() - t0;
  int v = 0;
  for (;;) {
    const long long t1 = clock64();
    // max |p^v - p^{v-1}| / mask over this CTA, from the warps' maxima of the
    // last power stage (0 before the first)
    const float dloc = warp_max(lane < kWarps ? sh.redf[lane] : 0.f);
    const float delta = rsqrtf((float)v + 1.f);
    if (!CL) {
      if ((v > 0 && dloc < (float)tol.tol_dual) || v >= Vmax) break;
      if (u >= 0) {  // residual sums, then the multiplier steps they give
        res_partials(c, r, x.xch0);
        asm volatile("bar.sync 1, %0;" ::"r"(P * 32) : "memory");
        if (u < M) xi_update(x, sh, u, x.xch0[u], delta);
        else if (u < M + Ks) zeta_update(x, szeta, u - M, x.xch0[u], x.xch0[u + Ks], delta);
        for (int ks = u - M + P * 32; ks < Ks; ks += P * 32)
          zeta_update(x, szeta, ks, x.xch0[M + ks], x.xch0[M + Ks + ks], delta);
      }
      stage_rows(c, sh, r, zc ^ 1, gi);
      __syncthreads();
    } else {
      // the per-CTA residual vectors (and maxima) are exchanged through a
      // split cluster barrier around the price and SIC sums, which do not
      // depend on them; peers read this parity's vector before their next
      // arrival, and it is rewritten two iterations later, after the next wait
      float *xv = (v & 1) ? x.xch1 : x.xch0;
      const int C = c.csize;
      if (u >= 0) res_partials(c, r, xv);
      if (threadIdx.x == kThreads - 1) xv[nq] = dloc;
      __syncwarp();
      cluster_arrive();  // release: this thread's part of the vector is written
      stage_rows(c, sh, r, zc ^ 1, gi);
      cluster_wait();
      // one round of peer loads: the maxima for the stop test and, on the
      // threads that take a step, the values it sums, all issued before the
      // first is used (totals in rank order)
      const int i0 = threadIdx.x;
      const bool upd = i0 < M + Ks, z0 = i0 >= M;
      float dv[8], a[8], b[8];
#pragma unroll
      for (int q = 0; q < 8; q++) {
        const float *pv = q < C ? peer(xv, q) : xv;
        dv[q] = q < C ? pv[nq] : 0.f;
        a[q] = q < C && upd ? pv[i0] : 0.f;
        b[q] = q < C && upd && z0 ? pv[i0 + Ks] : 0.f;
      }
      float d = dloc;
#pragma unroll
      for (int q = 0; q < 8; q++) d = fmaxf(d, dv[q]);
      const bool stop = (v > 0 && d < (float)tol.tol_dual) || v >= Vmax;
      if (!stop) {  // the steps
        for (int i = i0; i < M + Ks; i += kThreads) {
          const bool z = i >= M;
          if (i != i0) {  // only when M + Ks exceeds the block
#pragma unroll
            for (int q = 0; q < 8; q++) {
              const float *pv = q < C ? peer(xv, q) : xv;
              a[q] = q < C ? pv[i] : 0.f;
              b[q] = q < C && z ? pv[i + Ks] : 0.f;
            }
          }
          float t = a[0], t2 = b[0];
#pragma unroll
          for (int q = 1; q < 8; q++)
            if (q < C) {
              t += a[q];
              t2 += b[q];
            }
          if (!z) xi_update(x, sh, i, t, delta);
          else zeta_update(x, szeta, i - M, t, t2, delta);
        }
      }
      __syncthreads();
      if (stop) break;
    }
    const long long t2 = clock64();
    zc ^= 1;  // the multipliers of the last link stage become the committed ones
    float dl = stage_power<L>(c, sh, r, szeta, gi);
    dl = warp_max(dl);
    if (lane == 0) sh.redf[warp] = dl;
    __syncthreads();
    stage_link<L>(c, sh, r, szeta, rsqrtf((float)v + 2.f), zc, gi);
    __syncthreads();
    v++;
    const long long t3 = clock64();
    if (threadIdx.x == 0) {
      cyc[2] += t2 - t1;
      cyc[3] += t3 - t2;
    }
  }
  store_res(c, r, c.n0, zc);
  if (c.crank == 0) {
    for (int m = threadIdx.x; m < M; m += kThreads) c.xi[m] = (double)x.xih[m] + (double)x.xil[m];
    for (int k = threadIdx.x; k < Ks; k += kThreads) c.zeta[k] = exp2((double)x.lzh[k] + (double)x.lzl[k]);
  }
  // gamma, pi, X, totals and SIC sums at the final point for the later phases
  link_all<kLinkOnly>(c, sh, dyn, kd, szeta, 0.f, phase, pending);
  return v;
}

__device__ int dual_loop_res(const Ctx &c, Shared &sh, float *dyn, const KDims &kd, float *szeta, const Tol &tol,
                             long long *cyc, unsigned &phase, unsigned &pending) {
  if (c.csize > 1) {
    switch (c.l) {
      case 1: return dual_loop_res_l<1, true>(c, sh, dyn, kd, szeta, tol, cyc, phase, pending);
      case 2: return dual_loop_res_l<2, true>(c, sh, dyn, kd, szeta, tol, cyc, phase, pending);
      case 3: return dual_loop_res_l<3, true>(c, sh, dyn, kd, szeta, tol, cyc, phase, pending);
      case 4: return dual_loop_res_l<4, true>(c, sh, dyn, kd, szeta, tol, cyc, phase, pending);
      default: return dual_loop_res_l<0, true>(c, sh, dyn, kd, szeta, tol, cyc, phase, pending);
    }
  }
  switch (c.l) {
    case 1: return dual_loop_res_l<1, false>(c, sh, dyn, kd, szeta, tol, cyc, phase, pending);
    case 2: return dual_loop_res_l<2, false>(c, sh, dyn, kd, szeta, tol, cyc, phase, pending);
    case 3: return dual_loop_res_l<3, false>(c, sh, dyn, kd, szeta, tol, cyc, phase, pending);
    case 4: return dual_loop_res_l<4, false>(c, sh, dyn, kd, szeta, tol, cyc, phase, pending);
    default: return dual_loop_res_l<0, false>(c, sh, dyn, kd, szeta, tol, cyc, phase, pending);
  }
}

}  // namespace hcran
