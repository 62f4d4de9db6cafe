// hcran_dev_resident.cuh -- the dual loop of Algorithm 1 on shared-memory
// resident state (internal).
//
// At the start of a dual loop the CTA copies, for its subcarriers, the compact
// slab, the slot arrays and the SIC multipliers into shared memory (structure
// of arrays, sized by res_floats); every dual iteration then works on shared
// memory only, and the powers, the committed multipliers and xi', zeta' go
// back to global memory at the end.
//
// One iteration is four block-wide stages, each over a flat index space so
// that every thread has work and long independent loops:
//   power   per (n, m): closed-form KKT power of the l slots of RRH m on n
//           (eq. 653 / 683, log-power variable, Jacobi) and the RRH total
//   link    per (n, m): interference, SINR and victim prices of the l slots,
//           the streaming-rate contributions, and the step of the SIC
//           multipliers of (n, m) (C14 in divided form)
//   rows    per (n, j): the prices a transmitter of RRH j pays towards the
//           other RRHs' users (row j of the slab against pi) and the SIC+ /
//           SIC- sums of row j over the nonzero SIC multipliers of n
//   update  per RRH and per streaming user: the residual sums over n and the
//           projected subgradient steps of xi' (C12) and zeta' (C13-hat)
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
  float *xch0, *xch1;  // per-CTA partial sums, by iteration parity
  float *xtot;         // their totals over the cluster
  double *xi, *zeta;
  float *pmf, *xscale, *psi;  // pmax_m, 1 / (ln2 mask_m), Psi_k
};

__device__ __forceinline__ RScratch res_scratch(float *dyn, const KDims &kd) {
  float *b = dyn + al4(kd.KSmax > 0 ? kd.KSmax : 1);
  const int xf = res_xch_floats(kd);
  RScratch s;
  s.xch0 = b;
  s.xch1 = b + xf;
  s.xtot = b + 2 * xf;
  b += 3 * xf;
  s.xi = reinterpret_cast<double *>(b);
  b += 2 * al4(kd.Mmax);
  s.zeta = reinterpret_cast<double *>(b);
  b += 2 * al4(kd.KSmax > 0 ? kd.KSmax : 1);
  s.pmf = b;
  b += al4(kd.Mmax);
  s.xscale = b;
  b += al4(kd.Mmax);
  s.psi = b;
  return s;
}

__device__ __forceinline__ RView res_view(float *b, const Ctx &c, int Nc) {
  RView r;
  const int M = c.M, Up = c.Up;
  r.Nc = Nc;
  r.Rs = res_row_stride(M, c.l);
  r.Mi = M * c.npair;
  r.NW = (r.Mi + 31) / 32;
  r.slab = b; b += (size_t)Nc * M * r.Rs;
  const size_t su = (size_t)Nc * Up;
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
  const size_t sm = al4((int64_t)Nc * M), si = al4((int64_t)Nc * r.Mi), sw = al4((int64_t)Nc * r.NW),
               ss = al4((int64_t)Nc * c.Ks);
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
__device__ __forceinline__ void load_res(const Ctx &c, const RView &r, int n0) {
  const int M = c.M, Up = c.Up, Rs = r.Rs, Nc = r.Nc;
  const int q = Up / 4, rows = Nc * M;
  const float4 *src = reinterpret_cast<const float4 *>(c.slab + (size_t)n0 * M * Up);
  for (int i = threadIdx.x; i < rows * q; i += kThreads) {
    const int row = i / q, col = i - row * q;
    *reinterpret_cast<float4 *>(r.slab + (size_t)row * Rs + 4 * col) = src[i];
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
__device__ __forceinline__ void store_res(const Ctx &c, const RView &r, int n0, int zc) {
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
__device__ __forceinline__ void stage_totals(const Ctx &c, const RView &r, const GIt &gi) {
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

// KKT power of one slot (eq. 653 / 683): den = [elastic] q eta_m + xi'_m +
// prices paid towards other RRHs' users + weaker users of (m, n) + SIC+;
// num = c w alpha / ln2 + SIC- p_lin; p = clip(num / den, p_floor, mask)
struct PowerCtx {
  float PIO, SP, SM, qe, xf, mk, fl, im;
  int Ke;
};
__device__ __forceinline__ float kkt_power(const PowerCtx &q, const float *szeta, int k, float own, float wa,
                                           float pl) {
  const float den = (k < q.Ke ? q.qe : 0.f) + q.xf + (q.PIO + own + q.SP);
  const float cw = k < q.Ke ? 1.f : szeta[k - q.Ke];
  const float num = cw * (wa * kInvLn2) + q.SM * pl;
  const float pv = (den <= 0.f || num >= den * q.mk) ? q.mk : num * fast_rcp(den);
  return fmaxf(pv, q.fl);
}

// power stage: KKT power of the l slots of (n, m) from the sums of the last
// link / rows stages and the current multipliers; RRH total at the new point.
// Returns the thread's max |p_new - p| / mask.
__device__ __forceinline__ float stage_power(const Ctx &c, const Shared &sh, const RView &r, const float *szeta,
                                             const GIt &gi) {
  const int M = c.M, l = c.l, Up = c.Up, G = r.Nc * M;
  PowerCtx q;
  q.Ke = c.Ke;
  float dmax = 0.f;
  int t = gi.t0, m = gi.m0;
  for (int h = threadIdx.x; h < G; h += kThreads, group_next(gi, M, t, m)) {
    const int base = t * Up + m * l;
    q.PIO = r.pio[h];
    q.SP = r.Sp[h];
    q.SM = r.Sm[h];
    q.qe = sh.qeta[m];
    q.xf = sh.xif[m];
    q.mk = sh.maskf[m];
    q.fl = sh.floorf[m];
    q.im = sh.invmask[m];
    float tot = 0.f;
    if (l <= 4) {
      int k[4];
      float pi[4], g[4], p[4], wa[4], pl[4];
#pragma unroll
      for (int s = 0; s < 4; s++)
        if (s < l) {
          const int e = base + s;
          k[s] = r.k[e];
          pi[s] = r.pi[e];
          g[s] = r.g[e];
          p[s] = r.p[e];
          wa[s] = r.wa[e];
          pl[s] = r.pl[e];
        }
      float own = 0.f;  // weaker users of the same (m, n) that hear slot s
#pragma unroll
      for (int s = 3; s >= 0; s--)
        if (s < l) {
          if (k[s] >= 0) {
            const float pv = kkt_power(q, szeta, k[s], own, wa[s], pl[s]);
            dmax = fmaxf(dmax, fabsf(pv - p[s]) * q.im);
            r.p[base + s] = pv;
            tot += pv;
          }
          own += pi[s] * g[s];
        }
    } else {
      float own = 0.f;
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
  r.sr[t * Ks + ks] = wa * log2f(fmaxf(gam, kGammaFloor)) + r.wb[e];
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

// link stage at the point in r.p (Sec. II-A SINR with the SIC order), then the
// SIC step of (n, m): generation zc -> zc ^ 1 with step delta
__device__ __forceinline__ void stage_link(const Ctx &c, const Shared &sh, const RView &r, const float *szeta,
                                           float delta, int zc, const GIt &gi) {
  const int M = c.M, l = c.l, Up = c.Up, Rs = r.Rs, np = c.npair, Ks = c.Ks, Ke = c.Ke, G = r.Nc * M;
  const float sigma = c.sigma;
  const float *zh0 = zc ? r.zh1 : r.zh0, *zl0 = zc ? r.zl1 : r.zl0;
  float *nh0 = zc ? r.zh0 : r.zh1, *nl0 = zc ? r.zl0 : r.zl1;
  int t = gi.t0, m = gi.m0;
  for (int h = threadIdx.x; h < G; h += kThreads, group_next(gi, M, t, m)) {
    const int base = t * Up + m * l;
    const float *Pt = r.Pt + t * M;
    const float *SL = r.slab + (size_t)t * M * Rs + m * l;
    const int o = t * r.Mi + m * np;
    const float *zh = zh0 + o, *zl = zl0 + o;
    float *nh = nh0 + o, *nl = nl0 + o;
    const float scale = sh.sicscale[m];
    unsigned bits = 0u;
    if (l <= 4) {
      // interference of the l slots in one pass over the slab rows (own entry is zero)
      float X[4] = {0.f, 0.f, 0.f, 0.f};
      for (int j = 0; j < M; j++) {
        const float pt = Pt[j];
        const float *row = SL + j * Rs;
#pragma unroll
        for (int s = 0; s < 4; s++)
          if (s < l) X[s] += row[s] * pt;
      }
      int k[4];
      float gi4[4];
      float intra = 0.f;
#pragma unroll
      for (int s = 0; s < 4; s++)
        if (s < l) {
          const int e = base + s;
          k[s] = r.k[e];
          gi4[s] = r.gi[e];
          const float ps = r.p[e];
          float pi = 0.f;
          if (k[s] >= 0) pi = slot_price(r, szeta, t, Ks, Ke, sigma, e, k[s], ps, r.g[e], r.wa[e], intra, X[s]);
          r.pi[e] = pi;
          intra += ps;  // empty slots hold p = 0
        }
      int pr = 0;
#pragma unroll
      for (int a = 0; a < 4; a++)
#pragma unroll
        for (int b = a + 1; b < 4; b++)
          if (b < l) {
            float hi = zh[pr], lo = zl[pr];
            if (k[a] >= 0 && k[b] >= 0 && sic_step(sigma, scale, delta, X[a], gi4[a], X[b], gi4[b], hi, lo))
              bits |= 1u << pr;
            nh[pr] = hi;
            nl[pr] = lo;
            pr++;
          }
    } else {
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
    }
    if (bits) {  // bits i0 + pr of subcarrier n's mask (np <= 28 bits, may straddle two words)
      const int i0 = m * np;
      const unsigned long long wide = (unsigned long long)bits << (i0 & 31);
      unsigned *wd = r.nz + t * r.NW + (i0 >> 5);
      if ((unsigned)wide) atomicOr(wd, (unsigned)wide);
      if ((unsigned)(wide >> 32)) atomicOr(wd + 1, (unsigned)(wide >> 32));
    }
  }
}

// rows stage per (n, j): pio = row j of the slab . pi, and the SIC+ / SIC-
// sums of row j over the nonzero multipliers of n (generation zn)
__device__ __forceinline__ void stage_rows(const Ctx &c, const Shared &sh, const RView &r, int zn, const GIt &gi) {
  const int M = c.M, Up = c.Up, Rs = r.Rs, q4 = Up / 4;
  int t = gi.t0, j = gi.m0;
  for (int h = threadIdx.x; h < r.Nc * M; h += kThreads, group_next(gi, M, t, j)) {
    const float *row = r.slab + (size_t)h * Rs;
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
      while (bits) {
        const int i = w * 32 + __ffs(bits) - 1;
        bits &= bits - 1u;
        const int ua = sh.item_a[i], ub = sh.item_b[i];
        const float z = zh[i];
        const float tt = row[ua] * (z * ginv[ua]) - row[ub] * (z * ginv[ub]);
        if (tt > 0.f) sp += tt;
        else sm -= tt;
      }
    }
    r.pio[h] = (a0 + a1) + (a2 + a3);
    r.Sp[h] = sp;
    r.Sm[h] = sm;
  }
}

// this CTA's residual sums over its subcarriers into xv: RRH totals [M],
// streaming rates [Ks], streaming alphas [Ks]; then the max |dp| / mask
__device__ __forceinline__ void res_partials(const Ctx &c, Shared &sh, const RView &r, float *xv, float dl) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int M = c.M, Ks = c.Ks;
  for (int q = warp; q < M + 2 * Ks; q += kWarps) {
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
    float a = 0.f;
    for (int t = lane; t < r.Nc; t += 32) a += src[t * stride];
    a = warp_sum(a);
    if (lane == 0) xv[q] = a;
  }
  dl = warp_max(dl);
  if (lane == 0) sh.redf[warp] = dl;
}

// One dual loop of Algorithm 1 (one SCALE pass) on resident state.  Same
// iteration as dual_loop: link at p^0 (SIC step delta_0 = 1); then per
// iteration the stop test on max |p^v - p^{v-1}| / mask, the projected
// subgradient step on xi' and zeta' from the residuals at p^v, the KKT power
// p^{v+1} and the link / rows stages at p^{v+1}.  Returns the iterations run.
__device__ int dual_loop_res(const Ctx &c, Shared &sh, float *dyn, const KDims &kd, float *szeta,
                             const Tol &tol, long long *cyc, unsigned &phase, unsigned &pending) {
  const int Vmax = tol.max_dual > 0 ? tol.max_dual : 1;
  const int M = c.M, Ks = c.Ks;
  const RView r = res_view(dyn + dyn_head_floats(kd), c, c.n1 - c.n0);
  const RScratch x = res_scratch(dyn, kd);
  const long long t0 = clock64();
  const GIt gi = group_iter(M);
  load_res(c, r, c.n0);
  for (int m = threadIdx.x; m < M; m += kThreads) {
    x.xi[m] = c.xi[m];
    x.pmf[m] = (float)c.pmax[m];
    x.xscale[m] = 1.f / (LN2F * sh.maskf[m]);
  }
  for (int k = threadIdx.x; k < Ks; k += kThreads) {
    x.zeta[k] = c.zeta[k];
    x.psi[k] = sh_psi(c, k);
  }
  __syncthreads();
  stage_totals(c, r, gi);
  __syncthreads();
  int zc = 0;  // generation of the committed SIC multipliers
  stage_link(c, sh, r, szeta, 1.f, zc, gi);
  __syncthreads();
  stage_rows(c, sh, r, zc ^ 1, gi);
  if (threadIdx.x == 0) cyc[1] += clock64() - t0;
  float dl = 0.f;
  int v = 0;
  for (;;) {
    const long long t1 = clock64();
    // residual sums at p^v and max |p^v - p^{v-1}| / mask, over the cluster
    float *xv = (v & 1) ? x.xch1 : x.xch0;
    const int nx = M + 2 * Ks;
    res_partials(c, sh, r, xv, dl);
    __syncthreads();
    if (threadIdx.x == 0) {
      float d = sh.redf[0];
      for (int i = 1; i < kWarps; i++) d = fmaxf(d, sh.redf[i]);
      xv[nx] = d;
    }
    const float *xt = xv;
    if (c.csize > 1) {
      // peers read this parity's vector before their next barrier; it is
      // rewritten two iterations later, after that barrier
      inst_sync(c);
      for (int i = threadIdx.x; i <= nx; i += kThreads) {
        float t = peer(xv, 0)[i];
        for (int q = 1; q < c.csize; q++) t = i < nx ? t + peer(xv, q)[i] : fmaxf(t, peer(xv, q)[i]);
        x.xtot[i] = t;
      }
      xt = x.xtot;
    }
    __syncthreads();
    const float d = xt[nx];
    if ((v > 0 && d < (float)tol.tol_dual) || v >= Vmax) break;
    const float delta = rsqrtf((float)v + 1.f);
    for (int t = threadIdx.x; t < M + Ks; t += kThreads) {
      if (t < M) {
        const int m = t;
        const float pm = x.pmf[m];
        const float step = delta * ((xt[m] - pm) / pm) * x.xscale[m];
        double xm = x.xi[m];
        if (xm != 0.0 || step > 0.f) {
          xm += (double)step;
          xm = xm > 0.0 ? xm : 0.0;
          x.xi[m] = xm;
        }
        sh.xif[m] = (float)xm;
      } else {
        const int ks = t - M;
        const float rr = xt[M + ks], as = xt[M + Ks + ks];
        const float e = fminf(fmaxf((x.psi[ks] - rr) / fmaxf(as, (float)kZetaAsumMin), -1.f), 1.f);
        const double z = fmin(fmax(x.zeta[ks] * (double)exp2f(e), kZetaMin), kZetaMax);
        x.zeta[ks] = z;
        szeta[ks] = (float)z;
      }
    }
    __syncthreads();
    const long long t2 = clock64();
    zc ^= 1;  // the multipliers of the last link stage become the committed ones
    dl = stage_power(c, sh, r, szeta, gi);
    __syncthreads();
    stage_link(c, sh, r, szeta, rsqrtf((float)v + 2.f), zc, gi);
    __syncthreads();
    stage_rows(c, sh, r, zc ^ 1, gi);
    v++;
    const long long t3 = clock64();
    if (threadIdx.x == 0) {
      cyc[2] += t2 - t1;
      cyc[3] += t3 - t2;
    }
  }
  store_res(c, r, c.n0, zc);
  if (c.crank == 0) {
    for (int m = threadIdx.x; m < M; m += kThreads) c.xi[m] = x.xi[m];
    for (int k = threadIdx.x; k < Ks; k += kThreads) c.zeta[k] = x.zeta[k];
  }
  // gamma, pi, X, totals and SIC sums at the final point for the later phases
  link_all<kLinkOnly>(c, sh, dyn, kd, szeta, 0.f, phase, pending);
  return v;
}

}  // namespace hcran
