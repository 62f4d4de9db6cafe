// hcran_dev_team.cuh -- team sweeps of the streamed schedule (internal).
//
// For instances whose dual-loop state fits no cluster's shared memory (the
// 33 x 1024 x 512 shape: 28 MB per instance), every dual iteration streams
// the state of each subcarrier from HBM.  The CTA's warps form kd.teams teams
// of kWarps / kd.teams warps; team t works on subcarriers n0 + t, n0 + t +
// teams, ... one at a time, while the next one is prefetched into the team's
// other staging buffer with one-dimensional bulk copies (cp.async.bulk)
// completed on the team's mbarrier: issued by a producer warp when the teams
// leave one over, else by the team's first thread.  The steps of one
// subcarrier are those of the warp sweep (hcran_dev_link.cuh), shared out
// over the team's threads and separated by the team's named barrier:
//   power     closed-form KKT power per slot (fused sweeps)
//   totals    RRH totals of the subcarrier
//   links     interference, SINR and victim price per slot
//   SIC       multiplier step per pair (C14 in divided form), compacted
//   rows      per (RRH j, chunk): SIC+ / SIC- sums over the nonzero
//             multipliers and the prices RRH j pays towards other RRHs' users
//   slots     the multiplier-free parts of the next KKT denominator/numerator
// A subcarrier's state is read from HBM once per sweep, so a fused sweep
// moves about 4 (M + 11) Up + 8 NPp bytes per subcarrier in and 16 Up + 8 NPp
// out.
#pragma once
#include "hcran_dev_link.cuh"

// included by hcran_dev_dual.cuh after SweepMode and issue_stage

namespace hcran {

struct TeamBuf {
  float *p, *pi, *X;               // [Upmax] per slot of the current subcarrier
  int *k;                          // [Upmax]
  float2 *zw;                      // [Mmax * NPmax] nonzero SIC multipliers, compact, in item order:
                                   //   (z / Gamma_{m,a}, z / Gamma_{m,b}) of pair (a, b)
  int2 *zq;                        // [Mmax * NPmax] their slots (a, b)
  float *Pt, *pio, *Sp, *Sm, *wp;  // [Mmax]
  float *zd;                       // [Mmax * NPmax] SIC multipliers of the subcarrier (0: inactive)
  float *part;                     // [3 * team threads] per-thread partial sums
  float *wr, *wa;                  // [KSmax] streaming rate / alpha partials of the team
  int *cnt;                        // [4] nonzero multipliers of the subcarrier
  float *stage0, *stage1;          // staging buffers
};

// Views are built from hcran_dyn itself and passed by value into inlined
// steps, so that every pointer stays a register holding a shared-memory
// address: a view passed by reference lives in local memory, and each access
// through it then waits on a local load first.
__device__ __forceinline__ TeamBuf team_buf(const KDims &kd, int team) {
  float *b = hcran_dyn + dyn_head_floats(kd) + team * team_stride(kd);
  const int np = kd.NPmax > 0 ? kd.NPmax : 1;
  TeamBuf t;
  t.stage0 = b;  // staging buffers first: 16-byte aligned
  t.stage1 = b + stage_buf_floats(kd);
  b += 2 * stage_buf_floats(kd);
  t.p = b; b += kd.Upmax;
  t.pi = b; b += kd.Upmax;
  t.X = b; b += kd.Upmax;
  t.k = reinterpret_cast<int *>(b); b += kd.Upmax;
  t.zw = reinterpret_cast<float2 *>(b); b += 2 * kd.Mmax * np;  // 8-byte aligned: Upmax is a multiple of 4
  t.zq = reinterpret_cast<int2 *>(b); b += 2 * kd.Mmax * np;
  t.Pt = b; b += kd.Mmax;
  t.pio = b; b += kd.Mmax;
  t.Sp = b; b += kd.Mmax;
  t.Sm = b; b += kd.Mmax;
  t.wp = b; b += kd.Mmax;
  t.zd = b; b += kd.Mmax * np;
  t.part = b; b += 3 * team_threads(kd);
  t.wr = b; b += (kd.KSmax > 0 ? kd.KSmax : 1);
  t.wa = b; b += (kd.KSmax > 0 ? kd.KSmax : 1);
  t.cnt = reinterpret_cast<int *>(b);
  return t;
}

// named barrier of one team (ids 2, 3, ...; 0 is the block barrier)
__device__ __forceinline__ void team_bar(int team, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(2 + team), "r"(nthreads) : "memory");
}

// Link pass of subcarrier n by one team (tt: thread in the team, TS: team
// size) at the point in tb.p / tb.k; same quantities as link_subcarrier.
// Ends with the team's barrier, after which the stage buffer may be refilled.
__device__ __forceinline__ void team_link(const Ctx &c, const Shared &sh, const TeamBuf tb, const SubView v,
                                          const float *szeta, int n, bool dual, float delta, int team, int tt,
                                          int TS) {
  const int M = c.M, U = c.U, l = c.l, Up = c.Up;
  const float *sl = v.slab;
  for (int j = tt; j < M; j += TS) {
    float t = 0.f;
    for (int s = 0; s < l; s++) t += tb.p[j * l + s];
    tb.Pt[j] = t;
    if (dual) tb.wp[j] += t;
    else c.Ptot[n * M + j] = t;
  }
  team_bar(team, TS);
  for (int u = tt; u < U; u += TS) {
    const int k = tb.k[u];
    float pi = 0.f, inter = 0.f, gam = 0.f;
    if (k >= 0) {
      const int m = sh.slot_m[u], s = sh.slot_s[u];
#pragma unroll 4
      for (int j = 0; j < M; j++) inter += sl[j * Up + u] * tb.Pt[j];  // own entry is zero
      float intra = 0.f;
      for (int b = 0; b < s; b++) intra += tb.p[m * l + b];
      const float g_own = v.gown[u];
      const float inv = fast_rcp(c.sigma + g_own * intra + inter);
      const float a = v.alpha[u];
      gam = tb.p[u] * g_own * inv;
      const float wk = v.w[u];
      pi = (k >= c.Ke ? szeta[k - c.Ke] * wk : wk) * a * kInvLn2 * inv;
      if (dual && k >= c.Ke) {  // a streaming user appears at most once per subcarrier
        const int ks = k - c.Ke;
        tb.wr[ks] += wk * (a * log2f(fmaxf(gam, kGammaFloor)) + v.beta[u]);
        tb.wa[ks] += a;
      }
    }
    tb.pi[u] = pi;
    tb.X[u] = inter;
    if (!dual) {
      const int e = n * Up + u;
      c.gam[e] = gam;
      c.pi[e] = pi;
      c.X[e] = inter;
    }
  }
  team_bar(team, TS);
  // C14 in divided form per selected pair: the step (dual), then the nonzero
  // multipliers in item order as a compact list for the SIC+ / SIC- sums
  int nnz = 0;
  if (c.npair > 0) {
    const int items = M * c.npair;
    for (int it = tt; it < items; it += TS) {
      const int ua = sh.item_a[it], ub = sh.item_b[it];
      double zz = v.z[it];
      const bool both = tb.k[ua] >= 0 && tb.k[ub] >= 0;
      if (both && dual) {
        // step in FP32, accumulated into the FP64 multiplier (skipped while it stays at 0)
        const float ra = (c.sigma + tb.X[ua]) * v.ginv[ua];
        const float rb = (c.sigma + tb.X[ub]) * v.ginv[ub];
        const float step = delta * (ra - rb) * fast_rcp(rb) * sh.sicscale[sh.item_m[it]];
        if (zz != 0.0 || step > 0.f) {
          zz += (double)step;
          zz = zz > 0.0 ? zz : 0.0;
        }
      }
      if (dual) c.zsic_next[n * c.NPp + it] = zz;
      tb.zd[it] = both ? (float)zz : 0.f;
    }
    team_bar(team, TS);
    if (tt < 32) {  // the team's first warp compacts, with the weights the row sums need
      int q0 = 0;
      for (int base = 0; base < items; base += 32) {
        const int it = base + tt;
        const float zf = it < items ? tb.zd[it] : 0.f;
        const unsigned bal = __ballot_sync(0xffffffffu, zf != 0.f);
        if (zf != 0.f) {
          const int q = q0 + __popc(bal & ((1u << tt) - 1u));
          const int ua = sh.item_a[it], ub = sh.item_b[it];
          tb.zq[q] = make_int2(ua, ub);
          tb.zw[q] = make_float2(zf * v.ginv[ua], zf * v.ginv[ub]);
        }
        q0 += __popc(bal);
      }
      if (tt == 0) tb.cnt[0] = q0;
    }
    team_bar(team, TS);
    nnz = tb.cnt[0];
  }
  // per (row j, chunk): coefficient of Ptot_j in Omega_bar is
  // Gamma_{j,a}/Gamma_{m,a} - Gamma_{j,b}/Gamma_{m,b} (0 for j = m: the own
  // entries are zeroed); the price row j of the slab against pi (dual)
  const int C = TS / M >= 1 ? TS / M : 1;
  for (int h = tt; h < M * C; h += TS) {
    const int j = h / C, ch = h - j * C;
    const float *row = sl + j * Up;
    float sp = 0.f, sm = 0.f, acc = 0.f;
#pragma unroll 2
    for (int q = ch; q < nnz; q += C) {  // z times the coefficient, whose sign it keeps
      const int2 ab = tb.zq[q];
      const float2 wz = tb.zw[q];
      const float t = row[ab.x] * wz.x - row[ab.y] * wz.y;
      if (t > 0.f) sp += t;
      else sm -= t;
    }
    if (dual)
      for (int u = ch; u < U; u += C) acc += row[u] * tb.pi[u];
    tb.part[h] = sp;
    tb.part[TS + h] = sm;
    tb.part[2 * TS + h] = acc;
  }
  team_bar(team, TS);
  for (int j = tt; j < M; j += TS) {  // chunks summed in a fixed order
    float sp = 0.f, sm = 0.f, acc = 0.f;
    for (int ch = 0; ch < C; ch++) {
      sp += tb.part[j * C + ch];
      sm += tb.part[TS + j * C + ch];
      acc += tb.part[2 * TS + j * C + ch];
    }
    tb.Sp[j] = sp;
    tb.Sm[j] = sm;
    tb.pio[j] = acc;
    if (!dual) {
      c.SICp[n * M + j] = sp;
      c.SICm[n * M + j] = sm;
    }
  }
  if (dual) {
    team_bar(team, TS);
    for (int u = tt; u < U; u += TS) {
      const int e = n * Up + u;
      const int k = tb.k[u];
      float A = 0.f, B = 0.f, Cn = 0.f;
      if (k >= 0) {
        const int m = sh.slot_m[u], s = sh.slot_s[u];
        float own = 0.f;  // weaker users of the same (m,n) hear this slot
        for (int b = s + 1; b < l; b++) own += tb.pi[m * l + b] * v.gown[m * l + b];
        A = tb.pio[m] + own + tb.Sp[m];
        B = v.w[u] * v.alpha[u] * kInvLn2;
        Cn = tb.Sm[m] * v.plin[u];
      }
      c.Aden[e] = A;
      c.Bnum[e] = B;
      c.Cnum[e] = Cn;
    }
  }
  team_bar(team, TS);
}

// Closed-form KKT power of every slot of subcarrier n by one team (as
// power_subcarrier); the caller synchronises the team afterwards.
__device__ __forceinline__ float team_power(const Ctx &c, const Shared &sh, const TeamBuf tb, const SubView v,
                                            const float *szeta, int n, int tt, int TS) {
  float dmax = 0.f;
  for (int u = tt; u < c.U; u += TS) {
    const int k = v.k[u];
    tb.k[u] = k;
    if (k < 0) {
      tb.p[u] = 0.f;
      continue;
    }
    const int m = sh.slot_m[u];
    const float p = v.p[u];
    const float den = sh.qeta[m] + sh.xif[m] + v.A[u];
    const float cw = k < c.Ke ? 1.f : szeta[k - c.Ke];
    const float num = cw * v.B[u] + v.C[u];
    const float mk = sh.maskf[m];
    float pv = (den <= 0.f || num >= den * mk) ? mk : num * fast_rcp(den);
    pv = fmaxf(pv, sh.floorf[m]);
    dmax = fmaxf(dmax, fabsf(pv - p) * sh.invmask[m]);
    c.p[n * c.Up + u] = pv;
    tb.p[u] = pv;
  }
  for (int it = tt; it < c.M * c.npair; it += TS) c.zsic[n * c.NPp + it] = v.z[it];
  return dmax;
}

__device__ __forceinline__ void mbar_arrive_cta(unsigned long long *bar) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(smem_addr(bar))
               : "memory");
}

// Producer of the team sweeps when kd.teams leaves a warp over (3 teams of 5
// warps): the first lane of the last warp issues every team's staging copies,
// in the order the teams consume them, so that no team's thread spends its
// time issuing them.  Team t's i-th subcarrier goes to its buffer i & 1; from
// the third on, the producer first waits until the team has released the
// buffer (its first thread arrives on ebar after the subcarrier's last
// barrier).  sh.eph keeps the parity of the next release phase of every
// buffer across sweeps: each use of a buffer completes one phase.
__device__ void team_produce(const Ctx &c, Shared &sh, const KDims &kd, const double *zsrc) {
  const int T = kd.teams;
  unsigned ph = sh.eph;
  const int rounds = (c.n1 - c.n0 + T - 1) / T;
  for (int i = 0; i < rounds; i++)
    for (int t = 0; t < T; t++) {
      const int n = c.n0 + t + i * T;
      if (n >= c.n1) continue;
      const int b = i & 1, bit = 2 * t + b;
      if (i >= 2) {
        if (!mbar_wait(&sh.ebar[t][b], (ph >> bit) & 1u, sh.spin_limit)) sh.abort = 1;
        ph ^= 1u << bit;
      }
      const TeamBuf tb = team_buf(kd, t);
      issue_stage(c, sh, kd, b ? tb.stage1 : tb.stage0, t, b, n, zsrc);
    }
  // the last use of each buffer completes a phase nobody waits for this sweep
  for (int t = 0; t < T; t++)
    for (int b = 0; b < 2; b++)
      if (c.n0 + t + b * T < c.n1) ph ^= 1u << (2 * t + b);
  sh.eph = ph;
}

// team of warp `warp` (kd.teams teams of kWarps / kd.teams warps; warps past
// the last team take no part in the sweeps, except the producer)
__device__ __forceinline__ int team_of(const KDims &kd, int warp) { return warp / (kWarps / kd.teams); }

// One sweep of every team over its subcarriers (same contract as sweep).
template <int MODE>
__device__ float team_sweep(const Ctx &c, Shared &sh, float *dyn, const KDims &kd, const float *szeta,
                            float delta, unsigned &phase, unsigned &pending) {
  const int warp = threadIdx.x >> 5;
  const int T = kd.teams, TS = team_threads(kd);
  const int team = team_of(kd, warp);
  const bool producer = (kWarps % T) != 0;  // a warp is left over: it issues the copies
  if (team >= T) {
    if (producer && warp == kWarps - 1 && (threadIdx.x & 31) == 0)
      team_produce(c, sh, kd, MODE == kFused ? c.zsic_next : c.zsic);
    return 0.f;
  }
  const int tt = (int)threadIdx.x - team * TS;
  const TeamBuf tb = team_buf(kd, team);
  (void)dyn;
  const double *zsrc = MODE == kFused ? c.zsic_next : c.zsic;
  if (MODE != kLinkOnly) {
    for (int j = tt; j < c.M; j += TS) tb.wp[j] = 0.f;
    for (int k = tt; k < c.Ks; k += TS) {
      tb.wr[k] = 0.f;
      tb.wa[k] = 0.f;
    }
  }
  team_bar(team, TS);
  float dl = 0.f;
  int i = 0;
  if (c.n0 + team < c.n1) {
    if (!producer && tt == 0) issue_stage(c, sh, kd, tb.stage0, team, 0, c.n0 + team, zsrc);
    pending |= 1u;
  }
  for (int n = c.n0 + team; n < c.n1; n += T, i++) {
    const int b = i & 1;
    const int nn = n + T;
    if (nn < c.n1) {  // buffer b^1 was released by the barrier that ended the last subcarrier
      if (!producer && tt == 0) issue_stage(c, sh, kd, b ? tb.stage0 : tb.stage1, team, b ^ 1, nn, zsrc);
      pending |= 2u >> b;
    }
    const bool ok = mbar_wait(&sh.bar[team][b], (phase >> b) & 1u, sh.spin_limit);
    phase ^= 1u << b;
    pending &= ~(1u << b);
    if (!ok) sh.abort = 1;
    const SubView v = staged_view(b ? tb.stage1 : tb.stage0, kd, c.M, c.Up);
    if (MODE == kFused) {
      dl = fmaxf(dl, team_power(c, sh, tb, v, szeta, n, tt, TS));
    } else {
      for (int u = tt; u < c.U; u += TS) {
        const int k = v.k[u];
        tb.k[u] = k;
        tb.p[u] = k >= 0 ? v.p[u] : 0.f;
      }
    }
    team_bar(team, TS);
    team_link(c, sh, tb, v, szeta, n, MODE != kLinkOnly, delta, team, tt, TS);
    if (producer && tt == 0) mbar_arrive_cta(&sh.ebar[team][b]);  // buffer b is free again
  }
  return warp_max(dl);
}

}  // namespace hcran
