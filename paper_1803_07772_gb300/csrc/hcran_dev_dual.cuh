// hcran_dev_dual.cuh -- the Lagrangian dual loop of Algorithm 1 (internal).
//
// Warp w owns subcarriers n = w, w+16, ... .  A sweep visits them in order;
// in staged mode the warp's first lane prefetches the next subcarrier's SIC
// multipliers, slab rows and slot arrays into the other shared staging buffer
// with one-dimensional bulk copies (cp.async.bulk) completed on an mbarrier,
// while the lanes work on the current one.  When the double buffers of every
// warp do not fit, teams of warps share them (hcran_dev_team.cuh).
#pragma once
#include "hcran_dev_link.cuh"

namespace hcran {

enum SweepMode { kLinkOnly = 0, kLinkDual = 1, kFused = 2 };

__device__ __forceinline__ float sh_psi(const Ctx &c, int ks) { return (float)c.Psi[ks]; }

// issue the bulk copies of subcarrier n into staging buffer b (first lane only)
__device__ __forceinline__ void issue_stage(const Ctx &c, Shared &sh, const KDims &kd, float *buf,
                                            int warp, int b, int n, const double *zsrc) {
  const uint32_t fz = 8u * c.NPp, fs = 4u * c.M * c.Up, fa = 4u * c.Up;
  unsigned long long *bar = &sh.bar[warp][b];
  mbar_expect_tx(bar, fz + fs + kStagedArrays * fa);
  bulk_g2s(buf, zsrc + (size_t)n * c.NPp, fz, bar);
  float *f = buf + 2 * kd.NPPmax;
  bulk_g2s(f, c.slab + (size_t)n * c.M * c.Up, fs, bar);
  f += kd.Mmax * kd.Upmax;
  const size_t o = (size_t)n * c.Up;
  const void *src[kStagedArrays] = {c.S + o,    c.p + o,    c.Aden + o,  c.Bnum + o,
                                    c.Cnum + o, c.alpha + o, c.beta + o, c.plin + o,
                                    c.gown + o, c.ginv + o, c.wslot + o};
  for (int i = 0; i < kStagedArrays; i++) bulk_g2s(f + i * kd.Upmax, src[i], fa, bar);
}

}  // namespace hcran

#include "hcran_dev_team.cuh"

namespace hcran {

// One sweep of the warp over its subcarriers.  The caller fences the proxies
// and synchronises the block before it (bulk copies read what the previous
// phase wrote).  Returns the warp's max |dp| / mask (fused mode).
template <int MODE>
__device__ float sweep(const Ctx &c, Shared &sh, float *dyn, const KDims &kd, const float *szeta,
                       float delta, unsigned &phase, unsigned &pending) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const WarpBuf wb = warp_buf(dyn, kd, warp);
  const double *zsrc = MODE == kFused ? c.zsic_next : c.zsic;
  if (MODE != kLinkOnly) {
    for (int j = lane; j < c.M; j += 32) wb.wp[j] = 0.f;
    for (int k = lane; k < c.Ks; k += 32) {
      wb.wr[k] = 0.f;
      wb.wa[k] = 0.f;
    }
    __syncwarp();
  }
  float dl = 0.f;
  int i = 0;
  if (kd.staged && c.n0 + warp < c.n1 && lane == 0) {
    issue_stage(c, sh, kd, wb.stage0, warp, 0, c.n0 + warp, zsrc);
    pending |= 1u;
  }
  for (int n = c.n0 + warp; n < c.n1; n += kWarps, i++) {
    SubView v;
    if (kd.staged) {
      const int b = i & 1;
      const int nn = n + kWarps;
      if (nn < c.n1) {
        __syncwarp();  // every lane is done reading buffer b^1 before the copy refills it
        if (lane == 0) issue_stage(c, sh, kd, b ? wb.stage0 : wb.stage1, warp, b ^ 1, nn, zsrc);
        pending |= 2u >> b;  // bit of buffer b^1
      }
      const bool ok = mbar_wait(&sh.bar[warp][b], (phase >> b) & 1u, sh.spin_limit);
      phase ^= 1u << b;
      pending &= ~(1u << b);
      if (!ok) sh.abort = 1;
      v = staged_view(b ? wb.stage1 : wb.stage0, kd, c.M, c.Up);
    } else {
      v = global_view(c, n, zsrc);
    }
    if (MODE == kFused) {
      dl = fmaxf(dl, power_subcarrier(c, sh, wb, v, szeta, n));
    } else {
      for (int u = lane; u < c.U; u += 32) {
        const int k = v.k[u];
        wb.k[u] = k;
        wb.p[u] = k >= 0 ? v.p[u] : 0.f;
      }
      __syncwarp();
    }
    link_subcarrier(c, sh, wb, v, szeta, n, MODE != kLinkOnly, delta);
  }
  return warp_max(dl);
}

// link pass over every subcarrier, bracketed by block barriers
template <int MODE>
__device__ void link_all(const Ctx &c, Shared &sh, float *dyn, const KDims &kd, const float *szeta,
                         float delta, unsigned &phase, unsigned &pending) {
  fence_proxy_async();
  __syncthreads();
  if (kd.teams > 0) team_sweep<MODE>(c, sh, dyn, kd, szeta, delta, phase, pending);
  else sweep<MODE>(c, sh, dyn, kd, szeta, delta, phase, pending);
  __syncthreads();
}

// One dual loop of Algorithm 1 (one SCALE pass).  Returns the iterations run.
__device__ int dual_loop(const Ctx &c, Shared &sh, float *dyn, const KDims &kd, float *szeta,
                         const Tol &tol, long long *cyc, unsigned &phase, unsigned &pending) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int Vmax = tol.max_dual > 0 ? tol.max_dual : 1;
  const long long t0 = clock64();
  link_all<kLinkDual>(c, sh, dyn, kd, szeta, 1.f, phase, pending);  // residuals at p^0, SIC step delta_0
  if (threadIdx.x == 0) cyc[1] += clock64() - t0;
  int v = 0;
  for (;;) {
    const long long t1 = clock64();
    // stop test of the previous iteration (max |p^{v} - p^{v-1}| / mask)
    float d = sh.redf[0];
    for (int i = 1; i < kWarps; i++) d = fmaxf(d, sh.redf[i]);
    if (sh.abort || (v > 0 && d < (float)tol.tol_dual) || v >= Vmax) break;
    // projected subgradient step on xi' (C12) and zeta' (C13 hat) at p^v:
    // steps in FP32, accumulated into the FP64 multiplier values
    const float delta = rsqrtf((float)v + 1.f);
    // the partials of the warps (warp sweeps) or of the teams (team sweeps)
    const int parts = kd.teams > 0 ? kd.teams : kWarps;
    const int wstride = kd.teams > 0 ? team_stride(kd) : warp_stride(kd);
    const float *wp0 = kd.teams > 0 ? team_buf(kd, 0).wp : warp_buf(dyn, kd, 0).wp;
    const float *wr0 = kd.teams > 0 ? team_buf(kd, 0).wr : warp_buf(dyn, kd, 0).wr;
    const float *wa0 = kd.teams > 0 ? team_buf(kd, 0).wa : warp_buf(dyn, kd, 0).wa;
    for (int t = threadIdx.x; t < c.M + c.Ks; t += kThreads) {
      if (t < c.M) {
        const int m = t;
        float tot = 0.f;
        for (int i = 0; i < parts; i++) tot += wp0[i * wstride + m];
        const float pm = (float)c.pmax[m];
        const float step = delta * ((tot - pm) / pm) / (LN2F * sh.maskf[m]);
        double x = c.xi[m];
        if (x != 0.0 || step > 0.f) {
          x += (double)step;
          x = x > 0.0 ? x : 0.0;
          c.xi[m] = x;
        }
        sh.xif[m] = (float)x;
      } else {
        const int ks = t - c.M;
        float r = 0.f, as = 0.f;
        for (int i = 0; i < parts; i++) {
          r += wr0[i * wstride + ks];
          as += wa0[i * wstride + ks];
        }
        const float x = delta * fminf(fmaxf((sh_psi(c, ks) - r) / fmaxf(as, (float)kZetaAsumMin), -1.f), 1.f);
        const double z = fmin(fmax(c.zeta[ks] * (double)exp2f(x), kZetaMin), kZetaMax);
        c.zeta[ks] = z;
        szeta[ks] = (float)z;
      }
    }
    fence_proxy_async();
    __syncthreads();
    const long long t2 = clock64();
    const float dl = kd.teams > 0
                         ? team_sweep<kFused>(c, sh, dyn, kd, szeta, rsqrtf((float)v + 2.f), phase, pending)
                         : sweep<kFused>(c, sh, dyn, kd, szeta, rsqrtf((float)v + 2.f), phase, pending);
    if (lane == 0) sh.redf[warp] = dl;
    v++;
    __syncthreads();
    const long long t3 = clock64();
    if (threadIdx.x == 0) {
      cyc[2] += t2 - t1;
      cyc[3] += t3 - t2;
    }
  }
  // gamma, pi, X, totals and SIC sums at the final point for the later phases
  link_all<kLinkOnly>(c, sh, dyn, kd, szeta, 0.f, phase, pending);
  return v;
}

// alpha/beta of the SCALE bound at the current point (gamma of the last link pass)
__device__ void scale_update(const Ctx &c) {
  for (int e = c.n0 * c.Up + threadIdx.x; e < c.n1 * c.Up; e += kThreads) {
    if (c.S[e] < 0) continue;
    const float z = fmaxf(c.gam[e], kGammaFloor);
    const float a = z / (1.f + z);
    c.alpha[e] = a;
    c.beta[e] = log1pf(z) / LN2F - a * log2f(z);
  }
  __syncthreads();
}

// exact R (elastic, weighted) of problem (eq7) and P of the Sec. II-A power
// model (eta_m times the transmit power of every selected link) from the last
// link pass
__device__ void exact_R_P(const Ctx &c, Shared &sh, double &R, double &P) {
  double r = 0.0, tx = 0.0;
  for (int e = c.n0 * c.Up + threadIdx.x; e < c.n1 * c.Up; e += kThreads) {
    const int k = c.S[e];
    if (k < 0) continue;
    const int m = (e % c.Up) / c.l;
    tx += c.eta[m] * (double)c.p[e];
    if (k >= c.Ke) continue;
    r += (double)c.w[(size_t)m * c.K + k] * (double)(log1pf(c.gam[e]) / LN2F);
  }
  R = cl_sum(r, sh, c);
  P = c.Pconst + cl_sum(tx, sh, c);
}

// exact C12: scale an RRH's powers down when its total exceeds pmax
__device__ void project_power(const Ctx &c, Shared &sh) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int m = warp; m < c.M; m += kWarps) {
    double t = 0.0;
    for (int n = c.n0 + lane; n < c.n1; n += 32)
      for (int s = 0; s < c.l; s++) {
        const int e = n * c.Up + m * c.l + s;
        if (c.S[e] >= 0) t += (double)c.p[e];
      }
    t = warp_sum(t);
    if (lane == 0) sh.vpart[m] = t;
  }
  cl_vsum(sh, c, c.M);
  for (int m = threadIdx.x; m < c.M; m += kThreads) {
    const double t = sh.vtot[m];
    sh.fac[m] = t > c.pmax[m] ? (float)(c.pmax[m] / t) : 1.f;
  }
  __syncthreads();
  for (int e = c.n0 * c.Up + threadIdx.x; e < c.n1 * c.Up; e += kThreads) {
    if (c.S[e] < 0) continue;
    const int m = (e % c.Up) / c.l;
    const float f = sh.fac[m];
    if (f < 1.f) c.p[e] *= f;
  }
  __syncthreads();
}

}  // namespace hcran
