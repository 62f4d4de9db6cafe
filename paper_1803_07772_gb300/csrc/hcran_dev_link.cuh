// hcran_dev_link.cuh -- per-subcarrier link pass and KKT power update of the
// dual loop (internal).  One warp handles one subcarrier at a time.  The slab
// holds every RRH's gain to the users of the subcarrier's slots with the
// serving RRH's entry zeroed, so the interference at a slot and the price an
// RRH pays towards the other RRHs' users are plain dot products; the serving
// gain and its reciprocal come as separate per-slot arrays.
#pragma once
#include "hcran_dev_common.cuh"

namespace hcran {

// Link pass of subcarrier n at the point in wb.p / wb.k (Sec. II-A SINR with
// the SIC order): RRH totals, inter-cell interference X, SINR gamma, victim
// prices pi = c alpha / (ln2 (sigma + I)).  Without `dual` it stores gamma,
// pi, X, the RRH totals and the SIC sums for the phases that read them
// (selection, SCALE update, R and P).  With `dual` it instead produces what
// the next KKT update needs: the SIC multiplier step of this subcarrier (into
// zsic_next, step delta, from v.z), the residual partials of C12 and C13-hat,
// and the multiplier-free parts of the next denominator and numerator:
// Aden = prices paid towards other RRHs' users + weaker users of the same
// (m,n) + SIC+ sum, Bnum = w alpha / ln2, Cnum = SIC- sum * p_lin.
__device__ void link_subcarrier(const Ctx &c, const Shared &sh, const WarpBuf &wb, const SubView &v,
                                const float *szeta, int n, bool dual, float delta) {
  const int lane = threadIdx.x & 31;
  const int M = c.M, U = c.U, l = c.l, Up = c.Up;
  const float *sl = v.slab;
  for (int j = lane; j < M; j += 32) {
    float t = 0.f;
    for (int s = 0; s < l; s++) t += wb.p[j * l + s];
    wb.Pt[j] = t;
    if (dual) wb.wp[j] += t;
    else c.Ptot[n * M + j] = t;
  }
  __syncwarp();
  for (int u = lane; u < U; u += 32) {
    const int k = wb.k[u];
    float pi = 0.f, inter = 0.f, gam = 0.f;
    if (k >= 0) {
      const int m = sh.slot_m[u], s = sh.slot_s[u];
#pragma unroll 4
      for (int j = 0; j < M; j++) inter += sl[j * Up + u] * wb.Pt[j];  // own entry is zero
      float intra = 0.f;
      for (int b = 0; b < s; b++) intra += wb.p[m * l + b];
      const float g_own = v.gown[u];
      const float inv = fast_rcp(c.sigma + g_own * intra + inter);
      const float a = v.alpha[u];
      gam = wb.p[u] * g_own * inv;
      const float wk = v.w[u];
      pi = (k >= c.Ke ? szeta[k - c.Ke] * wk : wk) * a * kInvLn2 * inv;
      if (dual && k >= c.Ke) {  // a streaming user appears at most once per subcarrier
        const int ks = k - c.Ke;
        wb.wr[ks] += wk * (a * log2f(fmaxf(gam, kGammaFloor)) + v.beta[u]);
        wb.wa[ks] += a;
      }
    }
    wb.pi[u] = pi;
    wb.X[u] = inter;
    if (!dual) {
      const int e = n * Up + u;
      c.gam[e] = gam;
      c.pi[e] = pi;
      c.X[e] = inter;
    }
  }
  __syncwarp();
  // C14 in divided form per selected pair; the nonzero multipliers go to a
  // compact list, from which the SIC+ / SIC- sums per RRH are formed
  int nnz = 0;
  if (c.npair > 0) {
    const int items = M * c.npair;
    for (int base = 0; base < items; base += 32) {
      const int it = base + lane;
      float zf = 0.f;
      if (it < items) {
        const int ua = sh.item_a[it], ub = sh.item_b[it];
        double zz = v.z[it];
        const bool both = wb.k[ua] >= 0 && wb.k[ub] >= 0;
        if (both && dual) {
          // step in FP32, accumulated into the FP64 multiplier (skipped while it stays at 0)
          const float ra = (c.sigma + wb.X[ua]) * v.ginv[ua];
          const float rb = (c.sigma + wb.X[ub]) * v.ginv[ub];
          const float step = delta * (ra - rb) * fast_rcp(rb) * sh.sicscale[sh.item_m[it]];
          if (zz != 0.0 || step > 0.f) {
            zz += (double)step;
            zz = zz > 0.0 ? zz : 0.0;
          }
        }
        if (dual) c.zsic_next[n * c.NPp + it] = zz;
        zf = both ? (float)zz : 0.f;
      }
      const unsigned bal = __ballot_sync(0xffffffffu, zf != 0.f);
      if (zf != 0.f) {
        const int q = nnz + __popc(bal & ((1u << lane) - 1u));
        wb.zl[q] = it;
        wb.zs[q] = zf;
      }
      nnz += __popc(bal);
    }
    __syncwarp();
  }
  // coefficient of Ptot_j in Omega_bar is Gamma_{j,a}/Gamma_{m,a} - Gamma_{j,b}/Gamma_{m,b};
  // the zeroed own entries make it 0 for j = m
  for (int j = lane; j < M; j += 32) {
    const float *row = sl + j * Up;
    float sp = 0.f, sm = 0.f;
    for (int q = 0; q < nnz; q++) {
      const int it = wb.zl[q];
      const int ua = sh.item_a[it], ub = sh.item_b[it];
      const float cc = row[ua] * v.ginv[ua] - row[ub] * v.ginv[ub];
      const float z = wb.zs[q];
      if (cc > 0.f) sp += z * cc;
      else sm -= z * cc;
    }
    wb.Sp[j] = sp;
    wb.Sm[j] = sm;
    if (!dual) {
      c.SICp[n * M + j] = sp;
      c.SICm[n * M + j] = sm;
    }
  }
  if (dual) {
    __syncwarp();
    // price a transmitter of RRH j pays towards the other RRHs' users on n:
    // row j of the slab against pi, split over lanes (j, chunk), summed per j
    // in a fixed order
    if (M <= 32) {
      const int C = sh.pio_chunks, j = sh.pio_j[lane], ch = sh.pio_ch[lane];
      if (ch < C) {
        const float *row = sl + j * Up;
        float acc = 0.f;
        for (int u = ch; u < U; u += C) acc += row[u] * wb.pi[u];
        wb.part[ch * M + j] = acc;
      }
      __syncwarp();
      if (lane < M) {
        float t = 0.f;
        for (int q = 0; q < C; q++) t += wb.part[q * M + lane];
        wb.pio[lane] = t;
      }
    } else {
      for (int j = lane; j < M; j += 32) {
        const float *row = sl + j * Up;
        float acc = 0.f;
        for (int u = 0; u < U; u++) acc += row[u] * wb.pi[u];
        wb.pio[j] = acc;
      }
    }
    __syncwarp();
    for (int u = lane; u < U; u += 32) {
      const int e = n * Up + u;
      const int k = wb.k[u];
      float A = 0.f, B = 0.f, Cn = 0.f;
      if (k >= 0) {
        const int m = sh.slot_m[u], s = sh.slot_s[u];
        float own = 0.f;  // weaker users of the same (m,n) hear this slot
        for (int b = s + 1; b < l; b++) own += wb.pi[m * l + b] * v.gown[m * l + b];
        A = wb.pio[m] + own + wb.Sp[m];
        B = v.w[u] * v.alpha[u] * kInvLn2;
        Cn = wb.Sm[m] * v.plin[u];
      }
      c.Aden[e] = A;
      c.Bnum[e] = B;
      c.Cnum[e] = Cn;
    }
  }
  __syncwarp();
}

// Closed-form KKT power of every slot of subcarrier n (eq. 653 / 683 in the
// log-power variable, Jacobi: all slots from the same point) with the current
// multipliers; commits the SIC step of this subcarrier (v.z holds it).  Puts
// the new point in wb.p / wb.k and returns the lane's max |p_new - p| / mask.
__device__ float power_subcarrier(const Ctx &c, const Shared &sh, const WarpBuf &wb, const SubView &v,
                                  const float *szeta, int n) {
  const int lane = threadIdx.x & 31;
  float dmax = 0.f;
  for (int u = lane; u < c.U; u += 32) {
    const int k = v.k[u];
    wb.k[u] = k;
    if (k < 0) {
      wb.p[u] = 0.f;
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
    wb.p[u] = pv;
  }
  for (int it = lane; it < c.M * c.npair; it += 32) c.zsic[n * c.NPp + it] = v.z[it];
  __syncwarp();
  return dmax;
}

}  // namespace hcran
