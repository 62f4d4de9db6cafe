// hcran_dev_select.cuh -- RRH / subcarrier / NOMA selection and the initial
// point (internal).  Selection is the explicit form of the binaries of C1, C2,
// C5, C6 once C10/C11 are relaxed with rho -> 0: at the current prices, the
// water-filling utility of every (m, k, n) decides A_k = argmax_m sum_n u,
// then each (m, n) admits users of m greedily by utility while the set stays
// SIC-feasible (C14) and has at most l members.
#pragma once
#include "hcran_dev_resident.cuh"

namespace hcran {

// Water-filling candidate of user k on (m, n) at the current prices:
// maximise c log2(1 + g p) - den p on [0, mask].
__device__ float cand_utility(const Ctx &c, const Shared &sh, const float *szeta, int n, int m, int k,
                              float *ps_out, float *X_out, float *key_out) {
  const int a = c.A[k];
  float pk = 0.f;
  if (a >= 0) {
    const int u = c.uslot[(size_t)k * c.N + n];
    if (u >= 0) pk = c.p[n * c.Up + u];
  }
  float X = 0.f;
  for (int j = 0; j < c.M; j++)
    if (j != m) X += gain(c, n, j, k) * (c.Ptot[n * c.M + j] - (j == a ? pk : 0.f));
  const float gk = gain(c, n, m, k);
  float Y = 0.f, Pi = 0.f;
  for (int j = 0; j < c.M; j++)
    for (int b = 0; b < c.l; b++) {
      const int ub = j * c.l + b;
      const int v = c.S[n * c.Up + ub];
      if (v < 0) break;
      if (v == k) continue;
      if (j != m) {
        Pi += c.pi[n * c.Up + ub] * sgain(c, n, m, ub);
      } else {
        const float gv = c.gown[n * c.Up + ub];
        if (stronger(gv, v, gk, k)) Y += c.p[n * c.Up + ub];
        else Pi += c.pi[n * c.Up + ub] * gv;
      }
    }
  const float g = gk / (c.sigma + X + gk * Y);
  const float den = sh.qeta[m] + sh.xif[m] + Pi + c.SICp[n * c.M + m];
  const float cw = weight_c(c, szeta, m, k);
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

// repack the gains of the selected users: slab[n][j][u] = Gamma_{j, S[n][u]}^{(n)}
// for the RRHs j other than the slot's own, gown/ginv = the serving gain and its reciprocal
__device__ void build_slab(const Ctx &c) {
  const int Nc = c.n1 - c.n0;
  for (int t = threadIdx.x; t < c.K * Nc; t += kThreads) {
    const int k = t / Nc;
    c.uslot[(size_t)k * c.N + c.n0 + (t - k * Nc)] = -1;
  }
  __syncthreads();
  for (int e = c.n0 * c.Up + threadIdx.x; e < c.n1 * c.Up; e += kThreads) {
    const int k = c.S[e];
    if (k >= 0) c.uslot[(size_t)k * c.N + e / c.Up] = e % c.Up;
  }
  const int MU = c.M * c.Up;
  for (int t = c.n0 * MU + threadIdx.x; t < c.n1 * MU; t += kThreads) {
    const int n = t / MU, r = t - n * MU, j = r / c.Up, u = r - j * c.Up;
    const int k = u < c.U ? c.S[n * c.Up + u] : -1;
    const bool own = u < c.U && j == u / c.l;
    c.slab[t] = (k >= 0 && !own) ? gain(c, n, j, k) : 0.f;
  }
  for (int e = c.n0 * c.Up + threadIdx.x; e < c.n1 * c.Up; e += kThreads) {
    const int k = c.S[e], u = e % c.Up;
    const float g = k >= 0 ? gain(c, e / c.Up, u / c.l, k) : 0.f;
    c.gown[e] = g;
    c.ginv[e] = k >= 0 ? 1.f / g : 0.f;
    c.wslot[e] = k >= 0 ? c.wf[(u / c.l) * c.K + k] : 0.f;
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

// SIC order on (m, n): gain descending, lower id first (insertion sort of a
// short list)
__device__ __forceinline__ void sort_sic(const Ctx &c, int n, int m, int *ids, int cnt) {
  float cg[kMaxL];
  for (int i = 0; i < cnt; i++) cg[i] = gain(c, n, m, ids[i]);
  for (int i = 1; i < cnt; i++) {
    const int x = ids[i];
    const float gx = cg[i];
    int j = i - 1;
    while (j >= 0 && stronger(gx, x, cg[j], ids[j])) {
      ids[j + 1] = ids[j];
      cg[j + 1] = cg[j];
      j--;
    }
    ids[j + 1] = x;
    cg[j + 1] = gx;
  }
}

// greedy SIC-feasible admission on (n, m): the users of m in (utility desc,
// id asc) order while their utility is positive, each kept when every pair
// with the users kept before satisfies Omega_bar <= 0, at most l; written to
// Snew in SIC order
__device__ void admit(const Ctx &c, int n, int m, float tie_eps, float &mm, int &nt) {
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
      if (ra - rb > 0.f) feasible = false;  // Omega_bar > 0: SIC would fail
    }
    if (feasible) chosen[nc++] = bk;
  }
  if (nc == c.l) {  // first user left out by the cap
    float bu2;
    const int k2 = next_candidate(c, n, m, lu, lk, bu2);
    const float ul = c.cu[(size_t)n * c.K + chosen[c.l - 1]];
    if (k2 >= 0 && bu2 > 0.f) track((ul - bu2) / ul, tie_eps, mm, nt);
  }
  sort_sic(c, n, m, chosen, nc);
  const int base = n * c.Up + m * c.l;
  for (int s = 0; s < c.l; s++) c.Snew[base + s] = s < nc ? chosen[s] : -1;
}

// C9 needs every streaming user served.  A streaming user that admission left
// without a link gets one, in user order, on the subcarrier of its RRH (A_k,
// or Again_k when A_k = -1) with the largest gain (lowest n on equal gains)
// where Snew has a free slot or an elastic user; a full (m, n) gives up its
// elastic user of least utility (higher id on equal utility).  Runs on the
// whole cluster; a user costs a few cluster barriers, and there is usually
// none.
__device__ void fixup_streaming(const Ctx &c, Shared &sh, float tie_eps, float &mm, int &nt) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // served flags of this CTA's subcarriers (admission only places k on A_k)
  for (int ks = warp; ks < c.Ks; ks += kWarps) {
    const int k = c.Ke + ks, m = c.Anew[k];
    int f = 0;
    if (m >= 0)
      for (int n = c.n0 + lane; n < c.n1 && !f; n += 32)
        for (int s = 0; s < c.l; s++)
          if (c.Snew[n * c.Up + m * c.l + s] == k) f = 1;
    f = __any_sync(0xffffffffu, f);
    if (lane == 0) c.srv[c.crank * c.Ks + ks] = f;
  }
  inst_sync(c);
  for (int ks = 0; ks < c.Ks; ks++) {
    int f = 0;
    for (int r = 0; r < c.csize; r++) f |= c.srv[r * c.Ks + ks];
    if (f) continue;  // the same decision on every thread of the cluster
    const int k = c.Ke + ks;
    const int m = c.Anew[k] >= 0 ? c.Anew[k] : c.Again[k];
    // this CTA's eligible subcarrier of largest gain (lowest n on ties)
    if (warp == 0) {
      float bg = -1.f;
      int bn = -1;
      for (int n = c.n0 + lane; n < c.n1; n += 32) {
        int cnt = 0, el = 0;
        for (int s = 0; s < c.l; s++) {
          const int v = c.Snew[n * c.Up + m * c.l + s];
          if (v < 0) continue;
          cnt++;
          if (v < c.Ke) el = 1;
        }
        if (cnt == c.l && !el) continue;
        const float g = gain(c, n, m, k);
        if (g > bg) {  // lanes visit n in increasing order: ties keep the lower n
          bg = g;
          bn = n;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const float og = __shfl_xor_sync(0xffffffffu, bg, o);
        const int on = __shfl_xor_sync(0xffffffffu, bn, o);
        if (on >= 0 && (bn < 0 || og > bg || (og == bg && on < bn))) {
          bg = og;
          bn = on;
        }
      }
      if (lane == 0) {
        sh.cxf = bg;
        sh.cxi = bn;
      }
    }
    inst_sync(c);
    float bg = -1.f;
    int bn = -1;
    for (int r = 0; r < c.csize; r++) {  // CTA r holds higher subcarriers than r - 1
      const float og = c.csize > 1 ? *peer(&sh.cxf, r) : sh.cxf;
      const int on = c.csize > 1 ? *peer(&sh.cxi, r) : sh.cxi;
      if (on >= 0 && (bn < 0 || og > bg)) {
        bg = og;
        bn = on;
      }
    }
    if (bn >= c.n0 && bn < c.n1 && threadIdx.x == 0) {
      const int base = bn * c.Up + m * c.l;
      int ids[kMaxL], cnt = 0, rs = -1;
      float ur = 0.f;
      for (int s = 0; s < c.l; s++) {
        const int v = c.Snew[base + s];
        if (v < 0 || v >= c.Ke) continue;
        const float uv = c.cu[(size_t)bn * c.K + v];
        const int vr = rs >= 0 ? c.Snew[base + rs] : -1;
        if (rs < 0 || uv < ur || (uv == ur && v > vr)) {
          rs = s;
          ur = uv;
        }
      }
      int full = 0;
      for (int s = 0; s < c.l; s++) full += c.Snew[base + s] >= 0;
      const int drop = full < c.l ? -1 : rs;
      for (int s = 0; s < c.l; s++) {
        const int v = c.Snew[base + s];
        if (v >= 0 && s != drop) ids[cnt++] = v;
      }
      if (drop >= 0)  // margin of the displaced user against the other elastic users
        for (int i = 0; i < cnt; i++)
          if (ids[i] < c.Ke) {
            const float uo = c.cu[(size_t)bn * c.K + ids[i]];
            track(fabsf(uo - ur) / fmaxf(fabsf(uo), fabsf(ur)), tie_eps, mm, nt);
          }
      ids[cnt++] = k;
      sort_sic(c, bn, m, ids, cnt);
      for (int s = 0; s < c.l; s++) c.Snew[base + s] = s < cnt ? ids[s] : -1;
    }
    if (c.crank == 0 && threadIdx.x == 0) c.Anew[k] = m;
    inst_sync(c);
  }
}

// the new selection of (n, m) from Snew: kept links keep their power, new
// links start at the water-filling power (at least the floor), dropped links
// go to 0; alpha = 1, beta = 0; SIC multipliers reset where the set changed.
// Returns true when the set changed.
__device__ bool apply_selection(const Ctx &c, const Shared &sh, int n, int m) {
  const int base = n * c.Up + m * c.l;
  int oldk[kMaxL];
  float oldp[kMaxL], oldl[kMaxL];
  bool same = true;
  for (int s = 0; s < c.l; s++) {
    oldk[s] = c.S[base + s];
    oldp[s] = c.p[base + s];
    oldl[s] = c.plin[base + s];
    if (oldk[s] != c.Snew[base + s]) same = false;
  }
  for (int s = 0; s < c.l; s++) {
    const int e = base + s;
    const int k = c.Snew[e];
    c.S[e] = k;
    if (k < 0) {
      c.p[e] = 0.f;
      c.plin[e] = 0.f;
    } else {
      int old = -1;
      for (int b = 0; b < c.l; b++)
        if (oldk[b] == k) old = b;
      if (old >= 0) {
        c.p[e] = oldp[old];
        c.plin[e] = oldl[old];
      } else {
        c.p[e] = fmaxf(c.cp[(size_t)n * c.K + k], sh.floorf[m]);
        c.plin[e] = c.p[e];
      }
    }
    c.alpha[e] = 1.f;
    c.beta[e] = 0.f;
  }
  if (!same)
    for (int pr = 0; pr < c.npair; pr++) c.zsic[(size_t)n * c.NPp + m * c.npair + pr] = 0.0;
  return !same;
}

// Returns 1 when the selection changed.
__device__ int selection(const Ctx &c, Shared &sh, float *dyn, const KDims &kd, const float *szeta,
                         float tie_eps, unsigned &phase, unsigned &pending) {
  link_all<kLinkOnly>(c, sh, dyn, kd, szeta, 0.f, phase, pending);  // prices, totals, SIC sums
  float mm = 1.f;
  int nt = 0;
  // (A) per-chunk sums over n of the candidate utilities; the chunks split this
  // CTA's subcarriers, chunk ch of CTA r is global chunk r * nch + ch
  const int nch = c.nchunk / c.csize, Nc = c.n1 - c.n0;
  for (int t = threadIdx.x; t < nch * c.K; t += kThreads) {
    const int ch = t / c.K, k = t - ch * c.K;
    const int n0 = c.n0 + (int)((int64_t)Nc * ch / nch), n1 = c.n0 + (int)((int64_t)Nc * (ch + 1) / nch);
    float *up = c.Upart + (size_t)(c.crank * nch + ch) * c.M * c.K + k;
    for (int m = 0; m < c.M; m++) {
      float acc = 0.f;
      for (int n = n0; n < n1; n++) acc += cand_utility(c, sh, szeta, n, m, k, nullptr, nullptr, nullptr);
      up[(size_t)m * c.K] = acc;
    }
  }
  inst_sync(c);
  // (B) A_k = argmax_m sum_n u, lowest m on equal sums, -1 when all zero
  // (users shared out over the cluster)
  int ch_local = 0;
  for (int k = cl_first(c); k < c.K; k += cl_stride(c)) {
    int best = -1;
    float b1 = 0.f, b2 = 0.f;
    for (int m = 0; m < c.M; m++) {
      float U = 0.f;
      for (int ch = 0; ch < nch * c.csize; ch++) U += c.Upart[((size_t)ch * c.M + m) * c.K + k];
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
  inst_sync(c);
  // (C) the candidate of every (n, k) on its chosen RRH
  // (users with A_k = -1 have no candidate, except streaming users, whose
  // candidate on Again_k gives the start power if the fix-up places them)
  for (int t = c.n0 * c.K + threadIdx.x; t < c.n1 * c.K; t += kThreads) {
    const int n = t / c.K, k = t - n * c.K;
    const int m = c.Anew[k] >= 0 ? c.Anew[k] : (k >= c.Ke ? c.Again[k] : -1);
    if (m < 0) {
      c.cu[t] = 0.f;
      c.cp[t] = 0.f;
      c.cX[t] = 0.f;
      c.ckey[t] = 1.f;
      continue;
    }
    float ps, X, key;
    c.cu[t] = cand_utility(c, sh, szeta, n, m, k, &ps, &X, &key);
    c.cp[t] = ps;
    c.cX[t] = X;
    c.ckey[t] = key;
  }
  __syncthreads();
  // (D) admission per (n, m) into Snew
  for (int nm = c.n0 * c.M + threadIdx.x; nm < c.n1 * c.M; nm += kThreads) admit(c, nm / c.M, nm % c.M, tie_eps, mm, nt);
  __syncthreads();
  // (E) every streaming user served (synchronises the cluster)
  if (c.Ks > 0) fixup_streaming(c, sh, tie_eps, mm, nt);
  // (F) the new state from Snew
  for (int nm = c.n0 * c.M + threadIdx.x; nm < c.n1 * c.M; nm += kThreads)
    if (apply_selection(c, sh, nm / c.M, nm % c.M)) ch_local = 1;
  inst_sync(c);  // every CTA has read A
  for (int k = cl_first(c); k < c.K; k += cl_stride(c)) c.A[k] = c.Anew[k];
  __syncthreads();
  build_slab(c);
  // fold decision margins and the change flag (the reductions synchronise the cluster)
  const float bm = cl_min(mm, sh, c);
  const int bt = cl_isum(nt, sh, c);
  const int anych = cl_isum(ch_local, sh, c);
  if (threadIdx.x == 0) {
    sh.min_margin = fminf(sh.min_margin, bm);
    sh.n_ties += bt;
  }
  __syncthreads();
  return anych > 0;
}

// The start point written by hcran_set_state (A, S, p, alpha, beta, xi',
// zeta', zeta_sic' in the workspace): Again, the slab and the FP32 copy of
// zeta' derived from it, as initial_state derives them for p^0.  Sec. III
// carries the point p^{i-1} and its multipliers into iteration i; a solve
// that starts here continues a solve stopped after iteration i - 1.
// Returns the number of non-finite or negative gains this thread read.
__device__ int resume_state(const Ctx &c, float *szeta) {
  int bad = 0;
  for (int k = cl_first(c); k < c.K; k += cl_stride(c)) {  // FP64 sums in subcarrier order
    int best = 0;
    double bv = -1.0;
    for (int m = 0; m < c.M; m++) {
      double t = 0.0;
      for (int n = 0; n < c.N; n++) {
        const float g = gain(c, n, m, k);
        bad += !(g >= 0.f && g < INFINITY);
        t += (double)g;
      }
      if (t > bv) {
        bv = t;
        best = m;
      }
    }
    c.Again[k] = best;
  }
  for (int e = c.n0 * c.Up + threadIdx.x; e < c.n1 * c.Up; e += kThreads) c.plin[e] = c.p[e];
  for (int t = c.n0 * c.NPp + threadIdx.x; t < c.n1 * c.NPp; t += kThreads) c.zsic_next[t] = c.zsic[t];
  for (int k = threadIdx.x; k < c.Ks; k += kThreads) szeta[k] = (float)c.zeta[k];
  inst_sync(c);
  build_slab(c);
  return bad;
}

// p^0: A_k = Again_k = argmax_m sum_n Gamma, the l strongest users of m on every
// subcarrier (already in SIC order), p = mask / l; xi' = 0, zeta' = 1.
// Returns the number of non-finite or negative gains this thread read.
__device__ int initial_state(const Ctx &c, float *szeta) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int bad = 0;
  for (int e = c.n0 * c.Up + threadIdx.x; e < c.n1 * c.Up; e += kThreads) {
    c.S[e] = -1;
    c.p[e] = 0.f;
    c.plin[e] = 0.f;
    c.alpha[e] = 1.f;
    c.beta[e] = 0.f;
  }
  for (int k = cl_first(c); k < c.K; k += cl_stride(c)) {  // FP64 sums in subcarrier order
    int best = 0;
    double bv = -1.0;
    for (int m = 0; m < c.M; m++) {
      double t = 0.0;
      for (int n = 0; n < c.N; n++) {
        const float g = gain(c, n, m, k);
        bad += !(g >= 0.f && g < INFINITY);
        t += (double)g;
      }
      if (t > bv) {
        bv = t;
        best = m;
      }
    }
    c.A[k] = best;
    c.Again[k] = best;
  }
  inst_sync(c);
  for (int nm = c.n0 * c.M + warp; nm < c.n1 * c.M; nm += kWarps) {
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
      if (bk < 0) break;
      if (lane == 0) {
        const int e = n * c.Up + m * c.l + s;
        c.S[e] = bk;
        c.p[e] = p0;
        c.plin[e] = p0;
      }
      pg = bg;
      pk = bk;
    }
  }
  if (c.crank == 0) {
    for (int m = threadIdx.x; m < c.M; m += kThreads) c.xi[m] = 0.0;
    for (int k = threadIdx.x; k < c.Ks; k += kThreads) c.zeta[k] = 1.0;
  }
  for (int k = threadIdx.x; k < c.Ks; k += kThreads) szeta[k] = 1.f;
  for (int t = c.n0 * c.NPp + threadIdx.x; t < c.n1 * c.NPp; t += kThreads) {
    c.zsic[t] = 0.0;
    c.zsic_next[t] = 0.0;
  }
  __syncthreads();
  build_slab(c);
  return bad;
}

}  // namespace hcran
