// hcran_kernel.cu -- persistent batched solver for sm_103a.
//
// A thread-block cluster of C CTAs (C = 1 .. 8, 512 threads and 16 warps each)
// solves one instance at a time and pulls the next one from the LPT-ordered
// queue of its launch (largest M*N*K*l first).  CTA r of the cluster owns a
// contiguous range of subcarriers; the CTAs exchange their per-iteration sums
// through distributed shared memory, and no cluster ever waits on another:
//
//   p^0 (gain-based RRH choice, l strongest users, p = mask/l); E^1 = R/P
//   Dinkelbach i (Sec. III):  selection  ->  Algorithm 1  ->  E^{i+1} = R/P;
//     when Algorithm 1 ends below p^{i-1} (F < 0; Lemma 1 has p^{i-1} attain
//     F = 0), p^{i-1} is kept and the loop ends, unless p^{i-1} misses the
//     streaming rates that p^i meets better
//     Algorithm 1 (Sec. IV-A): alpha = 1, beta = 0; SCALE passes, each a
//       dual loop of [interference/SINR/prices -> projected subgradient on
//       xi', zeta', zeta_sic' -> closed-form KKT power of eq. (653)/(683)],
//       then alpha/beta at the new point (eq. scale_approximation)
//
// Precision: FP32 for SINR, prices, powers and residuals; inside a dual loop
// the multipliers accumulate their subgradient steps as (hi, lo) float pairs,
// and between dual loops they are kept in FP64; FP64 for q = R/P, the F(q)
// test and the R and P sums.  Reductions run in a fixed order, so results are
// bit-reproducible run to run.  The pieces live in hcran_dev_*.cuh.
#include "hcran_dev_warm.cuh"

namespace hcran {

// min over streaming users of (r_k - Psi_k) / Psi_k with exact rates (C13)
// from the last link pass, over the cluster (INFINITY without streaming users)
__device__ float rate_slack_min(const Ctx &c, Shared &sh) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float rmin = INFINITY;
  for (int base = 0; base < c.Ks; base += kMaxM) {  // streaming users in groups of kMaxM
    const int cnt = c.Ks - base < kMaxM ? c.Ks - base : kMaxM;
    for (int i = warp; i < cnt; i += kWarps) {
      const int k = c.Ke + base + i;
      const int a = c.A[k];
      float r = 0.f;
      if (a >= 0) {
        const float wk = c.wf[(size_t)a * c.K + k];
        for (int n = c.n0 + lane; n < c.n1; n += 32) {
          const int u = c.uslot[(size_t)k * c.N + n];
          if (u >= 0) r += wk * log1pf(c.gam[n * c.Up + u]) / LN2F;
        }
      }
      r = warp_sum(r);
      if (lane == 0) sh.vpart[i] = r;
    }
    cl_vsum(sh, c, cnt);
    for (int i = threadIdx.x; i < cnt; i += kThreads)
      rmin = fminf(rmin, (float)((sh.vtot[i] - c.Psi[base + i]) / c.Psi[base + i]));
  }
  return block_min(rmin, sh);
}

// copy of the Dinkelbach iterate p^{i-1} (this CTA's subcarriers; A, xi',
// zeta' shared out over the cluster), and its restoration with the slab
__device__ void save_iterate(const Ctx &c) {
  for (int e = c.n0 * c.Up + threadIdx.x; e < c.n1 * c.Up; e += kThreads) {
    c.S_prev[e] = c.S[e];
    c.p_prev[e] = c.p[e];
    c.alpha_prev[e] = c.alpha[e];
    c.beta_prev[e] = c.beta[e];
  }
  for (int t = c.n0 * c.NPp + threadIdx.x; t < c.n1 * c.NPp; t += kThreads) c.zsic_prev[t] = c.zsic[t];
  for (int k = cl_first(c); k < c.K; k += cl_stride(c)) c.A_prev[k] = c.A[k];
  for (int m = cl_first(c); m < c.M; m += cl_stride(c)) c.xi_prev[m] = c.xi[m];
  for (int k = cl_first(c); k < c.Ks; k += cl_stride(c)) c.zeta_prev[k] = c.zeta[k];
  inst_sync(c);
}
__device__ void restore_iterate(const Ctx &c, float *szeta) {
  for (int e = c.n0 * c.Up + threadIdx.x; e < c.n1 * c.Up; e += kThreads) {
    c.S[e] = c.S_prev[e];
    c.p[e] = c.p_prev[e];
    c.plin[e] = c.p_prev[e];
    c.alpha[e] = c.alpha_prev[e];
    c.beta[e] = c.beta_prev[e];
  }
  for (int t = c.n0 * c.NPp + threadIdx.x; t < c.n1 * c.NPp; t += kThreads) c.zsic[t] = c.zsic_prev[t];
  for (int k = cl_first(c); k < c.K; k += cl_stride(c)) c.A[k] = c.A_prev[k];
  for (int m = cl_first(c); m < c.M; m += cl_stride(c)) c.xi[m] = c.xi_prev[m];
  for (int k = cl_first(c); k < c.Ks; k += cl_stride(c)) c.zeta[k] = c.zeta_prev[k];
  inst_sync(c);
  for (int k = threadIdx.x; k < c.Ks; k += kThreads) szeta[k] = (float)c.zeta[k];
  build_slab(c);
}

__device__ void solve_instance(const Ctx &c, Shared &sh, float *dyn, const KDims &kd, const Tol &tol,
                               InstOut *out, int index, unsigned &phase, unsigned &pending) {
  float *szeta = dyn;  // streaming multipliers in FP32, first in dynamic shared memory
  for (int m = threadIdx.x; m < c.M; m += kThreads) {
    sh.maskf[m] = (float)c.mask[m];
    sh.floorf[m] = (float)c.mask[m] * kPFloorRel;
    sh.sicscale[m] = 1.f / (LN2F * (float)c.mask[m]);
    sh.invmask[m] = 1.f / (float)c.mask[m];
  }
  for (int u = threadIdx.x; u < c.U; u += kThreads) {
    sh.slot_m[u] = (unsigned char)(u / c.l);
    sh.slot_s[u] = (unsigned char)(u % c.l);
  }
  for (int it = threadIdx.x; it < c.M * c.npair; it += kThreads) {
    const int m = it / c.npair;
    int r = it - m * c.npair, a = 0;
    while (r >= c.l - 1 - a) {
      r -= c.l - 1 - a;
      a++;
    }
    sh.item_m[it] = (unsigned char)m;
    sh.item_a[it] = (unsigned char)(m * c.l + a);
    sh.item_b[it] = (unsigned char)(m * c.l + a + 1 + r);
  }
  if (threadIdx.x < 32) {
    const int C = c.M <= 32 ? 32 / c.M : 1;
    if (threadIdx.x == 0) sh.pio_chunks = C;
    sh.pio_j[threadIdx.x] = (unsigned char)(threadIdx.x % c.M);
    sh.pio_ch[threadIdx.x] = (unsigned char)(threadIdx.x / c.M);
  }
  for (int t = cl_first(c); t < c.M * c.K; t += cl_stride(c)) c.wf[t] = (float)c.w[t];
  if (threadIdx.x == 0) {
    for (int i = 0; i < 8; i++) sh.cyc[i] = 0;
    sh.min_margin = 1.f;
    sh.n_ties = 0;
    sh.abort = 0;
  }
  __syncthreads();
  // test of the failure path (Tol::stall_instance): a bounded wait on a
  // barrier that nothing completes, with no copy in flight, gives up after
  // spin_limit tries; every CTA of the cluster waits and gives up alike, so
  // they skip the solve together and report HCRAN_ST_TIMEOUT
  if (index == tol.stall_instance && threadIdx.x == 0 && !mbar_wait(&sh.stall_bar, 0u, sh.spin_limit))
    sh.abort = 1;
  long long *cyc = sh.cyc;  // written by thread 0 only
  const long long t_begin = clock64();
  // the set-up reads every gain once: a non-finite or negative one makes the
  // instance's results invalid (HCRAN_ST_NUMERIC), decided by the whole cluster
  const int bad_gains = cl_isum(tol.mode == kModeCold && c.start == 1 ? resume_state(c, szeta)
                                                                       : initial_state(c, szeta), sh, c);
  if (tol.mode == kModeFeatures) {  // initial selection and the warm-start features only
    warm_features(c);
    inst_sync(c);
    return;
  }
  if (tol.mode == kModeWarm) warm_apply(c, sh, szeta);
  double R, P;
  link_all<kLinkOnly>(c, sh, dyn, kd, szeta, 0.f, phase, pending);
  exact_R_P(c, sh, R, P);
  double q = tol.q_init > 0.0 ? tol.q_init : R / P;
  int it_d = 0, it_s = 0, it_v = 0, status = bad_gains ? 8 : 1;  // not converged until the stop test fires
  const int Imax = tol.max_dinkelbach > 0 ? tol.max_dinkelbach : 1;
  const int Smax = tol.max_scale > 0 ? tol.max_scale : 1;
  float slack_prev = rate_slack_min(c, sh);
  double ee_best = R / P;
  for (int i = 0; i < Imax && !sh.abort && !bad_gains; i++) {
    save_iterate(c);  // p^{i-1}, kept if Algorithm 1 ends below it
    const double q_prev = q;
    for (int m = threadIdx.x; m < c.M; m += kThreads) {
      sh.qeta[m] = (float)(q * c.eta[m]);
      sh.xif[m] = (float)c.xi[m];
    }
    // the streaming multipliers as stored between dual loops, so that a solve
    // resumed from an exported state takes the same steps
    for (int k = threadIdx.x; k < c.Ks; k += kThreads) szeta[k] = (float)c.zeta[k];
    __syncthreads();
    const long long ta = clock64();
    selection(c, sh, dyn, kd, szeta, tol.tie_eps, phase, pending);
    if (threadIdx.x == 0) cyc[0] += clock64() - ta;
    // Algorithm 1 at E^i = q (alpha = 1, beta = 0 written by the selection)
    for (int s = 0; s < Smax && !sh.abort; s++) {
      for (int e = c.n0 * c.Up + threadIdx.x; e < c.n1 * c.Up; e += kThreads) {
        c.pstart[e] = c.p[e];
        c.plin[e] = c.p[e];
      }
      __syncthreads();
      it_v += kd.resident ? dual_loop_res(c, sh, dyn, kd, szeta, tol, cyc, phase, pending)
                          : dual_loop(c, sh, dyn, kd, szeta, tol, cyc, phase, pending);
      const long long t5 = clock64();
      scale_update(c);
      it_s++;
      float dm = 0.f;
      for (int e = c.n0 * c.Up + threadIdx.x; e < c.n1 * c.Up; e += kThreads)
        if (c.S[e] >= 0) dm = fmaxf(dm, fabsf(c.p[e] - c.pstart[e]) / sh.maskf[(e % c.Up) / c.l]);
      dm = cl_max(dm, sh, c);
      if (threadIdx.x == 0) cyc[4] += clock64() - t5;
      if (dm < (float)tol.tol_scale) break;
    }
    const long long t6 = clock64();
    project_power(c, sh);
    link_all<kLinkOnly>(c, sh, dyn, kd, szeta, 0.f, phase, pending);
    exact_R_P(c, sh, R, P);
    if (threadIdx.x == 0) cyc[5] += clock64() - t6;
    it_d++;
    if (!isfinite(R) || !isfinite(P) || P <= 0.0) {
      status = 8;
      break;
    }
    const double F = R - q * P, qn = R / P;
    const float slack = rate_slack_min(c, sh);
    if (F < 0.0) {
      // the inner solve ended below p^{i-1}, which attains F = 0 (Lemma 1):
      // keep p^{i-1} and stop, unless p^{i-1} misses the streaming rates that
      // p^i meets better
      if (slack_prev >= -1e-3f || slack_prev >= slack) {
        restore_iterate(c, szeta);
        link_all<kLinkOnly>(c, sh, dyn, kd, szeta, 0.f, phase, pending);
        exact_R_P(c, sh, R, P);
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
    ee_best = fmax(ee_best, qn);
    if (F <= tol.tol_dinkelbach * R) {  // stop test of Sec. III, relative
      status = 0;
      break;
    }
  }
  // slacks (exact rates from the last link pass), summed over the cluster
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int m = warp; m < c.M; m += kWarps) {
    double t = 0.0;
    for (int n = c.n0 + lane; n < c.n1; n += 32) t += (double)c.Ptot[n * c.M + m];
    t = warp_sum(t);
    if (lane == 0) sh.vpart[m] = t;
  }
  cl_vsum(sh, c, c.M);
  float smin = INFINITY;
  for (int m = threadIdx.x; m < c.M; m += kThreads)
    smin = fminf(smin, (float)((c.pmax[m] - sh.vtot[m]) / c.pmax[m]));
  const float slack_power = block_min(smin, sh);
  const float slack_rate = rate_slack_min(c, sh);
  float smax = -INFINITY;
  for (int nm = c.n0 * c.M + threadIdx.x; nm < c.n1 * c.M; nm += kThreads) {
    const int n = nm / c.M, m = nm - n * c.M;
    const int base = n * c.Up + m * c.l;
    for (int a = 0; a < c.l; a++) {
      if (c.S[base + a] < 0) break;
      for (int b = a + 1; b < c.l; b++) {
        if (c.S[base + b] < 0) break;
        const float ra = (c.sigma + c.X[base + a]) * c.ginv[base + a];
        const float rb = (c.sigma + c.X[base + b]) * c.ginv[base + b];
        smax = fmaxf(smax, (ra - rb) / sh.maskf[m]);
      }
    }
  }
  const float slack_sic = cl_max(smax, sh, c);
  if (threadIdx.x == 0 && c.crank == 0) {
    if (c.Ks > 0 && slack_rate < -1e-3f) status |= 2;
    if (R / P < ee_best * (1.0 - 1e-9)) status |= 4;  // an earlier iterate was more efficient
    if (sh.abort) status |= kStatusTimeout;
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
    cyc[6] = clock64() - t_begin;
    for (int i = 0; i < 8; i++) out->cycles[i] = cyc[i];
  }
  __syncthreads();
}

__device__ void bind(Ctx &c, const InstDesc &d, const float *gains, double *darena, float *farena,
                     int *iarena) {
  c.M = d.M; c.N = d.N; c.K = d.K; c.Ks = d.Ks; c.Ke = d.K - d.Ks; c.l = d.l;
  c.U = d.U; c.Up = slot_stride(d.M, d.l); c.NPp = pair_stride(d.M, d.l);
  c.npair = d.npair; c.nchunk = d.nchunk; c.start = d.start;
  c.G = gains + d.g_off;
  c.sigma = (float)d.sigma;
  c.Pconst = d.Pconst;
  const DLayout dl = dlayout(d.M, d.N, d.K, d.Ks, d.l);
  double *db = darena + d.d_off;
  c.pmax = db + dl.pmax; c.eta = db + dl.eta; c.mask = db + dl.mask; c.Psi = db + dl.Psi;
  c.Tdel = db + dl.Tdel;
  c.s_off = d.s_off;
  c.w = db + dl.w; c.xi = db + dl.xi; c.zeta = db + dl.zeta; c.zsic = db + dl.zsic;
  c.zsic_next = db + dl.zsic_next;
  c.xi_prev = db + dl.xi_prev; c.zeta_prev = db + dl.zeta_prev; c.zsic_prev = db + dl.zsic_prev;
  const FLayout fl = flayout(d.M, d.N, d.K, d.l, nchunk_cap(d.N, d.K));
  float *fb = farena + d.f_off;
  c.p = fb + fl.p; c.plin = fb + fl.plin; c.pstart = fb + fl.pstart; c.alpha = fb + fl.alpha;
  c.beta = fb + fl.beta; c.pi = fb + fl.pi; c.gam = fb + fl.gam; c.X = fb + fl.X;
  c.Aden = fb + fl.Aden; c.Bnum = fb + fl.Bnum; c.Cnum = fb + fl.Cnum;
  c.slab = fb + fl.slab; c.SICp = fb + fl.SICp; c.SICm = fb + fl.SICm; c.Ptot = fb + fl.Ptot;
  c.cu = fb + fl.cu; c.cp = fb + fl.cp; c.cX = fb + fl.cX; c.ckey = fb + fl.ckey;
  c.Upart = fb + fl.Upart;
  c.wf = fb + fl.wf;
  c.gown = fb + fl.gown;
  c.ginv = fb + fl.ginv;
  c.wslot = fb + fl.wslot;
  c.p_prev = fb + fl.p_prev; c.alpha_prev = fb + fl.alpha_prev; c.beta_prev = fb + fl.beta_prev;
  const ILayout il = ilayout(d.M, d.N, d.K, d.Ks, d.l);
  int *ib = iarena + d.i_off;
  c.A = ib + il.A; c.Anew = ib + il.Anew; c.S = ib + il.S; c.uslot = ib + il.uslot;
  c.Snew = ib + il.Snew; c.Again = ib + il.Again; c.srv = ib + il.srv;
  c.A_prev = ib + il.A_prev; c.S_prev = ib + il.S_prev;
}

__global__ void __launch_bounds__(kThreads, 1)
    solve_kernel(const InstDesc *__restrict__ descs, const int *__restrict__ order, int n_inst,
                 const float *__restrict__ gains, double *darena, float *farena, int *iarena,
                 InstOut *outs, Tol tol, KDims kd, int *counter, WarmIO wio) {
  __shared__ Shared sh;
  __shared__ Ctx sc;
  float *dyn = hcran_dyn;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // a launch with clusters solves each instance on one cluster; CTA r of the
  // cluster owns a contiguous share of the subcarriers
  const int csize = (int)cooperative_groups::this_cluster().num_blocks();
  const int crank = (int)cooperative_groups::this_cluster().block_rank();
  if (lane == 0) {
    mbar_init(&sh.bar[warp][0], 1);
    mbar_init(&sh.bar[warp][1], 1);
    mbar_init(&sh.ebar[warp][0], 1);
    mbar_init(&sh.ebar[warp][1], 1);
  }
  if (threadIdx.x == 0) {
    sh.eph = 0u;
    mbar_init(&sh.stall_bar, 1);
    sh.spin_limit = tol.spin_limit > 0 ? tol.spin_limit : (long long)kSpinLimit;
  }
  fence_mbar_init();
  __syncthreads();
  unsigned phase = 0, pending = 0;  // per-warp mbarrier parity and copies in flight
  for (;;) {
    if (crank == 0 && threadIdx.x == 0) sh.inst = atomicAdd(counter, 1);
    if (csize > 1) cooperative_groups::this_cluster().sync();
    else __syncthreads();
    const int w = csize > 1 ? *peer(&sh.inst, 0) : sh.inst;
    // nobody reads the leader's slot after this barrier until it is rewritten
    if (csize > 1) cooperative_groups::this_cluster().sync();
    else __syncthreads();
    if (w >= n_inst) break;
    const int b = order[w];
    // the instance context lives in shared memory: every field read is a
    // shared load instead of a local-memory one
    if (threadIdx.x == 0) {
      bind(sc, descs[b], gains, darena, farena, iarena);
      sc.csize = csize;
      sc.crank = crank;
      sc.nchunk = class_nchunk(sc.N, sc.K, csize);  // candidate-utility chunks, a multiple of csize
      sc.wout = wio.out;
      sc.feat = wio.feat;
      sc.n0 = (int)((int64_t)sc.N * crank / csize);
      sc.n1 = (int)((int64_t)sc.N * (crank + 1) / csize);
    }
    __syncthreads();
    solve_instance(sc, sh, dyn, kd, tol, outs + b, b, phase, pending);
  }
  // never leave a bulk copy in flight (bounded; set only after a timed-out wait)
  const int bi = kd.teams > 0 ? team_of(kd, warp) : warp;  // the barriers this thread's copies complete on
  for (int bb = 0; bb < 2; bb++)
    if (pending & (1u << bb)) {
      mbar_wait(&sh.bar[bi][bb], (phase >> bb) & 1u, sh.spin_limit);
    }
}

// One persistent launch over n_inst instances (indices order[0..n_inst)),
// each solved by a cluster of csize CTAs (csize = 1: one CTA).  The grid is
// as many clusters as can be resident at once, capped at n_inst.
cudaError_t launch_solve(const InstDesc *descs, const int *order, int n_inst, const float *gains,
                         double *darena, float *farena, int *iarena, InstOut *outs, const Tol &tol,
                         const KDims &kd, int csize, int *counter, cudaStream_t stream, int *launches,
                         const WarmIO &wio) {
  *launches = 0;
  if (n_inst <= 0) return cudaSuccess;
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (err != cudaSuccess) return err;
  const int smem = (int)dyn_smem_bytes(kd);
  err = cudaFuncSetAttribute(solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (err != cudaSuccess) return err;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  int clusters = 0;
  if (csize > 1) {
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = csize;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3(csize * sms, 1, 1);
    err = cudaOccupancyMaxActiveClusters(&clusters, solve_kernel, &cfg);
    if (err != cudaSuccess) return err;
    if (clusters < 1) return cudaErrorInvalidConfiguration;
  } else {
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, solve_kernel, kThreads, smem);
    if (err != cudaSuccess) return err;
    clusters = sms * (per_sm > 0 ? per_sm : 1);
  }
  if (clusters > n_inst) clusters = n_inst;
  cfg.gridDim = dim3(clusters * csize, 1, 1);
  err = cudaMemsetAsync(counter, 0, sizeof(int), stream);
  if (err != cudaSuccess) return err;
  err = cudaLaunchKernelEx(&cfg, solve_kernel, descs, order, n_inst, gains, darena, farena, iarena, outs,
                           tol, kd, counter, wio);
  if (err != cudaSuccess) return err;
  *launches = 1;
  return cudaGetLastError();
}

}  // namespace hcran
