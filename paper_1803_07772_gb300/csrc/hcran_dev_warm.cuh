// hcran_dev_warm.cuh -- learned warm start (internal): the per-link features
// the network reads, and the initial point the solver takes from its outputs.
//
// Rows: one per slot of the initial selection (the cold p^0 rule: A_k =
// argmax_m sum_n Gamma, the l strongest users of A_k's RRH per subcarrier),
// row s_off + n * Up + u of the instance.  Features of a selected slot (user
// k, RRH m = u / l, subcarrier n), in the first four of 16 BF16 columns:
//   f0 = (log10 Gamma_{m,k,n} + 11) / 3      (gains span about 1e-17 .. 1e-5)
//   f1 = rank of Gamma_{m,k,n} among the K users on (m, n) / K
//   f2 = 1 for a streaming user, 0 for an elastic one
//   f3 = delay target T_k / 0.1 s (0 for an elastic user)
// Empty and padding slots get zeros.  Network outputs of a row (FP32):
//   y0 = log(p / mask_m) -> p^0 = clip(mask_m e^y0, 1e-9 mask_m, mask_m)
//   y1 -> xi'_m = (ln2 mask_m)^-1 * max(mean over m's slots of e^y1 - 1e-3, 0)
//   y2 -> zeta'_k = clip(mean over k's slots of e^y2, 1e-6, 1e6) (streaming)
// after which the C12 projection makes p^0 feasible.
#pragma once
#include <cuda_bf16.h>

#include "hcran_dev_select.cuh"

namespace hcran {

constexpr float kWarmXiEps = 1e-3f;  // offset of the xi' encoding (xi' = 0 is reachable)

__device__ void warm_features(const Ctx &c) {
  __nv_bfloat16 *F = static_cast<__nv_bfloat16 *>(c.feat);
  for (int e = c.n0 * c.Up + threadIdx.x; e < c.n1 * c.Up; e += kThreads) {
    const int n = e / c.Up, u = e - n * c.Up;
    const int k = u < c.U ? c.S[e] : -1;
    float f[4] = {0.f, 0.f, 0.f, 0.f};
    if (k >= 0) {
      const int m = u / c.l;
      const float g = gain(c, n, m, k);
      int stronger_users = 0;
      for (int j = 0; j < c.K; j++) stronger_users += gain(c, n, m, j) > g;
      f[0] = (log10f(fmaxf(g, 1e-30f)) + 11.f) * (1.f / 3.f);
      f[1] = (float)stronger_users / (float)c.K;
      f[2] = k >= c.Ke ? 1.f : 0.f;
      f[3] = k >= c.Ke ? (float)(c.Tdel[k - c.Ke] / 0.1) : 0.f;
    }
    __nv_bfloat162 h01 = __floats2bfloat162_rn(f[0], f[1]), h23 = __floats2bfloat162_rn(f[2], f[3]);
    uint4 lo = make_uint4(*reinterpret_cast<uint32_t *>(&h01), *reinterpret_cast<uint32_t *>(&h23), 0u, 0u);
    uint4 *row = reinterpret_cast<uint4 *>(F + (size_t)(c.s_off + e) * 16);
    row[0] = lo;
    row[1] = make_uint4(0u, 0u, 0u, 0u);
  }
}

// p^0 and the multipliers from the network outputs (cluster-wide means)
__device__ void warm_apply(const Ctx &c, Shared &sh, float *szeta) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float *Y = c.wout;
  for (int e = c.n0 * c.Up + threadIdx.x; e < c.n1 * c.Up; e += kThreads) {
    if (c.S[e] < 0) continue;
    const int m = (e % c.Up) / c.l;
    const float mk = sh.maskf[m];
    const float p = fminf(fmaxf(mk * expf(Y[(size_t)(c.s_off + e) * 16]), sh.floorf[m]), mk);
    c.p[e] = p;
    c.plin[e] = p;
  }
  // xi'_m: sum and count of e^y1 over the slots of RRH m
  for (int pass = 0; pass < 2; pass++) {
    for (int m = warp; m < c.M; m += kWarps) {
      double t = 0.0;
      for (int n = c.n0 + lane; n < c.n1; n += 32)
        for (int s = 0; s < c.l; s++) {
          const int e = n * c.Up + m * c.l + s;
          if (c.S[e] >= 0) t += pass == 0 ? (double)expf(Y[(size_t)(c.s_off + e) * 16 + 1]) : 1.0;
        }
      t = warp_sum(t);
      if (lane == 0) sh.vpart[m] = t;
    }
    cl_vsum(sh, c, c.M);
    for (int m = threadIdx.x; m < c.M; m += kThreads) {
      if (pass == 0) {
        sh.fac[m] = (float)sh.vtot[m];  // sum, kept until the counts arrive
      } else if (c.crank == 0) {
        const double cnt = sh.vtot[m];
        const double mean = cnt > 0.0 ? (double)sh.fac[m] / cnt : 0.0;
        c.xi[m] = fmax(mean - (double)kWarmXiEps, 0.0) / (LN2D * c.mask[m]);
      }
    }
    __syncthreads();
  }
  // zeta'_k: mean of e^y2 over the slots of streaming user k, in groups of kMaxM users
  for (int base = 0; base < c.Ks; base += kMaxM) {
    const int cnt = c.Ks - base < kMaxM ? c.Ks - base : kMaxM;
    for (int pass = 0; pass < 2; pass++) {
      for (int i = warp; i < cnt; i += kWarps) {
        const int k = c.Ke + base + i;
        double t = 0.0;
        for (int n = c.n0 + lane; n < c.n1; n += 32) {
          const int u = c.uslot[(size_t)k * c.N + n];
          if (u >= 0) t += pass == 0 ? (double)expf(Y[(size_t)(c.s_off + n * c.Up + u) * 16 + 2]) : 1.0;
        }
        t = warp_sum(t);
        if (lane == 0) sh.vpart[i] = t;
      }
      cl_vsum(sh, c, cnt);
      for (int i = threadIdx.x; i < cnt; i += kThreads) {
        if (pass == 0) {
          sh.fac[i] = (float)sh.vtot[i];
        } else {
          const double n_ = sh.vtot[i];
          const double z = n_ > 0.0 ? fmin(fmax((double)sh.fac[i] / n_, kZetaMin), kZetaMax) : 1.0;
          szeta[base + i] = (float)z;
          if (c.crank == 0) c.zeta[base + i] = z;
        }
      }
      __syncthreads();
    }
  }
  project_power(c, sh);  // exact C12 at the warm point (synchronises the cluster)
}

}  // namespace hcran
