// hcran_dev_common.cuh -- device-side context, shared-memory views, reductions
// and the bulk-copy / mbarrier primitives used by the solver (internal).
#pragma once
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "hcran_layout.h"

namespace hcran {

#define LN2F 0.69314718f
#define LN2D 0.69314718055994530942

constexpr float kPFloorRel = 1e-9f;
constexpr float kGammaFloor = 1e-12f;
constexpr float kInvLn2 = 1.44269504f;
constexpr double kZetaAsumMin = 0.05;
constexpr double kZetaMin = 1e-6, kZetaMax = 1e6;
constexpr float kLog2ZetaMin = -19.9315686f, kLog2ZetaMax = 19.9315686f;  // log2 of the bounds
constexpr int kSpinLimit = 1 << 22;  // default bound on every mbarrier wait (tries)
constexpr int kStatusTimeout = 16;   // per-instance status bit: a bounded wait gave up

// dynamic shared memory of the solver kernel (one declaration for every
// device function, so that pointers into it stay in the shared state space)
extern __shared__ __align__(16) float hcran_dyn[];

struct Ctx {
  int M, N, K, Ks, Ke, l, U, Up, NPp, npair, nchunk;
  int crank, csize;  // rank of this CTA in the cluster that solves the instance, cluster size
  int n0, n1;        // subcarriers [n0, n1) belong to this CTA
  int start;         // InstDesc::start
  const float *G;  // Gamma[n][m][k]
  const double *pmax, *eta, *mask, *Psi, *w;
  double *xi, *zeta, *zsic, *zsic_next;
  float *p, *plin, *pstart, *alpha, *beta, *pi, *gam, *X, *Aden, *Bnum, *Cnum, *slab, *SICp, *SICm,
      *Ptot, *cu, *cp, *cX, *ckey, *Upart, *wf, *gown, *ginv, *wslot;
  int *A, *Anew, *S, *uslot;
  int *Snew;   // [N][Up] selection being built, in SIC order
  int *Again;  // [K] argmax_m sum_n Gamma_{m,k}
  int *srv;    // [csize][Ks] streaming user served on this CTA's subcarriers
  // the previous Dinkelbach iterate (kept when Algorithm 1 ends below it)
  int *A_prev, *S_prev;
  float *p_prev, *alpha_prev, *beta_prev;
  double *xi_prev, *zeta_prev, *zsic_prev;
  float sigma;
  double Pconst;
  const double *Tdel;  // [Ks] delay targets (warm-start features)
  int64_t s_off;       // first warm-start row of the instance
  const float *wout;   // warm-start network outputs (warm mode)
  void *feat;          // warm-start features (features mode)
};

struct Shared {
  float maskf[kMaxM], invmask[kMaxM], floorf[kMaxM], qeta[kMaxM], xif[kMaxM], fac[kMaxM],
      sicscale[kMaxM];
  unsigned char slot_m[kMaxU], slot_s[kMaxU];  // RRH and SIC rank of slot u
  int pio_chunks;                              // lanes per slab row in the price sums
  unsigned char pio_j[32], pio_ch[32];         // lane -> (row, chunk)
  unsigned char item_m[kMaxItems], item_a[kMaxItems], item_b[kMaxItems];  // pair item -> RRH, slots
  double redd[kWarps];
  float redf[kWarps];
  int redi[kWarps];
  unsigned long long bar[kWarps][2];   // per-warp (or per-team) mbarriers of the two staging buffers: filled
  unsigned long long ebar[kWarps][2];  // per-team mbarriers of the two staging buffers: released (team sweeps
                                       // with a producer warp)
  unsigned eph;                        // parity of the next phase of each ebar the producer waits for
  long long cyc[8];  // SM clock cycles per phase of the current instance (thread 0)
  double cxd;        // cluster reductions: this CTA's value, read by the peers
  float cxf;
  int cxi;
  double vpart[kMaxM], vtot[kMaxM];  // per-RRH vectors summed over the cluster
  int inst;
  int abort;
  long long spin_limit;          // tries of a bounded mbarrier wait (Tol::spin_limit or the default)
  unsigned long long stall_bar;  // initialised once, never arrived at: a wait on it can only give up
  float min_margin;
  int n_ties;
};

// One subcarrier's inputs: in a shared staging buffer or straight in global memory.
struct SubView {
  const double *z;    // [NPp] SIC multipliers the step starts from
  const float *slab;  // [M][Up] gains from every RRH, own-RRH entry of each slot zeroed
  const int *k;       // [Up] user per slot, -1 = empty
  const float *p, *A, *B, *C, *alpha, *beta, *plin, *gown, *ginv, *w;  // [Up]
};

// per-warp working buffers (dynamic shared memory)
struct WarpBuf {
  float *p, *pi, *X;               // [Upmax] per slot of the current subcarrier
  int *k;                          // [Upmax]
  float *Pt, *pio, *Sp, *Sm, *wp;  // [Mmax]
  float *zs;                       // [Mmax * NPmax] nonzero SIC multipliers (compact)
  int *zl;                         // [Mmax * NPmax] their pair items
  float *part;                     // [32] per-lane partial sums
  float *wr, *wa;                  // [KSmax] streaming rate / alpha partials
  float *stage0, *stage1;          // staging buffers (staged mode)
};

__device__ __forceinline__ WarpBuf warp_buf(float *dyn, const KDims &kd, int warp) {
  float *b = dyn + dyn_head_floats(kd) + (size_t)warp * warp_stride(kd);
  WarpBuf w;
  if (kd.staged) {  // staging buffers first: 16-byte aligned
    w.stage0 = b;
    w.stage1 = b + stage_buf_floats(kd);
    b += 2 * stage_buf_floats(kd);
  } else {
    w.stage0 = w.stage1 = nullptr;
  }
  w.p = b; b += kd.Upmax;
  w.pi = b; b += kd.Upmax;
  w.X = b; b += kd.Upmax;
  w.k = reinterpret_cast<int *>(b); b += kd.Upmax;
  w.Pt = b; b += kd.Mmax;
  w.pio = b; b += kd.Mmax;
  w.Sp = b; b += kd.Mmax;
  w.Sm = b; b += kd.Mmax;
  w.wp = b; b += kd.Mmax;
  b += kd.Mmax;  // spare
  w.zs = b; b += kd.Mmax * (kd.NPmax > 0 ? kd.NPmax : 1);
  w.zl = reinterpret_cast<int *>(b); b += kd.Mmax * (kd.NPmax > 0 ? kd.NPmax : 1);
  w.part = b; b += 32;
  w.wr = b; b += (kd.KSmax > 0 ? kd.KSmax : 1);
  w.wa = b;
  return w;
}

// view of staging buffer `buf` laid out as stage_buf_floats describes
__device__ __forceinline__ SubView staged_view(const float *buf, const KDims &kd, int M, int Up) {
  SubView v;
  v.z = reinterpret_cast<const double *>(buf);
  const float *f = buf + 2 * kd.NPPmax;
  v.slab = f; f += kd.Mmax * kd.Upmax;
  v.k = reinterpret_cast<const int *>(f); f += kd.Upmax;
  v.p = f; f += kd.Upmax;
  v.A = f; f += kd.Upmax;
  v.B = f; f += kd.Upmax;
  v.C = f; f += kd.Upmax;
  v.alpha = f; f += kd.Upmax;
  v.beta = f; f += kd.Upmax;
  v.plin = f; f += kd.Upmax;
  v.gown = f; f += kd.Upmax;
  v.ginv = f; f += kd.Upmax;
  v.w = f;
  (void)M;
  (void)Up;
  return v;
}

// view of subcarrier n in global memory
__device__ __forceinline__ SubView global_view(const Ctx &c, int n, const double *zsrc) {
  SubView v;
  const size_t o = (size_t)n * c.Up;
  v.z = zsrc + (size_t)n * c.NPp;
  v.slab = c.slab + (size_t)n * c.M * c.Up;
  v.k = c.S + o;
  v.p = c.p + o;
  v.A = c.Aden + o;
  v.B = c.Bnum + o;
  v.C = c.Cnum + o;
  v.alpha = c.alpha + o;
  v.beta = c.beta + o;
  v.plin = c.plin + o;
  v.gown = c.gown + o;
  v.ginv = c.ginv + o;
  v.w = c.wslot + o;
  return v;
}

// ------------------------------------------------------------------ bulk copy + mbarrier (PTX)

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// order this thread's earlier generic-proxy accesses before later bulk copies
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
// one-dimensional bulk copy global -> shared (16-byte aligned, size % 16 == 0)
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         unsigned long long *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait; returns false when the limit was reached
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, uint32_t parity, long long limit) {
  for (long long i = 0; i < limit; i++)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// FP32 reciprocal of the fast division (max 2 ulp); every divisor is a
// positive normal number in the solver's ranges
__device__ __forceinline__ float fast_rcp(float x) { return __fdividef(1.f, x); }

// ------------------------------------------------------------------ reductions

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
__device__ inline double block_sum(double v, Shared &sh) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  v = warp_sum(v);
  if (lane == 0) sh.redd[warp] = v;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < kWarps; i++) t += sh.redd[i];
  __syncthreads();
  return t;
}
__device__ inline float block_max(float v, Shared &sh) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  v = warp_max(v);
  if (lane == 0) sh.redf[warp] = v;
  __syncthreads();
  float t = sh.redf[0];
  for (int i = 1; i < kWarps; i++) t = fmaxf(t, sh.redf[i]);
  __syncthreads();
  return t;
}
__device__ inline float block_min(float v, Shared &sh) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  v = warp_min(v);
  if (lane == 0) sh.redf[warp] = v;
  __syncthreads();
  float t = sh.redf[0];
  for (int i = 1; i < kWarps; i++) t = fminf(t, sh.redf[i]);
  __syncthreads();
  return t;
}
__device__ inline int block_isum(int v, Shared &sh) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  v = warp_isum(v);
  if (lane == 0) sh.redi[warp] = v;
  __syncthreads();
  int t = 0;
  for (int i = 0; i < kWarps; i++) t += sh.redi[i];
  __syncthreads();
  return t;
}

// ------------------------------------------------------------------ cluster of CTAs
//
// An instance is solved by a cluster of csize CTAs (csize = 1: one CTA); CTA r
// owns subcarriers [n0, n1).  Sums over subcarriers are formed per CTA, then
// combined in rank order through distributed shared memory, so every CTA of
// the cluster gets bit-identical totals and takes the same decisions.

// barrier over the CTAs that solve the instance; orders their global and
// shared memory accesses (release / acquire at cluster scope)
__device__ __forceinline__ void inst_sync(const Ctx &c) {
  if (c.csize > 1) cooperative_groups::this_cluster().sync();
  else __syncthreads();
}
// split cluster barrier: every thread of every CTA arrives, then waits
__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
template <typename T>
__device__ __forceinline__ T *peer(T *p, int rank) {
  return cooperative_groups::this_cluster().map_shared_rank(p, rank);
}

__device__ inline double cl_sum(double v, Shared &sh, const Ctx &c) {
  v = block_sum(v, sh);
  if (c.csize == 1) return v;
  if (threadIdx.x == 0) sh.cxd = v;
  inst_sync(c);
  double t = 0.0;
  for (int r = 0; r < c.csize; r++) t += *peer(&sh.cxd, r);
  inst_sync(c);
  return t;
}
__device__ inline float cl_max(float v, Shared &sh, const Ctx &c) {
  v = block_max(v, sh);
  if (c.csize == 1) return v;
  if (threadIdx.x == 0) sh.cxf = v;
  inst_sync(c);
  float t = *peer(&sh.cxf, 0);
  for (int r = 1; r < c.csize; r++) t = fmaxf(t, *peer(&sh.cxf, r));
  inst_sync(c);
  return t;
}
__device__ inline float cl_min(float v, Shared &sh, const Ctx &c) {
  v = block_min(v, sh);
  if (c.csize == 1) return v;
  if (threadIdx.x == 0) sh.cxf = v;
  inst_sync(c);
  float t = *peer(&sh.cxf, 0);
  for (int r = 1; r < c.csize; r++) t = fminf(t, *peer(&sh.cxf, r));
  inst_sync(c);
  return t;
}
__device__ inline int cl_isum(int v, Shared &sh, const Ctx &c) {
  v = block_isum(v, sh);
  if (c.csize == 1) return v;
  if (threadIdx.x == 0) sh.cxi = v;
  inst_sync(c);
  int t = 0;
  for (int r = 0; r < c.csize; r++) t += *peer(&sh.cxi, r);
  inst_sync(c);
  return t;
}
// sh.vtot[i] = sum over the cluster of sh.vpart[i], i < n (each CTA has
// filled its sh.vpart; the call synchronises before and after)
__device__ inline void cl_vsum(Shared &sh, const Ctx &c, int n) {
  inst_sync(c);
  for (int i = threadIdx.x; i < n; i += kThreads) {
    double t = 0.0;
    for (int r = 0; r < c.csize; r++) t += c.csize == 1 ? sh.vpart[i] : peer(sh.vpart, r)[i];
    sh.vtot[i] = t;
  }
  inst_sync(c);
}
// work items [0, count) shared out over the cluster: first index and stride
__device__ __forceinline__ int cl_first(const Ctx &c) { return c.crank * kThreads + (int)threadIdx.x; }
__device__ __forceinline__ int cl_stride(const Ctx &c) { return c.csize * kThreads; }

// ------------------------------------------------------------------ model helpers

__device__ __forceinline__ float gain(const Ctx &c, int n, int m, int k) {
  return __ldg(c.G + ((size_t)n * c.M + m) * c.K + k);
}
// slab[n][j][u] = Gamma_{j, user in slot u}^{(n)}
__device__ __forceinline__ float sgain(const Ctx &c, int n, int j, int u) {
  return c.slab[((size_t)n * c.M + j) * c.Up + u];
}
// SIC order on (m,n): user a decoded after (is stronger than) user b
__device__ __forceinline__ bool stronger(float ga, int a, float gb, int b) {
  return ga > gb || (ga == gb && a < b);
}
__device__ __forceinline__ float weight_c(const Ctx &c, const float *szeta, int m, int k) {
  const float w = c.wf[m * c.K + k];
  return k >= c.Ke ? szeta[k - c.Ke] * w : w;
}
__device__ __forceinline__ void track(float margin, float eps, float &mm, int &nt) {
  mm = fminf(mm, margin);
  if (margin < eps) nt++;
}

}  // namespace hcran
