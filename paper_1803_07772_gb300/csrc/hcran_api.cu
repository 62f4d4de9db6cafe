// hcran_api.cu -- host side of the C ABI declared in include/hcran.h:
// argument checking, workspace planning, constant upload, launch, results.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <numeric>
#include <vector>

#include "../../include/hcran.h"
#include "hcran_layout.h"

namespace hcran {
cudaError_t launch_solve(const InstDesc *descs, const int *order, int n_inst, const float *gains,
                         double *darena, float *farena, int *iarena, InstOut *outs, const Tol &tol,
                         const KDims &kd, int csize, int *counter, cudaStream_t stream, int *launches,
                         const WarmIO &wio);
}

using namespace hcran;

// one launch: the instances of a class (cluster size) with the launch's dimensions
struct LaunchClass {
  int csize = 1;
  KDims kd{0, 0, 0, 0, 0, 0, 0, 0};
  int first = 0, count = 0;  // segment of the order array
};

struct hcran_s {
  int32_t n = 0;
  std::vector<InstDesc> descs;
  std::vector<int32_t> order;     // instances grouped by class, LPT within a class
  std::vector<int32_t> cls;       // launch class of every instance
  LaunchClass classes[kNumClasses];
  std::vector<double> dimage;   // full double arena (constants + zeroed multipliers)
  int64_t gain_elems = 0, dtot = 0, ftot = 0, itot = 0;
  int64_t warm_rows = 0;          // rows of the warm-start feature / output arrays
  WsLayout ws{};
  void *last_ws = nullptr;
  cudaStream_t last_stream = nullptr;
  int32_t last_launches = 0;
  std::vector<InstOut> outs_host;
  bool plan_dirty = false;  // descriptors / order changed since they were uploaded
  int64_t spin_limit = 0;        // tries of a bounded device wait (0: the default)
  int32_t stall_instance = -1;   // test of the failure path (hcran_set_wait_limit)
  int32_t stream_teams = 0;      // > 0: the streamed class sweeps with this many teams (hcran_set_schedule)
  // captured launch sequence of hcran_solve_graph and the arguments it was captured for
  cudaGraphExec_t graph = nullptr;
  const void *graph_gains = nullptr, *graph_ws = nullptr;
  hcran_tol graph_tol{};
  // second stream: classes of small clusters run beside those of large ones
  // and fill the SMs that whole clusters leave free
  cudaStream_t side = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  ~hcran_s() {
    if (graph) cudaGraphExecDestroy(graph);
    if (side) cudaStreamDestroy(side);
    if (fork) cudaEventDestroy(fork);
    if (join) cudaEventDestroy(join);
  }
};

// Launch classes from the per-instance classes h->cls: launch dimensions per
// class (an instance that would push its class over the shared-memory limit
// moves on to the next larger cluster), chunk counts, and the launch order
// (classes largest cluster first; longest-processing-time order, largest
// M*N*K*l first, inside a class).  Returns nonzero when the streamed class
// does not fit shared memory either.
static int build_classes(hcran_s *h) {
  const int32_t n = h->n;
  for (;;) {
    bool moved = false;
    for (int k = 0; k < kNumClasses; k++) h->classes[k] = LaunchClass();
    for (int32_t b = 0; b < n; b++) {
      const InstDesc &d = h->descs[b];
      LaunchClass &L = h->classes[h->cls[b]];
      const KDims one = h->cls[b] < kNumClasses - 1
                            ? resident_kdims(d.M, d.l, d.Ks, d.N, class_csize(h->cls[b]))
                            : KDims{slot_stride(d.M, d.l), d.M, d.npair, pair_stride(d.M, d.l), d.Ks, 0, 0, 0};
      if (L.count == 0) L.kd = one;
      else kdims_merge(L.kd, one);
      L.count++;
    }
    for (int k = 0; k < kNumClasses - 1 && !moved; k++) {
      LaunchClass &L = h->classes[k];
      if (L.count == 0 || dyn_smem_bytes(L.kd) <= kMaxDynSmem) continue;
      int worst = -1;  // the instance with the largest resident state of the class
      int64_t wr = -1;
      for (int32_t b = 0; b < n; b++)
        if (h->cls[b] == k) {
          const InstDesc &d = h->descs[b];
          const int64_t r = res_floats(d.M, d.l, d.Ks, (d.N + class_csize(k) - 1) / class_csize(k));
          if (r > wr) {
            wr = r;
            worst = b;
          }
        }
      h->cls[worst] = k == 0 ? kNumClasses - 1 : k - 1;
      moved = true;
    }
    if (!moved) break;
  }
  {  // streamed class: staging when the double buffers fit, else global reads
    LaunchClass &L = h->classes[kNumClasses - 1];
    if (L.count > 0 && plan_kdims(L.kd, int64_t(1) << 40) != 0) return 1;
    if (L.count > 0 && h->stream_teams > 0) {  // team sweeps requested by hcran_set_schedule
      KDims t = L.kd;
      t.resident = 0;
      t.res_floats = 0;
      t.staged = 1;
      t.teams = h->stream_teams;
      if (dyn_smem_bytes(t) > kMaxDynSmem) return 1;
      L.kd = t;
    }
  }
  for (int32_t b = 0; b < n; b++) {
    InstDesc &d = h->descs[b];
    d.nchunk = class_nchunk(d.N, d.K, class_csize(h->cls[b]));
  }
  h->order.resize(n);
  std::iota(h->order.begin(), h->order.end(), 0);
  std::stable_sort(h->order.begin(), h->order.end(), [&](int a, int b) {
    if (h->cls[a] != h->cls[b]) return h->cls[a] < h->cls[b];
    const InstDesc &x = h->descs[a], &y = h->descs[b];
    return int64_t(x.N) * x.M * x.K * x.l > int64_t(y.N) * y.M * y.K * y.l;
  });
  for (int k = 0, first = 0; k < kNumClasses; k++) {
    h->classes[k].csize = class_csize(k);
    h->classes[k].first = first;
    first += h->classes[k].count;
  }
  if (h->graph) {  // the captured launch sequence no longer matches
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
  h->plan_dirty = true;
  return 0;
}

static uint64_t al256(uint64_t x) { return (x + 255) & ~uint64_t(255); }

static bool finite_pos(double x) { return isfinite(x) && x > 0.0; }
static bool finite_nonneg(double x) { return isfinite(x) && x >= 0.0; }

// C9: Psi = Psi_hat / B_n with Psi_hat = lambda zbar / (1 + lambda T - sqrt(1 + lambda^2 T^2)),
// the smaller root of the quadratic in the mean service time (Eq6b-Eq6d).
static double min_rate(double T, double lam, double zbar, double Bn) {
  const double x = lam * T;
  const double den = 1.0 + x - sqrt(1.0 + x * x);
  return lam * zbar / den / Bn;
}

static int check_config(const hcran_config &c) {
  if (c.M < 1 || c.M > kMaxM || c.N < 1 || c.K < 1 || c.Ks < 0 || c.Ks > c.K || c.l < 1 ||
      c.l > kMaxL || c.M * c.l > kMaxU)
    return HCRAN_EINVAL;
  if (int64_t(c.N) * c.M * c.K > (int64_t(1) << 40)) return HCRAN_EINVAL;
  if (!c.pmax || !c.eta || !c.Pc || !c.Pf) return HCRAN_EINVAL;
  if (!finite_pos(c.Bn_hz) || !finite_pos(c.N0_w_per_hz)) return HCRAN_EINVAL;
  for (int m = 0; m < c.M; m++)
    if (!finite_pos(c.pmax[m]) || !finite_pos(c.eta[m]) || !finite_nonneg(c.Pc[m]) ||
        !finite_nonneg(c.Pf[m]))
      return HCRAN_EINVAL;
  if (c.Ks > 0) {
    if (!c.T_s || !c.lambda_pps || !finite_pos(c.zbar_bits)) return HCRAN_EINVAL;
    for (int k = 0; k < c.Ks; k++)
      if (!finite_pos(c.T_s[k]) || !finite_pos(c.lambda_pps[k])) return HCRAN_EINVAL;
  }
  if (c.w)
    for (int64_t t = 0; t < int64_t(c.M) * c.K; t++)
      if (!finite_nonneg(c.w[t])) return HCRAN_EINVAL;
  return HCRAN_OK;
}

extern "C" int hcran_create(hcran_t *out, const hcran_config *cfgs, int32_t n,
                            const int64_t *gain_offsets) {
  if (!out || !cfgs || n < 1) return HCRAN_EINVAL;
  *out = nullptr;
  for (int32_t b = 0; b < n; b++) {
    const int rc = check_config(cfgs[b]);
    if (rc != HCRAN_OK) return rc;
  }
  hcran_s *h = new (std::nothrow) hcran_s();
  if (!h) return HCRAN_ENOMEM;
  try {
    h->n = n;
    h->descs.resize(n);
    int64_t goff = 0, doff = 0, foff = 0, ioff = 0;
    h->cls.resize(n);
    for (int32_t b = 0; b < n; b++) {
      const hcran_config &c = cfgs[b];
      InstDesc &d = h->descs[b];
      memset(&d, 0, sizeof(d));
      d.M = c.M; d.N = c.N; d.K = c.K; d.Ks = c.Ks; d.l = c.l;
      d.U = c.M * c.l;
      d.L = c.N * d.U;
      d.npair = c.l * (c.l - 1) / 2;
      h->cls[b] = pick_class(c.M, c.l, c.Ks, c.N);
      const int64_t cost = int64_t(c.N) * c.M * c.K;
      if (gain_offsets) {
        if (gain_offsets[b] < 0 || (gain_offsets[b] & 3)) { delete h; return HCRAN_EINVAL; }
        d.g_off = gain_offsets[b];
      } else {
        d.g_off = goff;
        goff += al4(cost);
      }
      h->gain_elems = std::max(h->gain_elems, d.g_off + cost);
      d.sigma = c.N0_w_per_hz * c.Bn_hz;
      double pc = 0.0;
      for (int m = 0; m < c.M; m++) pc += c.Pc[m] + c.Pf[m];
      d.Pconst = pc;
    }
    if (build_classes(h) != 0) { delete h; return HCRAN_EINVAL; }
    // arenas (sized for any schedule of the instance)
    doff = foff = ioff = 0;
    int64_t soff = 0;
    for (int32_t b = 0; b < n; b++) {
      const hcran_config &c = cfgs[b];
      InstDesc &d = h->descs[b];
      const DLayout dl = dlayout(c.M, c.N, c.K, c.Ks, c.l);
      const FLayout fl = flayout(c.M, c.N, c.K, c.l, nchunk_cap(c.N, c.K));
      const ILayout il = ilayout(c.M, c.N, c.K, c.Ks, c.l);
      d.d_off = doff; doff += al4(dl.total);
      d.f_off = foff; foff += al4(fl.total);
      d.i_off = ioff; ioff += al4(il.total);
      d.s_off = soff; soff += int64_t(c.N) * slot_stride(c.M, c.l);
    }
    h->warm_rows = soff;
    h->gain_elems = al4(h->gain_elems);
    h->dtot = doff; h->ftot = foff; h->itot = ioff;
    // constants image of the double arena
    h->dimage.assign(doff, 0.0);
    for (int32_t b = 0; b < n; b++) {
      const hcran_config &c = cfgs[b];
      const DLayout dl = dlayout(c.M, c.N, c.K, c.Ks, c.l);
      double *db = h->dimage.data() + h->descs[b].d_off;
      for (int m = 0; m < c.M; m++) {
        db[dl.pmax + m] = c.pmax[m];
        db[dl.eta + m] = c.eta[m];
        db[dl.mask + m] = c.pmax[m] / c.N;   // spectral mask p^mask = pmax / N
      }
      for (int k = 0; k < c.Ks; k++) {
        db[dl.Psi + k] = min_rate(c.T_s[k], c.lambda_pps[k], c.zbar_bits, c.Bn_hz);
        db[dl.Tdel + k] = c.T_s[k];
      }
      for (int64_t t = 0; t < int64_t(c.M) * c.K; t++) db[dl.w + t] = c.w ? c.w[t] : 1.0;
    }
    WsLayout &w = h->ws;
    uint64_t o = 0;
    w.descs = o; o = al256(o + sizeof(InstDesc) * n);
    w.order = o; o = al256(o + sizeof(int32_t) * n);
    w.counter = o; o = al256(o + sizeof(int32_t) * kNumClasses);
    w.outs = o; o = al256(o + sizeof(InstOut) * n);
    w.darena = o; o = al256(o + sizeof(double) * h->dtot);
    w.farena = o; o = al256(o + sizeof(float) * h->ftot);
    w.iarena = o; o = al256(o + sizeof(int32_t) * h->itot);
    w.staging = o; o = al256(o + sizeof(float) * h->gain_elems);
    w.total = o;
    h->outs_host.resize(n);
  } catch (...) {
    delete h;
    return HCRAN_ENOMEM;
  }
  *out = h;
  return HCRAN_OK;
}

extern "C" int hcran_workspace_size(hcran_t h, uint64_t *bytes) {
  if (!h || !bytes) return HCRAN_EINVAL;
  *bytes = h->ws.total;
  return HCRAN_OK;
}

extern "C" int hcran_gain_elems(hcran_t h, int64_t *elems) {
  if (!h || !elems) return HCRAN_EINVAL;
  *elems = h->gain_elems;
  return HCRAN_OK;
}

constexpr int32_t kStatusNumericHost = HCRAN_ST_NUMERIC, kStatusTimeoutHost = HCRAN_ST_TIMEOUT;

static bool ws_ok(void *ws) { return ws && (reinterpret_cast<uintptr_t>(ws) & 255) == 0; }

// descriptors and launch order -> workspace (stream-ordered)
static int upload_plan(hcran_t h, char *ws, cudaStream_t st) {
  if (cudaMemcpyAsync(ws + h->ws.descs, h->descs.data(), sizeof(InstDesc) * h->n, cudaMemcpyHostToDevice,
                      st) != cudaSuccess ||
      cudaMemcpyAsync(ws + h->ws.order, h->order.data(), sizeof(int32_t) * h->n, cudaMemcpyHostToDevice,
                      st) != cudaSuccess)
    return HCRAN_ECUDA;
  h->plan_dirty = false;
  return HCRAN_OK;
}

extern "C" int hcran_prepare(hcran_t h, void *workspace_dev, void *stream) {
  if (!h || !ws_ok(workspace_dev)) return HCRAN_EINVAL;
  char *ws = static_cast<char *>(workspace_dev);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (upload_plan(h, ws, st) != HCRAN_OK ||
      cudaMemcpyAsync(ws + h->ws.darena, h->dimage.data(), sizeof(double) * h->dtot,
                      cudaMemcpyHostToDevice, st) != cudaSuccess)
    return HCRAN_ECUDA;
  return HCRAN_OK;
}

static int check_tol(const hcran_tol *t) {
  if (!t) return HCRAN_EINVAL;
  if (!(t->tol_dinkelbach >= 0) || !(t->tol_scale >= 0) || !(t->tol_dual >= 0)) return HCRAN_EINVAL;
  if (t->max_dinkelbach < 1 || t->max_scale < 1 || t->max_dual < 1) return HCRAN_EINVAL;
  if (!(t->tie_eps >= 0) || !(t->q_init >= 0) || !isfinite(t->q_init)) return HCRAN_EINVAL;
  return HCRAN_OK;
}

static Tol to_tol(const hcran_tol *tol) {
  Tol t;
  t.tol_dinkelbach = tol->tol_dinkelbach;
  t.tol_scale = tol->tol_scale;
  t.tol_dual = tol->tol_dual;
  t.max_dinkelbach = tol->max_dinkelbach;
  t.max_scale = tol->max_scale;
  t.max_dual = tol->max_dual;
  t.tie_eps = (float)tol->tie_eps;
  t.q_init = tol->q_init;
  t.mode = kModeCold;
  t.spin_limit = 0;
  t.stall_instance = -1;
  return t;
}

// one persistent launch of class L over the first `count` instances of its
// segment of the order array
static cudaError_t launch_class(hcran_t h, const LaunchClass &L, const KDims &kd, int csize, int count, int k,
                                const float *gains_dev, const Tol &t, char *ws, cudaStream_t st, int *launches,
                                const WarmIO &wio = WarmIO{nullptr, nullptr}) {
  return launch_solve(reinterpret_cast<const InstDesc *>(ws + h->ws.descs),
                      reinterpret_cast<const int *>(ws + h->ws.order) + L.first, count, gains_dev,
                      reinterpret_cast<double *>(ws + h->ws.darena), reinterpret_cast<float *>(ws + h->ws.farena),
                      reinterpret_cast<int *>(ws + h->ws.iarena), reinterpret_cast<InstOut *>(ws + h->ws.outs), t,
                      kd, csize, reinterpret_cast<int *>(ws + h->ws.counter) + k, st, launches, wio);
}

static int do_solve(hcran_t h, const float *gains_dev, const hcran_tol *tol, void *workspace_dev,
                    void *stream, int mode = kModeCold, const WarmIO &wio = WarmIO{nullptr, nullptr}) {
  char *ws = static_cast<char *>(workspace_dev);
  if (h->plan_dirty && upload_plan(h, ws, static_cast<cudaStream_t>(stream)) != HCRAN_OK) return HCRAN_ECUDA;
  Tol t = to_tol(tol);
  t.mode = mode;
  t.spin_limit = h->spin_limit;
  t.stall_instance = h->stall_instance;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!h->side) {
    if (cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->join, cudaEventDisableTiming) != cudaSuccess)
      return HCRAN_ECUDA;
  }
  // clusters of 8 down to 4 CTAs on the caller's stream; single CTAs, then
  // clusters of 2 and 3, then the streamed class on a side stream forked from
  // and joined back into it, so that they fill the SMs the large clusters
  // leave free
  int launches = 0;
  cudaError_t err = cudaEventRecord(h->fork, st);
  if (err == cudaSuccess) err = cudaStreamWaitEvent(h->side, h->fork, 0);
  static const int kOrder[kNumClasses] = {class_of(8), class_of(7), class_of(6), class_of(5), class_of(4),
                                          class_of(1), class_of(2), class_of(3), kNumClasses - 1};
  for (int i = 0; i < kNumClasses && err == cudaSuccess; i++) {
    const int k = kOrder[i];
    const LaunchClass &L = h->classes[k];
    if (L.count == 0) continue;
    int l = 0;
    const bool on_main = k < kNumClasses - 1 && L.csize >= 4;
    err = launch_class(h, L, L.kd, L.csize, L.count, k, gains_dev, t, ws, on_main ? st : h->side, &l, wio);
    launches += l;
  }
  if (err == cudaSuccess) err = cudaEventRecord(h->join, h->side);
  if (err == cudaSuccess) err = cudaStreamWaitEvent(st, h->join, 0);
  h->last_ws = workspace_dev;
  h->last_stream = static_cast<cudaStream_t>(stream);
  h->last_launches = launches;
  return err == cudaSuccess ? HCRAN_OK : HCRAN_ECUDA;
}

// a state set by hcran_set_state applies to one solve: once the descriptors
// that carry it are enqueued, the host copies go back to the cold start
static void clear_start_flags(hcran_t h) {
  bool any = false;
  for (InstDesc &d : h->descs)
    if (d.start) {
      d.start = 0;
      any = true;
    }
  if (any) h->plan_dirty = true;
}
static bool start_pending(hcran_t h) {
  for (const InstDesc &d : h->descs)
    if (d.start) return true;
  return false;
}

extern "C" int hcran_solve(hcran_t h, const float *gains_dev, const hcran_tol *tol,
                           void *workspace_dev, void *stream) {
  if (!h || !gains_dev || !ws_ok(workspace_dev) || (reinterpret_cast<uintptr_t>(gains_dev) & 15))
    return HCRAN_EINVAL;
  const int rc = check_tol(tol);
  if (rc != HCRAN_OK) return rc;
  const int r = do_solve(h, gains_dev, tol, workspace_dev, stream);
  clear_start_flags(h);
  return r;
}

extern "C" int hcran_set_wait_limit(hcran_t h, int64_t max_tries, int32_t stall_instance) {
  if (!h || max_tries < 0 || stall_instance < -1 || stall_instance >= h->n) return HCRAN_EINVAL;
  h->spin_limit = max_tries;
  h->stall_instance = stall_instance;
  if (h->graph) {  // the captured launches carry the old settings
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
  return HCRAN_OK;
}

extern "C" int hcran_set_state(hcran_t h, void *workspace_dev, int32_t index, const hcran_result *st,
                               void *stream) {
  if (!h || !ws_ok(workspace_dev) || !st || index < 0 || index >= h->n || !st->A || !st->S || !st->p)
    return HCRAN_EINVAL;
  const InstDesc &d = h->descs[index];
  const DLayout dl = dlayout(d.M, d.N, d.K, d.Ks, d.l);
  const FLayout fl = flayout(d.M, d.N, d.K, d.l, nchunk_cap(d.N, d.K));
  const ILayout il = ilayout(d.M, d.N, d.K, d.Ks, d.l);
  const double *cst = h->dimage.data() + d.d_off;  // the instance's constants (pmax)
  const int M = d.M, N = d.N, K = d.K, l = d.l, U = d.U;
  const int Up = slot_stride(M, l), NPp = pair_stride(M, l), npair = d.npair;
  // the state must be a valid allocation: A_k in [-1, M); per (n, m) at most
  // l distinct users of m, packed at the front; powers finite in [0, mask];
  // multipliers finite, xi' and zeta_sic' >= 0, zeta' in [1e-6, 1e6]
  for (int k = 0; k < K; k++)
    if (st->A[k] < -1 || st->A[k] >= M) return HCRAN_EINVAL;
  std::vector<int32_t> Simg(size_t(N) * Up, -1);
  std::vector<float> pimg(size_t(N) * Up, 0.f), aimg(size_t(N) * Up, 1.f), bimg(size_t(N) * Up, 0.f);
  for (int n = 0; n < N; n++)
    for (int m = 0; m < M; m++) {
      const double mask = cst[dl.pmax + m] / N;
      bool ended = false;
      for (int s2 = 0; s2 < l; s2++) {
        const size_t i = (size_t(n) * M + m) * l + s2, e = size_t(n) * Up + m * l + s2;
        const int32_t k = st->S[i];
        if (k < 0) {
          if (k != -1) return HCRAN_EINVAL;
          ended = true;
          continue;
        }
        if (ended || k >= K || st->A[k] != m) return HCRAN_EINVAL;
        for (int b = 0; b < s2; b++)
          if (st->S[i - s2 + b] == k) return HCRAN_EINVAL;
        const float pv = st->p[i];
        if (!(pv >= 0.f) || !(pv <= mask * (1.0 + 1e-6))) return HCRAN_EINVAL;
        Simg[e] = k;
        pimg[e] = pv;
        if (st->alpha) aimg[e] = st->alpha[i];
        if (st->beta) bimg[e] = st->beta[i];
        if (!isfinite(aimg[e]) || !isfinite(bimg[e])) return HCRAN_EINVAL;
      }
    }
  (void)U;
  std::vector<double> xi(M, 0.0), zeta(d.Ks > 0 ? d.Ks : 1, 1.0), zs(size_t(N) * NPp, 0.0);
  for (int m = 0; m < M; m++)
    if (st->xi) {
      xi[m] = st->xi[m];
      if (!(xi[m] >= 0.0) || !isfinite(xi[m])) return HCRAN_EINVAL;
    }
  for (int k = 0; k < d.Ks; k++)
    if (st->zeta) {
      zeta[k] = st->zeta[k];
      if (!(zeta[k] >= 1e-6 && zeta[k] <= 1e6)) return HCRAN_EINVAL;
    }
  if (st->zeta_sic)
    for (int n = 0; n < N; n++)
      for (int t = 0; t < M * npair; t++) {
        const double z = st->zeta_sic[size_t(n) * M * npair + t];
        if (!(z >= 0.0) || !isfinite(z)) return HCRAN_EINVAL;
        zs[size_t(n) * NPp + t] = z;
      }
  char *ws = static_cast<char *>(workspace_dev);
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  char *db = ws + h->ws.darena + sizeof(double) * d.d_off;
  char *fb = ws + h->ws.farena + sizeof(float) * d.f_off;
  char *ib = ws + h->ws.iarena + sizeof(int32_t) * d.i_off;
  const cudaMemcpyKind hd = cudaMemcpyHostToDevice;
  // pageable sources: each call returns once its source is staged
  bool ok = cudaMemcpyAsync(ib + sizeof(int32_t) * il.A, st->A, sizeof(int32_t) * K, hd, cs) == cudaSuccess;
  ok = ok && cudaMemcpyAsync(ib + sizeof(int32_t) * il.S, Simg.data(), sizeof(int32_t) * Simg.size(), hd, cs) ==
                 cudaSuccess;
  ok = ok && cudaMemcpyAsync(fb + sizeof(float) * fl.p, pimg.data(), sizeof(float) * pimg.size(), hd, cs) ==
                 cudaSuccess;
  ok = ok && cudaMemcpyAsync(fb + sizeof(float) * fl.alpha, aimg.data(), sizeof(float) * aimg.size(), hd, cs) ==
                 cudaSuccess;
  ok = ok && cudaMemcpyAsync(fb + sizeof(float) * fl.beta, bimg.data(), sizeof(float) * bimg.size(), hd, cs) ==
                 cudaSuccess;
  ok = ok && cudaMemcpyAsync(db + sizeof(double) * dl.xi, xi.data(), sizeof(double) * M, hd, cs) == cudaSuccess;
  if (d.Ks > 0)
    ok = ok && cudaMemcpyAsync(db + sizeof(double) * dl.zeta, zeta.data(), sizeof(double) * d.Ks, hd, cs) ==
                   cudaSuccess;
  ok = ok && cudaMemcpyAsync(db + sizeof(double) * dl.zsic, zs.data(), sizeof(double) * zs.size(), hd, cs) ==
                 cudaSuccess;
  if (!ok) return HCRAN_ECUDA;
  h->descs[index].start = 1;
  h->plan_dirty = true;
  return HCRAN_OK;
}

extern "C" int hcran_solve_host(hcran_t h, const float *gains_host, const hcran_tol *tol,
                                void *workspace_dev, void *stream, double *ee_host,
                                int32_t *status_host) {
  if (!h || !gains_host || !ws_ok(workspace_dev)) return HCRAN_EINVAL;
  int rc = check_tol(tol);
  if (rc != HCRAN_OK) return rc;
  char *ws = static_cast<char *>(workspace_dev);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  float *staging = reinterpret_cast<float *>(ws + h->ws.staging);
  if (cudaMemcpyAsync(staging, gains_host, sizeof(float) * h->gain_elems, cudaMemcpyHostToDevice,
                      st) != cudaSuccess)
    return HCRAN_ECUDA;
  rc = do_solve(h, staging, tol, workspace_dev, stream);
  clear_start_flags(h);
  if (rc != HCRAN_OK) return rc;
  if (cudaMemcpyAsync(h->outs_host.data(), ws + h->ws.outs, sizeof(InstOut) * h->n,
                      cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return HCRAN_ECUDA;
  int worst = HCRAN_OK;
  for (int32_t b = 0; b < h->n; b++) {
    if (ee_host) ee_host[b] = h->outs_host[b].ee;
    if (status_host) status_host[b] = h->outs_host[b].status;
    if (h->outs_host[b].status & kStatusTimeoutHost) worst = HCRAN_ETIMEDOUT;
    else if ((h->outs_host[b].status & kStatusNumericHost) && worst == HCRAN_OK) worst = HCRAN_ENUMERIC;
  }
  return worst;
}

static int sync_last(hcran_t h) {
  if (!h->last_ws) return HCRAN_EINVAL;
  return cudaStreamSynchronize(h->last_stream) == cudaSuccess ? HCRAN_OK : HCRAN_ECUDA;
}

template <typename T>
static bool copy_out(T *dst, const char *src, size_t count) {
  if (!dst || count == 0) return true;
  return cudaMemcpy(dst, src, sizeof(T) * count, cudaMemcpyDeviceToHost) == cudaSuccess;
}

// rows of `width` elements stored with pitch `pitch` -> packed host array
template <typename T>
static bool copy_rows(T *dst, const char *src, size_t width, size_t pitch, size_t rows) {
  if (!dst || width == 0 || rows == 0) return true;
  return cudaMemcpy2D(dst, sizeof(T) * width, src, sizeof(T) * pitch, sizeof(T) * width, rows,
                      cudaMemcpyDeviceToHost) == cudaSuccess;
}

extern "C" int hcran_get(hcran_t h, int32_t index, hcran_result *out) {
  if (!h || !out || index < 0 || index >= h->n) return HCRAN_EINVAL;
  int rc = sync_last(h);
  if (rc != HCRAN_OK) return rc;
  const char *ws = static_cast<const char *>(h->last_ws);
  const InstDesc &d = h->descs[index];
  const DLayout dl = dlayout(d.M, d.N, d.K, d.Ks, d.l);
  const FLayout fl = flayout(d.M, d.N, d.K, d.l, nchunk_cap(d.N, d.K));
  const ILayout il = ilayout(d.M, d.N, d.K, d.Ks, d.l);
  const char *db = ws + h->ws.darena + sizeof(double) * d.d_off;
  const char *fb = ws + h->ws.farena + sizeof(float) * d.f_off;
  const char *ib = ws + h->ws.iarena + sizeof(int32_t) * d.i_off;
  InstOut o;
  bool ok = cudaMemcpy(&o, ws + h->ws.outs + sizeof(InstOut) * index, sizeof(InstOut),
                       cudaMemcpyDeviceToHost) == cudaSuccess;
  const size_t Up = slot_stride(d.M, d.l), NPp = pair_stride(d.M, d.l);
  ok = ok && copy_out(out->A, ib + sizeof(int32_t) * il.A, d.K);
  ok = ok && copy_rows(out->S, ib + sizeof(int32_t) * il.S, d.U, Up, d.N);
  ok = ok && copy_rows(out->p, fb + sizeof(float) * fl.p, d.U, Up, d.N);
  ok = ok && copy_rows(out->alpha, fb + sizeof(float) * fl.alpha, d.U, Up, d.N);
  ok = ok && copy_rows(out->beta, fb + sizeof(float) * fl.beta, d.U, Up, d.N);
  ok = ok && copy_out(out->xi, db + sizeof(double) * dl.xi, d.M);
  ok = ok && copy_out(out->zeta, db + sizeof(double) * dl.zeta, d.Ks);
  ok = ok && copy_rows(out->zeta_sic, db + sizeof(double) * dl.zsic, size_t(d.M) * d.npair, NPp, d.N);
  if (!ok) return HCRAN_ECUDA;
  out->ee = o.ee; out->R = o.R; out->P = o.P;
  out->iters[0] = o.iters[0]; out->iters[1] = o.iters[1]; out->iters[2] = o.iters[2];
  out->status = o.status;
  out->slack_power_min = o.slack_power_min;
  out->slack_rate_min = o.slack_rate_min;
  out->slack_sic_max = o.slack_sic_max;
  out->min_margin = o.min_margin;
  out->n_ties = o.n_ties;
  if (o.status & kStatusTimeoutHost) return HCRAN_ETIMEDOUT;
  if (o.status & kStatusNumericHost) return HCRAN_ENUMERIC;
  return HCRAN_OK;
}

extern "C" int hcran_get_summary(hcran_t h, double *ee, double *R, double *P, int32_t *status,
                                 int32_t *iters3, double *min_margin, int32_t *n_ties) {
  if (!h) return HCRAN_EINVAL;
  int rc = sync_last(h);
  if (rc != HCRAN_OK) return rc;
  const char *ws = static_cast<const char *>(h->last_ws);
  if (cudaMemcpy(h->outs_host.data(), ws + h->ws.outs, sizeof(InstOut) * h->n,
                 cudaMemcpyDeviceToHost) != cudaSuccess)
    return HCRAN_ECUDA;
  for (int32_t b = 0; b < h->n; b++) {
    const InstOut &o = h->outs_host[b];
    if (ee) ee[b] = o.ee;
    if (R) R[b] = o.R;
    if (P) P[b] = o.P;
    if (status) status[b] = o.status;
    if (iters3) for (int i = 0; i < 3; i++) iters3[3 * b + i] = o.iters[i];
    if (min_margin) min_margin[b] = o.min_margin;
    if (n_ties) n_ties[b] = o.n_ties;
  }
  return HCRAN_OK;
}

extern "C" int hcran_get_phase_cycles(hcran_t h, int64_t *cycles) {
  if (!h || !cycles) return HCRAN_EINVAL;
  int rc = sync_last(h);
  if (rc != HCRAN_OK) return rc;
  const char *ws = static_cast<const char *>(h->last_ws);
  if (cudaMemcpy(h->outs_host.data(), ws + h->ws.outs, sizeof(InstOut) * h->n,
                 cudaMemcpyDeviceToHost) != cudaSuccess)
    return HCRAN_ECUDA;
  for (int32_t b = 0; b < h->n; b++)
    for (int i = 0; i < 8; i++) cycles[8 * b + i] = h->outs_host[b].cycles[i];
  return HCRAN_OK;
}

extern "C" int hcran_last_launch_count(hcran_t h, int32_t *launches) {
  if (!h || !launches) return HCRAN_EINVAL;
  *launches = h->last_launches;
  return HCRAN_OK;
}

extern "C" int hcran_get_schedule(hcran_t h, int32_t *cluster_size) {
  if (!h || !cluster_size) return HCRAN_EINVAL;
  for (int32_t b = 0; b < h->n; b++)
    cluster_size[b] = h->cls[b] < kNumClasses - 1 ? class_csize(h->cls[b]) : 0;
  return HCRAN_OK;
}

extern "C" int hcran_set_schedule(hcran_t h, const int32_t *cluster_size) {
  if (!h || !cluster_size) return HCRAN_EINVAL;
  std::vector<int32_t> cls(h->n);
  int32_t teams = 0;
  for (int32_t b = 0; b < h->n; b++) {
    const InstDesc &d = h->descs[b];
    const int C = cluster_size[b];
    if (C <= 0) {
      if (C < -4 || (C < 0 && teams != 0 && teams != -C)) return HCRAN_EINVAL;
      if (C < 0) teams = -C;
      cls[b] = kNumClasses - 1;
      continue;
    }
    int k = -1;
    for (int q = 0; q < kNumClasses - 1; q++)
      if (class_csize(q) == C) k = q;
    if (k < 0 || C > d.N) return HCRAN_EINVAL;
    if (dyn_smem_bytes(resident_kdims(d.M, d.l, d.Ks, d.N, C)) > kMaxDynSmem - kClassMargin) return HCRAN_EINVAL;
    cls[b] = k;
  }
  const std::vector<int32_t> keep = h->cls;
  const int32_t keep_teams = h->stream_teams;
  h->cls = cls;
  h->stream_teams = teams;
  if (build_classes(h) != 0) {
    h->cls = keep;
    h->stream_teams = keep_teams;
    build_classes(h);
    return HCRAN_EINVAL;
  }
  return HCRAN_OK;
}

// Autotuner: for every cluster size C < 8 in use, time the class's schedule
// against clusters of min(2 C, 8) CTAs on a probe of the class (the first S
// instances in launch order, S = min(class size, two waves of the current
// schedule); one Dinkelbach iteration, one SCALE pass, no early stop) and
// keep the faster.  Each schedule is timed twice, with max_dual_probe / 4 and
// with max_dual_probe dual iterations, and compared on the difference: the
// cost of the dual iterations alone, which make up almost all of a full solve,
// without the selection and set-up of the probe's single Dinkelbach
// iteration, which would otherwise dominate it.  A probe over S instances
// compares throughput when the class fills several waves and latency when it
// does not.
extern "C" int hcran_autotune(hcran_t h, const float *gains_dev, const hcran_tol *tol, void *workspace_dev,
                              void *stream, int32_t max_dual_probe) {
  if (!h || !gains_dev || !ws_ok(workspace_dev) || (reinterpret_cast<uintptr_t>(gains_dev) & 15) ||
      max_dual_probe < 1)
    return HCRAN_EINVAL;
  int rc = check_tol(tol);
  if (rc != HCRAN_OK) return rc;
  if (start_pending(h)) return HCRAN_EINVAL;  // a set state applies to hcran_solve / hcran_solve_host
  char *ws = static_cast<char *>(workspace_dev);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (h->plan_dirty && upload_plan(h, ws, st) != HCRAN_OK) return HCRAN_ECUDA;
  hcran_tol pt = *tol;
  pt.tol_dinkelbach = pt.tol_scale = pt.tol_dual = 0.0;
  pt.max_dinkelbach = 1;
  pt.max_scale = 1;
  const int V1 = max_dual_probe / 4 > 0 ? max_dual_probe / 4 : 1, V2 = V1 + max_dual_probe;
  pt.max_dual = V1;
  const Tol t1 = to_tol(&pt);
  pt.max_dual = V2;
  const Tol t2 = to_tol(&pt);
  int dev = 0, sms = 1;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return HCRAN_ECUDA;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return HCRAN_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return HCRAN_ECUDA;
  }
  std::vector<int32_t> cls = h->cls;
  for (int k = kNumClasses - 2; k >= 1 && rc == HCRAN_OK; k--) {  // cluster sizes 1 .. 7 (8 has no larger)
    const LaunchClass L = h->classes[k];
    if (L.count == 0) continue;
    const int C = L.csize, C2 = 2 * C < kMaxCluster ? 2 * C : kMaxCluster;
    // probe: the instances of the class in launch order (at most eight waves
    // of the current schedule); every one of them must have a subcarrier for
    // each CTA of the larger cluster
    std::vector<int32_t> probe;
    const int S = std::min(L.count, 8 * (sms / C));
    for (int i = 0; i < S; i++) probe.push_back(h->order[L.first + i]);
    bool fits = true;
    for (int32_t b : probe) fits = fits && h->descs[b].N >= C2;
    if (!fits) continue;
    KDims kd1{}, kd2{};
    for (size_t i = 0; i < probe.size(); i++) {
      const InstDesc &d = h->descs[probe[i]];
      const KDims a = resident_kdims(d.M, d.l, d.Ks, d.N, C), b = resident_kdims(d.M, d.l, d.Ks, d.N, C2);
      if (i == 0) {
        kd1 = a;
        kd2 = b;
      } else {
        kdims_merge(kd1, a);
        kdims_merge(kd2, b);
      }
    }
    // each probe timed twice, the shorter kept: the decision rests on a
    // difference of a few percent, and one timing can carry more noise
    float ms[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
    for (int v = 0; v < 2 && rc == HCRAN_OK; v++)
      for (int j = 0; j < 2 && rc == HCRAN_OK; j++)
        for (int rep = 0; rep < 2 && rc == HCRAN_OK; rep++) {
          int l = 0;
          float t = 0.f;
          if (cudaEventRecord(e0, st) != cudaSuccess ||
              launch_class(h, L, v ? kd2 : kd1, v ? C2 : C, (int)probe.size(), k, gains_dev, j ? t2 : t1, ws, st,
                           &l) != cudaSuccess ||
              cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
              cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)
            rc = HCRAN_ECUDA;
          if (rep == 0 || t < ms[v][j]) ms[v][j] = t;
        }
    if (rc == HCRAN_OK && ms[1][1] - ms[1][0] < ms[0][1] - ms[0][0])
      for (int i = 0; i < L.count; i++) {
        const int32_t b = h->order[L.first + i];
        if (h->descs[b].N >= C2) cls[b] = class_of(C2);
      }
  }
  // the streamed class: how many teams its sweeps run (the planner takes as
  // many as fit; fewer, larger teams give each subcarrier more threads)
  int32_t teams = h->stream_teams;
  {
    const LaunchClass L = h->classes[kNumClasses - 1];
    if (rc == HCRAN_OK && L.count > 0 && L.kd.staged && L.kd.teams > 0) {
      const int S = std::min(L.count, sms);  // the first wave of the class
      float best = 0.f;
      int best_t = 0;
      for (int t = 1; t <= L.kd.teams && rc == HCRAN_OK; t++) {
        KDims kd = L.kd;
        kd.teams = t;
        if (dyn_smem_bytes(kd) > kMaxDynSmem) continue;
        float ms[2] = {0.f, 0.f};
        for (int j = 0; j < 2 && rc == HCRAN_OK; j++) {
          int l = 0;
          if (cudaEventRecord(e0, st) != cudaSuccess ||
              launch_class(h, L, kd, 1, S, kNumClasses - 1, gains_dev, j ? t2 : t1, ws, st, &l) != cudaSuccess ||
              cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
              cudaEventElapsedTime(&ms[j], e0, e1) != cudaSuccess)
            rc = HCRAN_ECUDA;
        }
        if (rc == HCRAN_OK && (best_t == 0 || ms[1] - ms[0] < best)) {
          best = ms[1] - ms[0];
          best_t = t;
        }
      }
      if (rc == HCRAN_OK && best_t > 0) teams = best_t;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != HCRAN_OK) return rc;
  if (cls != h->cls || teams != h->stream_teams) {
    h->cls = cls;
    h->stream_teams = teams;
    if (build_classes(h) != 0) return HCRAN_EINVAL;
  }
  return HCRAN_OK;
}

extern "C" int hcran_get_stream_teams(hcran_t h, int32_t *teams) {
  if (!h || !teams) return HCRAN_EINVAL;
  const LaunchClass &L = h->classes[kNumClasses - 1];
  *teams = L.count > 0 ? L.kd.teams : 0;
  return HCRAN_OK;
}

extern "C" int hcran_solve_graph(hcran_t h, const float *gains_dev, const hcran_tol *tol, void *workspace_dev,
                                 void *stream) {
  if (!h || !gains_dev || !ws_ok(workspace_dev) || (reinterpret_cast<uintptr_t>(gains_dev) & 15) || !stream)
    return HCRAN_EINVAL;
  int rc = check_tol(tol);
  if (rc != HCRAN_OK) return rc;
  if (start_pending(h)) return HCRAN_EINVAL;  // a set state applies to hcran_solve / hcran_solve_host
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char *ws = static_cast<char *>(workspace_dev);
  if (h->plan_dirty && upload_plan(h, ws, st) != HCRAN_OK) return HCRAN_ECUDA;
  const bool same = h->graph && h->graph_gains == gains_dev && h->graph_ws == workspace_dev &&
                    memcmp(&h->graph_tol, tol, sizeof(hcran_tol)) == 0;
  if (!same) {
    if (h->graph) {
      cudaGraphExecDestroy(h->graph);
      h->graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return HCRAN_ECUDA;
    rc = do_solve(h, gains_dev, tol, workspace_dev, stream);
    const cudaError_t ec = cudaStreamEndCapture(st, &g);
    if (rc != HCRAN_OK || ec != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return HCRAN_ECUDA;
    }
    const cudaError_t ei = cudaGraphInstantiate(&h->graph, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
      h->graph = nullptr;
      return HCRAN_ECUDA;
    }
    h->graph_gains = gains_dev;
    h->graph_ws = workspace_dev;
    h->graph_tol = *tol;
  }
  if (cudaGraphLaunch(h->graph, st) != cudaSuccess) return HCRAN_ECUDA;
  h->last_ws = workspace_dev;
  h->last_stream = st;
  return HCRAN_OK;
}

extern "C" int hcran_warm_rows(hcran_t h, int64_t *rows) {
  if (!h || !rows) return HCRAN_EINVAL;
  *rows = h->warm_rows;
  return HCRAN_OK;
}

extern "C" int hcran_warm_features(hcran_t h, const float *gains_dev, void *workspace_dev, void *stream,
                                   void *features_dev) {
  if (!h || !gains_dev || !ws_ok(workspace_dev) || (reinterpret_cast<uintptr_t>(gains_dev) & 15) ||
      !features_dev || (reinterpret_cast<uintptr_t>(features_dev) & 15))
    return HCRAN_EINVAL;
  hcran_tol t{};
  t.max_dinkelbach = t.max_scale = t.max_dual = 1;
  return do_solve(h, gains_dev, &t, workspace_dev, stream, kModeFeatures, WarmIO{nullptr, features_dev});
}

extern "C" int hcran_solve_warm(hcran_t h, const float *gains_dev, const hcran_tol *tol, void *workspace_dev,
                                void *stream, const float *net_out_dev) {
  if (!h || !gains_dev || !ws_ok(workspace_dev) || (reinterpret_cast<uintptr_t>(gains_dev) & 15) || !net_out_dev ||
      (reinterpret_cast<uintptr_t>(net_out_dev) & 15))
    return HCRAN_EINVAL;
  const int rc = check_tol(tol);
  if (rc != HCRAN_OK) return rc;
  return do_solve(h, gains_dev, tol, workspace_dev, stream, kModeWarm, WarmIO{net_out_dev, nullptr});
}

extern "C" void hcran_destroy(hcran_t h) { delete h; }
