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
                         const KDims &kd, int csize, int *counter, cudaStream_t stream, int *launches);
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
  WsLayout ws{};
  void *last_ws = nullptr;
  cudaStream_t last_stream = nullptr;
  int32_t last_launches = 0;
  std::vector<InstOut> outs_host;
};

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
      d.nchunk = class_nchunk(c.N, c.K, class_csize(h->cls[b]));
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
    // launch dimensions per class; an instance that would push its class over
    // the shared-memory limit moves on to the next larger cluster
    for (;;) {
      bool moved = false;
      for (int k = 0; k < kNumClasses; k++) h->classes[k] = LaunchClass();
      for (int32_t b = 0; b < n; b++) {
        const hcran_config &c = cfgs[b];
        LaunchClass &L = h->classes[h->cls[b]];
        const KDims one = h->cls[b] < kNumClasses - 1
                              ? resident_kdims(c.M, c.l, c.Ks, c.N, class_csize(h->cls[b]))
                              : KDims{slot_stride(c.M, c.l), c.M, c.l * (c.l - 1) / 2, pair_stride(c.M, c.l),
                                      c.Ks, 0, 0, 0};
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
            const int64_t r = res_floats(cfgs[b].M, cfgs[b].l, cfgs[b].Ks,
                                         (cfgs[b].N + class_csize(k) - 1) / class_csize(k));
            if (r > wr) { wr = r; worst = b; }
          }
        h->cls[worst] = k == 0 ? kNumClasses - 1 : k - 1;
        h->descs[worst].nchunk = class_nchunk(cfgs[worst].N, cfgs[worst].K, class_csize(h->cls[worst]));
        moved = true;
      }
      if (!moved) break;
    }
    {  // streamed class: staging when the double buffers fit, else global reads
      LaunchClass &L = h->classes[kNumClasses - 1];
      if (L.count > 0 && plan_kdims(L.kd, int64_t(1) << 40) != 0) { delete h; return HCRAN_EINVAL; }
    }
    // arenas (the chunk count of an instance depends on its class)
    doff = foff = ioff = 0;
    for (int32_t b = 0; b < n; b++) {
      const hcran_config &c = cfgs[b];
      InstDesc &d = h->descs[b];
      const DLayout dl = dlayout(c.M, c.N, c.K, c.Ks, c.l);
      const FLayout fl = flayout(c.M, c.N, c.K, c.l, d.nchunk);
      const ILayout il = ilayout(c.M, c.N, c.K, c.l);
      d.d_off = doff; doff += al4(dl.total);
      d.f_off = foff; foff += al4(fl.total);
      d.i_off = ioff; ioff += al4(il.total);
    }
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
      for (int k = 0; k < c.Ks; k++) db[dl.Psi + k] = min_rate(c.T_s[k], c.lambda_pps[k], c.zbar_bits, c.Bn_hz);
      for (int64_t t = 0; t < int64_t(c.M) * c.K; t++) db[dl.w + t] = c.w ? c.w[t] : 1.0;
    }
    // classes in launch order (largest clusters first); longest-processing-time
    // order inside a class: largest M*N*K*l first
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

static bool ws_ok(void *ws) { return ws && (reinterpret_cast<uintptr_t>(ws) & 255) == 0; }

extern "C" int hcran_prepare(hcran_t h, void *workspace_dev, void *stream) {
  if (!h || !ws_ok(workspace_dev)) return HCRAN_EINVAL;
  char *ws = static_cast<char *>(workspace_dev);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(ws + h->ws.descs, h->descs.data(), sizeof(InstDesc) * h->n,
                      cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(ws + h->ws.order, h->order.data(), sizeof(int32_t) * h->n,
                      cudaMemcpyHostToDevice, st) != cudaSuccess ||
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

static int do_solve(hcran_t h, const float *gains_dev, const hcran_tol *tol, void *workspace_dev,
                    void *stream) {
  char *ws = static_cast<char *>(workspace_dev);
  Tol t;
  t.tol_dinkelbach = tol->tol_dinkelbach;
  t.tol_scale = tol->tol_scale;
  t.tol_dual = tol->tol_dual;
  t.max_dinkelbach = tol->max_dinkelbach;
  t.max_scale = tol->max_scale;
  t.max_dual = tol->max_dual;
  t.tie_eps = (float)tol->tie_eps;
  t.q_init = tol->q_init;
  int launches = 0;
  cudaError_t err = cudaSuccess;
  for (int k = 0; k < kNumClasses && err == cudaSuccess; k++) {
    const LaunchClass &L = h->classes[k];
    if (L.count == 0) continue;
    int l = 0;
    err = launch_solve(reinterpret_cast<const InstDesc *>(ws + h->ws.descs),
                       reinterpret_cast<const int *>(ws + h->ws.order) + L.first, L.count, gains_dev,
                       reinterpret_cast<double *>(ws + h->ws.darena), reinterpret_cast<float *>(ws + h->ws.farena),
                       reinterpret_cast<int *>(ws + h->ws.iarena), reinterpret_cast<InstOut *>(ws + h->ws.outs),
                       t, L.kd, L.csize, reinterpret_cast<int *>(ws + h->ws.counter) + k,
                       static_cast<cudaStream_t>(stream), &l);
    launches += l;
  }
  h->last_ws = workspace_dev;
  h->last_stream = static_cast<cudaStream_t>(stream);
  h->last_launches = launches;
  return err == cudaSuccess ? HCRAN_OK : HCRAN_ECUDA;
}

extern "C" int hcran_solve(hcran_t h, const float *gains_dev, const hcran_tol *tol,
                           void *workspace_dev, void *stream) {
  if (!h || !gains_dev || !ws_ok(workspace_dev) || (reinterpret_cast<uintptr_t>(gains_dev) & 15))
    return HCRAN_EINVAL;
  const int rc = check_tol(tol);
  if (rc != HCRAN_OK) return rc;
  return do_solve(h, gains_dev, tol, workspace_dev, stream);
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
  if (rc != HCRAN_OK) return rc;
  if (cudaMemcpyAsync(h->outs_host.data(), ws + h->ws.outs, sizeof(InstOut) * h->n,
                      cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return HCRAN_ECUDA;
  for (int32_t b = 0; b < h->n; b++) {
    if (ee_host) ee_host[b] = h->outs_host[b].ee;
    if (status_host) status_host[b] = h->outs_host[b].status;
  }
  return HCRAN_OK;
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
  const FLayout fl = flayout(d.M, d.N, d.K, d.l, d.nchunk);
  const ILayout il = ilayout(d.M, d.N, d.K, d.l);
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

extern "C" void hcran_destroy(hcran_t h) { delete h; }
