// hcran_noalloc.cu -- hcran_solve_noalloc: one instance solved with no memory
// allocation at all, for callers that cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is unavailable or forbidden,
// for instance inside a memory pool owned by another framework, in a process
// whose allocator is locked down after start-up, or in a real-time loop that
// must not touch the allocator (an allocation can block on a device-wide
// synchronisation).  Such a caller still owns its inputs (the gains on the
// device) and outputs (host result arrays); the solver's working memory comes
// from one file-scope device array instead of a caller-provided workspace.
//
// The array below is part of the module: every GPU that loads this library
// keeps it (kNoallocScratchBytes) until the process exits.  Every call looks
// up its device address on the current device.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include "../../include/hcran.h"
#include "hcran_layout.h"

namespace hcran {
cudaError_t launch_solve(const InstDesc *descs, const int *order, int n_inst, const float *gains,
                         double *darena, float *farena, int *iarena, InstOut *outs, const Tol &tol,
                         const KDims &kd, int csize, int *counter, cudaStream_t stream, int *launches,
                         const WarmIO &wio);
}

using namespace hcran;

namespace {

constexpr size_t kNoallocScratchBytes = size_t(HCRAN_NOALLOC_SCRATCH_BYTES);

// The solver's whole workspace for hcran_solve_noalloc.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

// In host code the name of the array is only a host-side stand-in, never a
// usable device pointer: every call asks cudaGetSymbolAddress for the array's
// address on the current device.

struct Plan {
  InstDesc d;
  KDims kd;
  int csize;
  int32_t order;
  uint64_t o_desc, o_order, o_counter, o_out, o_darena, o_farena, o_iarena, o_tmp, total;
};

uint64_t al256(uint64_t x) { return (x + 255) & ~uint64_t(255); }

bool pos(double x) { return isfinite(x) && x > 0.0; }
bool nonneg(double x) { return isfinite(x) && x >= 0.0; }

int check(const hcran_config &c) {
  if (c.M < 1 || c.M > kMaxM || c.N < 1 || c.K < 1 || c.Ks < 0 || c.Ks > c.K || c.l < 1 ||
      c.l > kMaxL || c.M * c.l > kMaxU)
    return HCRAN_EINVAL;
  if (!c.pmax || !c.eta || !c.Pc || !c.Pf || !pos(c.Bn_hz) || !pos(c.N0_w_per_hz)) return HCRAN_EINVAL;
  for (int m = 0; m < c.M; m++)
    if (!pos(c.pmax[m]) || !pos(c.eta[m]) || !nonneg(c.Pc[m]) || !nonneg(c.Pf[m])) return HCRAN_EINVAL;
  if (c.Ks > 0) {
    if (!c.T_s || !c.lambda_pps || !pos(c.zbar_bits)) return HCRAN_EINVAL;
    for (int k = 0; k < c.Ks; k++)
      if (!pos(c.T_s[k]) || !pos(c.lambda_pps[k])) return HCRAN_EINVAL;
  }
  if (c.w)
    for (int64_t t = 0; t < int64_t(c.M) * c.K; t++)
      if (!nonneg(c.w[t])) return HCRAN_EINVAL;
  return HCRAN_OK;
}

// Workspace plan of one instance inside the static array (no heap use).
int plan(const hcran_config &c, Plan &p) {
  memset(&p, 0, sizeof(p));
  InstDesc &d = p.d;
  d.M = c.M; d.N = c.N; d.K = c.K; d.Ks = c.Ks; d.l = c.l;
  d.U = c.M * c.l;
  d.L = c.N * d.U;
  d.npair = c.l * (c.l - 1) / 2;
  const int cls = pick_class(c.M, c.l, c.Ks, c.N);
  p.csize = class_csize(cls);
  d.nchunk = class_nchunk(c.N, c.K, p.csize);
  d.g_off = 0;
  d.sigma = c.N0_w_per_hz * c.Bn_hz;
  double pc = 0.0;
  for (int m = 0; m < c.M; m++) pc += c.Pc[m] + c.Pf[m];
  d.Pconst = pc;
  const DLayout dl = dlayout(c.M, c.N, c.K, c.Ks, c.l);
  const FLayout fl = flayout(c.M, c.N, c.K, c.l, nchunk_cap(c.N, c.K));
  const ILayout il = ilayout(c.M, c.N, c.K, c.Ks, c.l);
  if (cls < kNumClasses - 1) {
    p.kd = resident_kdims(c.M, c.l, c.Ks, c.N, p.csize);
  } else {
    p.kd.Upmax = slot_stride(c.M, c.l);
    p.kd.Mmax = c.M;
    p.kd.NPmax = d.npair;
    p.kd.NPPmax = pair_stride(c.M, c.l);
    p.kd.KSmax = c.Ks;
    if (plan_kdims(p.kd, int64_t(1) << 40) != 0) return HCRAN_EINVAL;
  }
  uint64_t o = 0;
  p.o_desc = o; o = al256(o + sizeof(InstDesc));
  p.o_order = o; o = al256(o + sizeof(int32_t));
  p.o_counter = o; o = al256(o + sizeof(int32_t));
  p.o_out = o; o = al256(o + sizeof(InstOut));
  p.o_darena = o; o = al256(o + sizeof(double) * dl.total);
  p.o_farena = o; o = al256(o + sizeof(float) * fl.total);
  p.o_iarena = o; o = al256(o + sizeof(int32_t) * il.total);
  p.o_tmp = o; o = al256(o + sizeof(double) * 2 * (c.Ks > 0 ? c.Ks : 1));  // T, lambda
  p.total = o;
  return p.total <= kNoallocScratchBytes ? HCRAN_OK : HCRAN_E2BIG;
}

// Derived constants on the device: spectral masks, minimum rates of C9 (the
// smaller root of (Eq6b)), and unit priority weights when none are given.
__global__ void noalloc_prep_kernel(double *db, DLayout dl, int M, int N, int K, int Ks, double zbar,
                                    double Bn, int fill_w, const double *tmp) {
  for (int m = threadIdx.x; m < M; m += blockDim.x) db[dl.mask + m] = db[dl.pmax + m] / N;
  for (int k = threadIdx.x; k < Ks; k += blockDim.x) {
    const double x = tmp[Ks + k] * tmp[k];  // lambda T
    db[dl.Psi + k] = tmp[Ks + k] * zbar / (1.0 + x - sqrt(1.0 + x * x)) / Bn;
    db[dl.Tdel + k] = tmp[k];
  }
  if (fill_w)
    for (int64_t t = threadIdx.x; t < int64_t(M) * K; t += blockDim.x) db[dl.w + t] = 1.0;
}

template <typename T>
bool rows_d2h(T *dst, const unsigned char *src, size_t width, size_t pitch, size_t rows) {
  if (!dst || width == 0 || rows == 0) return true;
  return cudaMemcpy2D(dst, sizeof(T) * width, src, sizeof(T) * pitch, sizeof(T) * width, rows,
                      cudaMemcpyDeviceToHost) == cudaSuccess;
}

template <typename T>
bool flat_d2h(T *dst, const unsigned char *src, size_t count) {
  if (!dst || count == 0) return true;
  return cudaMemcpy(dst, src, sizeof(T) * count, cudaMemcpyDeviceToHost) == cudaSuccess;
}

}  // namespace

extern "C" int hcran_solve_noalloc(const hcran_config *cfg, const float *gains_dev, const hcran_tol *tol,
                                   void *stream, hcran_result *out) {
  if (!cfg || !gains_dev || !tol || !out || (reinterpret_cast<uintptr_t>(gains_dev) & 15))
    return HCRAN_EINVAL;
  int rc = check(*cfg);
  if (rc != HCRAN_OK) return rc;
  if (tol->max_dinkelbach < 1 || tol->max_scale < 1 || tol->max_dual < 1 || !(tol->tol_dinkelbach >= 0) ||
      !(tol->tol_scale >= 0) || !(tol->tol_dual >= 0) || !(tol->tie_eps >= 0) || !(tol->q_init >= 0) ||
      !isfinite(tol->q_init))
    return HCRAN_EINVAL;
  Plan p;
  rc = plan(*cfg, p);
  if (rc != HCRAN_OK) return rc;

  // the device address of the static array on the current device, looked up
  // on every call (cheap), so that a re-created context or another current
  // device is always served from its own copy
  void *ptr = nullptr;
  if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return HCRAN_ECUDA;
  unsigned char *ws = static_cast<unsigned char *>(ptr);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const hcran_config &c = *cfg;
  const DLayout dl = dlayout(c.M, c.N, c.K, c.Ks, c.l);
  double *db = reinterpret_cast<double *>(ws + p.o_darena);
  double *tmp = reinterpret_cast<double *>(ws + p.o_tmp);
  const int32_t zero = 0;
  // inputs into the scratch (every field the solver reads first is written here or by the kernel)
  bool ok = cudaMemcpyAsync(ws + p.o_desc, &p.d, sizeof(InstDesc), cudaMemcpyHostToDevice, st) == cudaSuccess;
  ok = ok && cudaMemcpyAsync(ws + p.o_order, &zero, sizeof(int32_t), cudaMemcpyHostToDevice, st) == cudaSuccess;
  ok = ok && cudaMemsetAsync(db, 0, sizeof(double) * dl.total, st) == cudaSuccess;
  ok = ok && cudaMemcpyAsync(db + dl.pmax, c.pmax, sizeof(double) * c.M, cudaMemcpyHostToDevice, st) == cudaSuccess;
  ok = ok && cudaMemcpyAsync(db + dl.eta, c.eta, sizeof(double) * c.M, cudaMemcpyHostToDevice, st) == cudaSuccess;
  if (c.w)
    ok = ok && cudaMemcpyAsync(db + dl.w, c.w, sizeof(double) * c.M * c.K, cudaMemcpyHostToDevice, st) ==
                   cudaSuccess;
  if (c.Ks > 0) {
    ok = ok && cudaMemcpyAsync(tmp, c.T_s, sizeof(double) * c.Ks, cudaMemcpyHostToDevice, st) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(tmp + c.Ks, c.lambda_pps, sizeof(double) * c.Ks, cudaMemcpyHostToDevice, st) ==
                   cudaSuccess;
  }
  if (!ok) return HCRAN_ECUDA;
  noalloc_prep_kernel<<<1, 256, 0, st>>>(db, dl, c.M, c.N, c.K, c.Ks, c.zbar_bits, c.Bn_hz, c.w ? 0 : 1,
                                         tmp);
  if (cudaGetLastError() != cudaSuccess) return HCRAN_ECUDA;

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
  int launches = 0;
  if (launch_solve(reinterpret_cast<const InstDesc *>(ws + p.o_desc),
                   reinterpret_cast<const int *>(ws + p.o_order), 1, gains_dev, db,
                   reinterpret_cast<float *>(ws + p.o_farena), reinterpret_cast<int *>(ws + p.o_iarena),
                   reinterpret_cast<InstOut *>(ws + p.o_out), t, p.kd, p.csize,
                   reinterpret_cast<int *>(ws + p.o_counter), st, &launches, WarmIO{nullptr, nullptr}) != cudaSuccess)
    return HCRAN_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return HCRAN_ECUDA;

  // results into the caller's host arrays
  const FLayout fl = flayout(c.M, c.N, c.K, c.l, nchunk_cap(c.N, c.K));
  const ILayout il = ilayout(c.M, c.N, c.K, c.Ks, c.l);
  const unsigned char *fb = ws + p.o_farena, *ib = ws + p.o_iarena, *dbb = ws + p.o_darena;
  const size_t Up = slot_stride(c.M, c.l), NPp = pair_stride(c.M, c.l);
  InstOut o;
  ok = cudaMemcpy(&o, ws + p.o_out, sizeof(InstOut), cudaMemcpyDeviceToHost) == cudaSuccess;
  ok = ok && flat_d2h(out->A, ib + sizeof(int32_t) * il.A, c.K);
  ok = ok && rows_d2h(out->S, ib + sizeof(int32_t) * il.S, p.d.U, Up, c.N);
  ok = ok && rows_d2h(out->p, fb + sizeof(float) * fl.p, p.d.U, Up, c.N);
  ok = ok && rows_d2h(out->alpha, fb + sizeof(float) * fl.alpha, p.d.U, Up, c.N);
  ok = ok && rows_d2h(out->beta, fb + sizeof(float) * fl.beta, p.d.U, Up, c.N);
  ok = ok && flat_d2h(out->xi, dbb + sizeof(double) * dl.xi, c.M);
  ok = ok && flat_d2h(out->zeta, dbb + sizeof(double) * dl.zeta, c.Ks);
  ok = ok && rows_d2h(out->zeta_sic, dbb + sizeof(double) * dl.zsic, size_t(c.M) * p.d.npair, NPp, c.N);
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
