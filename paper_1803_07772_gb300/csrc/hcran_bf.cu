// hcran_bf.cu -- global-optimum comparator: the best energy efficiency of a
// small instance over every assignment, on the GPU.
//
// The paper measures its method against the optimum it finds by monotonic
// optimisation (Sec. IV-B).  Here the optimum of small instances (elastic
// users only) is found by enumeration: every RRH choice A_k in {-1 .. M-1}
// and, on every (n, m), every subset of the users of m of at most l members,
// with every user that has an RRH on at least one link.  For each assignment
// the EE = R / P (R over every link, P of the Sec. II-A power model) is
// maximised over the powers by coordinate golden-section search in
// [1e-6 mask, mask] from three starts p = f mask (f = 0.1, 0.4, 1): 8 sweeps
// over the links, 40 golden-section steps per link (the upper end moves when
// the lower point is at least as good), the midpoint kept when it improves.
// A point that breaks C12 (an RRH's total above pmax) or C14 (Omega_bar > 0
// for a pair of one (m, n) in SIC order) has value -1.
//
// One thread searches one (instance, assignment); a second kernel takes, per
// instance, the largest value (the lowest assignment index on equal values).
// The search is sequential arithmetic on a handful of links, ALU-bound and
// run in FP64 (this file is compiled without FMA contraction, so its
// operation order is the one written here).  The assignment table is built
// on the host in the enumeration order documented in include/hcran.h.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <vector>

#include "../../include/hcran.h"

namespace {

constexpr int kBfMaxLinks = 16;
constexpr int kBfSweeps = 8, kBfGolden = 40;
constexpr int kBfThreads = 128;

struct BfShape {
  int M, N, K, l;
  int64_t n_assign;
  int64_t g_stride;  // gain elements per instance (N M K rounded up to 4)
  int c_stride;      // doubles of constants per instance
};

// constants of one instance: pmax[M], eta[M], mask[M], w[M*K], then Pconst, sigma
__device__ __forceinline__ bool bf_stronger(const float *G, int M, int K, int n, int m, int a, int b) {
  const double ga = (double)G[((size_t)n * M + m) * K + a], gb = (double)G[((size_t)n * M + m) * K + b];
  return ga > gb || (ga == gb && a < b);
}

__device__ double bf_value(const BfShape &s, const float *G, const double *c, const unsigned char *L, int nl,
                           const double *p) {
  const int M = s.M, K = s.K;
  const double *pmax = c, *eta = c + M, *w = c + 3 * M;
  const double Pconst = c[3 * M + M * K], sigma = c[3 * M + M * K + 1];
  double tot[8];
  for (int m = 0; m < M; m++) tot[m] = 0.0;
  for (int j = 0; j < nl; j++) tot[L[3 * j + 1]] += p[j];
  for (int m = 0; m < M; m++)
    if (tot[m] > pmax[m] * (1.0 + 1e-12)) return -1.0;
  double R = 0.0, P = Pconst;
  for (int j = 0; j < nl; j++) {
    const int an = L[3 * j], am = L[3 * j + 1], ak = L[3 * j + 2];
    double intra = 0.0, inter = 0.0;
    for (int i = 0; i < nl; i++) {
      const int bn = L[3 * i], bm = L[3 * i + 1], bk = L[3 * i + 2];
      if (bn != an) continue;
      if (bm == am) {
        if (i != j && bf_stronger(G, M, K, an, am, bk, ak)) intra += p[i];
        if (i != j && bf_stronger(G, M, K, an, am, ak, bk)) {  // C14 for (stronger a, weaker b)
          double xa = 0.0, xb = 0.0;
          for (int q = 0; q < nl; q++) {
            const int tn = L[3 * q], tm = L[3 * q + 1];
            if (tn != an || tm == am) continue;
            xa += (double)G[((size_t)an * M + tm) * K + ak] * p[q];
            xb += (double)G[((size_t)an * M + tm) * K + bk] * p[q];
          }
          if ((sigma + xa) / (double)G[((size_t)an * M + am) * K + ak] -
                  (sigma + xb) / (double)G[((size_t)an * M + am) * K + bk] >
              0.0)
            return -1.0;
        }
      } else {
        inter += (double)G[((size_t)an * M + bm) * K + ak] * p[i];
      }
    }
    const double g = (double)G[((size_t)an * M + am) * K + ak];
    R += w[(size_t)am * K + ak] * log2(1.0 + p[j] * g / (sigma + g * intra + inter));
    P += eta[am] * p[j];
  }
  return R / P;
}

__global__ void __launch_bounds__(kBfThreads) bf_kernel(BfShape s, int n_inst, const float *gains,
                                                        const double *consts, const unsigned char *table,
                                                        double *values) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n_inst * s.n_assign) return;
  const int b = (int)(t / s.n_assign);
  const int64_t a = t - (int64_t)b * s.n_assign;
  const float *G = gains + (size_t)b * s.g_stride;
  const double *c = consts + (size_t)b * s.c_stride;
  const unsigned char *row = table + (size_t)a * (1 + 3 * kBfMaxLinks);
  const int nl = row[0];
  const unsigned char *L = row + 1;
  const double *mask = c + 2 * s.M;
  const double gr = (sqrt(5.0) - 1.0) / 2.0;
  const double starts[3] = {0.1, 0.4, 1.0};
  double best = -1.0, p[kBfMaxLinks], q[kBfMaxLinks];
  for (int st = 0; st < 3; st++) {
    for (int j = 0; j < nl; j++) p[j] = starts[st] * mask[L[3 * j + 1]];
    double cur = bf_value(s, G, c, L, nl, p);
    if (cur < 0.0) continue;
    for (int sw = 0; sw < kBfSweeps; sw++)
      for (int j = 0; j < nl; j++) {
        const double mk = mask[L[3 * j + 1]];
        double lo = 1e-6 * mk, hi = mk;
        for (int i = 0; i < nl; i++) q[i] = p[i];
        for (int it = 0; it < kBfGolden; it++) {
          const double x = hi - gr * (hi - lo), y = lo + gr * (hi - lo);
          q[j] = x;
          const double vx = bf_value(s, G, c, L, nl, q);
          q[j] = y;
          const double vy = bf_value(s, G, c, L, nl, q);
          if (vx >= vy) hi = y;
          else lo = x;
        }
        q[j] = 0.5 * (lo + hi);
        const double vn = bf_value(s, G, c, L, nl, q);
        if (vn > cur) {
          p[j] = q[j];
          cur = vn;
        }
      }
    if (cur > best) best = cur;
  }
  values[t] = best;
}

// per instance: the largest value above 0 and the lowest assignment index that has it
__global__ void __launch_bounds__(256) bf_reduce(int64_t n_assign, const double *values, double *best_ee,
                                                  int64_t *best_index) {
  __shared__ double sv[256];
  __shared__ int64_t si[256];
  const double *v = values + (size_t)blockIdx.x * n_assign;
  double bv = 0.0;
  int64_t bi = -1;
  for (int64_t a = threadIdx.x; a < n_assign; a += blockDim.x)
    if (v[a] > bv) {  // increasing a: the first (lowest) index keeps equal values
      bv = v[a];
      bi = a;
    }
  sv[threadIdx.x] = bv;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      const double ov = sv[threadIdx.x + o];
      const int64_t oi = si[threadIdx.x + o];
      if (oi >= 0 && (si[threadIdx.x] < 0 || ov > sv[threadIdx.x] ||
                      (ov == sv[threadIdx.x] && oi < si[threadIdx.x]))) {
        sv[threadIdx.x] = ov;
        si[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    best_ee[blockIdx.x] = sv[0];
    best_index[blockIdx.x] = si[0];
  }
}

// ------------------------------------------------------------------ host

int64_t al4(int64_t x) { return (x + 3) & ~int64_t(3); }
uint64_t al256(uint64_t x) { return (x + 255) & ~uint64_t(255); }

bool finite_pos(double x) { return x > 0.0 && x < INFINITY; }

// the assignment table in the enumeration order of include/hcran.h
void enumerate(int M, int N, int K, int l, std::vector<unsigned char> &table, int64_t &count) {
  const int NM = N * M, row = 1 + 3 * kBfMaxLinks;
  table.clear();
  count = 0;
  int64_t nA = 1;
  for (int k = 0; k < K; k++) nA *= (M + 1);
  std::vector<std::vector<std::vector<int>>> subs(NM);
  for (int64_t a = 0; a < nA; a++) {
    int A[8];
    int64_t r = a;
    for (int k = 0; k < K; k++) {
      A[k] = (int)(r % (M + 1)) - 1;
      r /= (M + 1);
    }
    int64_t nch = 1;
    for (int nm = 0; nm < NM; nm++) {
      const int m = nm % M;
      std::vector<int> users;
      for (int k = 0; k < K; k++)
        if (A[k] == m) users.push_back(k);
      subs[nm].clear();
      const int cnt = (int)users.size();
      for (int sz = 0; sz <= (cnt < l ? cnt : l); sz++) {  // by size, then lexicographic
        std::vector<int> comb(sz);
        for (int i = 0; i < sz; i++) comb[i] = i;
        for (;;) {
          std::vector<int> s(sz);
          for (int i = 0; i < sz; i++) s[i] = users[comb[i]];
          subs[nm].push_back(s);
          int i = sz - 1;
          while (i >= 0 && comb[i] == cnt - sz + i) i--;
          if (i < 0) break;
          comb[i]++;
          for (int j = i + 1; j < sz; j++) comb[j] = comb[j - 1] + 1;
        }
      }
      nch *= (int64_t)subs[nm].size();
    }
    for (int64_t ch = 0; ch < nch; ch++) {
      std::vector<int> digit(NM);
      int64_t rr = ch;
      for (int nm = NM - 1; nm >= 0; nm--) {  // the last (n, m) varies fastest
        digit[nm] = (int)(rr % (int64_t)subs[nm].size());
        rr /= (int64_t)subs[nm].size();
      }
      unsigned char rec[1 + 3 * kBfMaxLinks] = {0};
      int nl = 0;
      bool served[8] = {false};
      for (int nm = 0; nm < NM; nm++)
        for (int k : subs[nm][digit[nm]]) {
          rec[1 + 3 * nl] = (unsigned char)(nm / M);
          rec[2 + 3 * nl] = (unsigned char)(nm % M);
          rec[3 + 3 * nl] = (unsigned char)k;
          served[k] = true;
          nl++;
        }
      bool ok = nl > 0;
      for (int k = 0; k < K && ok; k++)
        if (A[k] >= 0 && !served[k]) ok = false;
      if (!ok) continue;
      rec[0] = (unsigned char)nl;
      table.insert(table.end(), rec, rec + row);
      count++;
    }
  }
}

int check_cfgs(const hcran_config *cfgs, int32_t n, BfShape &s) {
  if (!cfgs || n < 1) return HCRAN_EINVAL;
  const hcran_config &c0 = cfgs[0];
  s.M = c0.M; s.N = c0.N; s.K = c0.K; s.l = c0.l;
  if (s.M < 1 || s.M > 8 || s.N < 1 || s.K < 1 || s.K > 6 || s.l < 1 || s.l > 3 || s.N * s.M * s.l > kBfMaxLinks)
    return HCRAN_EINVAL;
  for (int32_t b = 0; b < n; b++) {
    const hcran_config &c = cfgs[b];
    if (c.M != s.M || c.N != s.N || c.K != s.K || c.l != s.l || c.Ks != 0) return HCRAN_EINVAL;
    if (!c.pmax || !c.eta || !c.Pc || !c.Pf || !finite_pos(c.Bn_hz) || !finite_pos(c.N0_w_per_hz))
      return HCRAN_EINVAL;
    for (int m = 0; m < s.M; m++)
      if (!finite_pos(c.pmax[m]) || !finite_pos(c.eta[m]) || !(c.Pc[m] >= 0.0) || !(c.Pf[m] >= 0.0) ||
          !(c.Pc[m] < INFINITY) || !(c.Pf[m] < INFINITY))
        return HCRAN_EINVAL;
    if (c.w)
      for (int t = 0; t < s.M * s.K; t++)
        if (!(c.w[t] >= 0.0 && c.w[t] <= 1.0)) return HCRAN_EINVAL;
  }
  s.g_stride = al4((int64_t)s.N * s.M * s.K);
  s.c_stride = 3 * s.M + s.M * s.K + 2;
  return HCRAN_OK;
}

struct BfLayout {
  uint64_t consts, table, values, ee, idx, total;
};
BfLayout bf_layout(const BfShape &s, int32_t n) {
  BfLayout L;
  uint64_t o = 0;
  L.consts = o; o = al256(o + sizeof(double) * (uint64_t)s.c_stride * n);
  L.table = o; o = al256(o + (uint64_t)s.n_assign * (1 + 3 * kBfMaxLinks));
  L.values = o; o = al256(o + sizeof(double) * (uint64_t)s.n_assign * n);
  L.ee = o; o = al256(o + sizeof(double) * n);
  L.idx = o; o = al256(o + sizeof(int64_t) * n);
  L.total = o;
  return L;
}

}  // namespace

extern "C" int hcran_bf_workspace_size(const hcran_config *cfgs, int32_t n, uint64_t *bytes, int64_t *n_assign) {
  BfShape s;
  if (!bytes || check_cfgs(cfgs, n, s) != HCRAN_OK) return HCRAN_EINVAL;
  std::vector<unsigned char> table;
  enumerate(s.M, s.N, s.K, s.l, table, s.n_assign);
  *bytes = bf_layout(s, n).total;
  if (n_assign) *n_assign = s.n_assign;
  return HCRAN_OK;
}

extern "C" int hcran_bruteforce(const hcran_config *cfgs, int32_t n, const float *gains_dev, void *workspace_dev,
                                void *stream, double *best_ee, int64_t *best_index) {
  BfShape s;
  if (!gains_dev || !workspace_dev || !best_ee || (reinterpret_cast<uintptr_t>(gains_dev) & 15) ||
      (reinterpret_cast<uintptr_t>(workspace_dev) & 255) || check_cfgs(cfgs, n, s) != HCRAN_OK)
    return HCRAN_EINVAL;
  std::vector<unsigned char> table;
  enumerate(s.M, s.N, s.K, s.l, table, s.n_assign);
  if (s.n_assign < 1) return HCRAN_EINVAL;
  const BfLayout L = bf_layout(s, n);
  std::vector<double> consts((size_t)s.c_stride * n);
  for (int32_t b = 0; b < n; b++) {
    const hcran_config &c = cfgs[b];
    double *d = consts.data() + (size_t)b * s.c_stride;
    double pc = 0.0;
    for (int m = 0; m < s.M; m++) {
      d[m] = c.pmax[m];
      d[s.M + m] = c.eta[m];
      d[2 * s.M + m] = c.pmax[m] / s.N;
      pc += c.Pc[m] + c.Pf[m];
    }
    for (int t = 0; t < s.M * s.K; t++) d[3 * s.M + t] = c.w ? c.w[t] : 1.0;
    d[3 * s.M + s.M * s.K] = pc;
    d[3 * s.M + s.M * s.K + 1] = c.N0_w_per_hz * c.Bn_hz;
  }
  char *ws = static_cast<char *>(workspace_dev);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // pageable sources: staged before each call returns
  if (cudaMemcpyAsync(ws + L.consts, consts.data(), sizeof(double) * consts.size(), cudaMemcpyHostToDevice, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(ws + L.table, table.data(), table.size(), cudaMemcpyHostToDevice, st) != cudaSuccess)
    return HCRAN_ECUDA;
  const int64_t threads = (int64_t)n * s.n_assign;
  const unsigned blocks = (unsigned)((threads + kBfThreads - 1) / kBfThreads);
  bf_kernel<<<blocks, kBfThreads, 0, st>>>(s, n, gains_dev, reinterpret_cast<const double *>(ws + L.consts),
                                           reinterpret_cast<const unsigned char *>(ws + L.table),
                                           reinterpret_cast<double *>(ws + L.values));
  bf_reduce<<<n, 256, 0, st>>>(s.n_assign, reinterpret_cast<const double *>(ws + L.values),
                               reinterpret_cast<double *>(ws + L.ee), reinterpret_cast<int64_t *>(ws + L.idx));
  if (cudaGetLastError() != cudaSuccess) return HCRAN_ECUDA;
  if (cudaMemcpyAsync(best_ee, ws + L.ee, sizeof(double) * n, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      (best_index &&
       cudaMemcpyAsync(best_index, ws + L.idx, sizeof(int64_t) * n, cudaMemcpyDeviceToHost, st) != cudaSuccess) ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return HCRAN_ECUDA;
  return HCRAN_OK;
}
