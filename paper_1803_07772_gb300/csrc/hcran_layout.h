// hcran_layout.h -- workspace layout shared by the host planner and the
// device solver (internal; not part of the C ABI).
//
// Every per-subcarrier segment of the solver state is padded to a multiple of
// 16 bytes, so one bulk asynchronous copy (cp.async.bulk) can move it between
// global and shared memory:
//   slot arrays      [n][Up]        Up  = M*l rounded up to 4 floats
//   compact slab     [n][j][Up]     gains of the selected users from RRH j
//   SIC multipliers  [n][NPp]       NPp = M*l(l-1)/2 rounded up to 2 doubles
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define HCRAN_HD __host__ __device__ __forceinline__
#else
#define HCRAN_HD inline
#endif

namespace hcran {

constexpr int kThreads = 512;          // threads per CTA (one CTA solves one instance)
constexpr int kWarps = kThreads / 32;
constexpr int kMaxM = 64;              // RRHs per instance
constexpr int kMaxL = 8;               // NOMA users per (RRH, subcarrier)
constexpr int kMaxU = 256;             // slots per subcarrier, M * l
constexpr int kMaxItems = kMaxM * kMaxL * (kMaxL - 1) / 2;  // SIC pairs per subcarrier
constexpr int kMaxDynSmem = 216 * 1024;

HCRAN_HD int64_t al4(int64_t x) { return (x + 3) & ~int64_t(3); }
HCRAN_HD int64_t al2(int64_t x) { return (x + 1) & ~int64_t(1); }

// slots per subcarrier rounded up to 4 floats (row stride of slot arrays and slab)
HCRAN_HD int slot_stride(int M, int l) { return int(al4(int64_t(M) * l)); }
// SIC multipliers per subcarrier rounded up to 2 doubles
HCRAN_HD int pair_stride(int M, int l) {
  const int np = l * (l - 1) / 2;
  return int(al2(int64_t(M) * (np > 0 ? np : 1)));
}

// per-instance descriptor (device copy lives at the start of the workspace)
struct InstDesc {
  int32_t M, N, K, Ks, l, U, L, npair, nchunk;
  int32_t start;   // 0: the cold initial point p^0; 1: the state hcran_set_state wrote (next solve only)
  int64_t g_off;   // element offset of Gamma[n][m][k] in the gain buffer
  int64_t d_off;   // element offset in the double arena
  int64_t f_off;   // element offset in the float arena
  int64_t i_off;   // element offset in the int arena
  double sigma;    // noise power per subcarrier, N0 * Bn
  double Pconst;   // sum_m (Pc_m + Pf_m)
  int64_t s_off;   // first row of the instance in the warm-start feature / output arrays
};

// double arena of one instance
struct DLayout {
  int64_t pmax, eta, mask, Psi, Tdel, w, xi, zeta, zsic, zsic_next, xi_prev, zeta_prev, zsic_prev, total;
};
HCRAN_HD DLayout dlayout(int M, int N, int K, int Ks, int l) {
  DLayout d;
  int64_t o = 0;
  const int64_t NZ = int64_t(N) * pair_stride(M, l);
  d.pmax = o; o = al4(o + M);
  d.eta = o; o = al4(o + M);
  d.mask = o; o = al4(o + M);
  d.Psi = o; o = al4(o + (Ks > 0 ? Ks : 1));
  d.Tdel = o; o = al4(o + (Ks > 0 ? Ks : 1));
  d.w = o; o = al4(o + int64_t(M) * K);
  d.xi = o; o = al4(o + M);
  d.zeta = o; o = al4(o + (Ks > 0 ? Ks : 1));
  d.zsic = o; o = al4(o + NZ);
  d.zsic_next = o; o = al4(o + NZ);
  d.xi_prev = o; o = al4(o + M);                      // the previous Dinkelbach iterate
  d.zeta_prev = o; o = al4(o + (Ks > 0 ? Ks : 1));
  d.zsic_prev = o; o = al4(o + NZ);
  d.total = o;
  return d;
}

HCRAN_HD int nchunk_for(int N, int K) {
  int c = kThreads / (K > 0 ? K : 1);
  if (c < 1) c = 1;
  if (c > N) c = N;
  return c;
}
// room for candidate-utility chunks in the float arena: enough for any
// cluster size of the schedule (class_nchunk <= nchunk_cap), so that the
// arena layout does not depend on the schedule
HCRAN_HD int nchunk_cap(int N, int K) {
  const int c = nchunk_for(N, K);
  return c > 8 ? c : 8;
}

// float arena of one instance (slot arrays are [n][Up])
struct FLayout {
  int64_t p, plin, pstart, alpha, beta, pi, gam, X, Aden, Bnum, Cnum, gown, ginv, wslot, slab, SICp, SICm,
      Ptot, cu, cp, cX, ckey, Upart, wf, p_prev, alpha_prev, beta_prev, total;
};
HCRAN_HD FLayout flayout(int M, int N, int K, int l, int nchunk) {  // nchunk: capacity (nchunk_cap)
  FLayout f;
  int64_t o = 0;
  const int64_t L = int64_t(N) * slot_stride(M, l);
  const int64_t NM = int64_t(N) * M, NK = int64_t(N) * K;
  f.p = o; o = al4(o + L);
  f.plin = o; o = al4(o + L);
  f.pstart = o; o = al4(o + L);
  f.alpha = o; o = al4(o + L);
  f.beta = o; o = al4(o + L);
  f.pi = o; o = al4(o + L);
  f.gam = o; o = al4(o + L);
  f.X = o; o = al4(o + L);
  f.Aden = o; o = al4(o + L);
  f.Bnum = o; o = al4(o + L);
  f.Cnum = o; o = al4(o + L);
  f.gown = o; o = al4(o + L);
  f.ginv = o; o = al4(o + L);
  f.wslot = o; o = al4(o + L);
  f.slab = o; o = al4(o + NM * slot_stride(M, l));
  f.SICp = o; o = al4(o + NM);
  f.SICm = o; o = al4(o + NM);
  f.Ptot = o; o = al4(o + NM);
  f.cu = o; o = al4(o + NK);
  f.cp = o; o = al4(o + NK);
  f.cX = o; o = al4(o + NK);
  f.ckey = o; o = al4(o + NK);
  f.Upart = o; o = al4(o + int64_t(nchunk) * M * K);
  f.wf = o; o = al4(o + int64_t(M) * K);
  f.p_prev = o; o = al4(o + L);                        // the previous Dinkelbach iterate
  f.alpha_prev = o; o = al4(o + L);
  f.beta_prev = o; o = al4(o + L);
  f.total = o;
  return f;
}

// int arena of one instance: serving RRHs, slot users, the user -> slot map,
// the selection being built (Snew), the RRH of largest summed gain of every
// user (Again), the per-CTA served flags of the streaming users (srv), and
// the previous Dinkelbach iterate (A_prev, S_prev)
struct ILayout {
  int64_t A, Anew, S, uslot, Snew, Again, srv, A_prev, S_prev, total;
};
HCRAN_HD ILayout ilayout(int M, int N, int K, int Ks, int l) {
  ILayout i;
  int64_t o = 0;
  const int64_t L = int64_t(N) * slot_stride(M, l);
  i.A = o; o = al4(o + K);
  i.Anew = o; o = al4(o + K);
  i.S = o; o = al4(o + L);
  i.uslot = o; o = al4(o + int64_t(K) * N);
  i.Snew = o; o = al4(o + L);
  i.Again = o; o = al4(o + K);
  i.srv = o; o = al4(o + int64_t(8) * (Ks > 0 ? Ks : 1));
  i.A_prev = o; o = al4(o + K);
  i.S_prev = o; o = al4(o + L);
  i.total = o;
  return i;
}


// per-instance scalar outputs
struct InstOut {
  double ee, R, P, slack_power_min, slack_rate_min, slack_sic_max, min_margin;
  int32_t iters[3];
  int32_t status, n_ties;
  int64_t cycles[8];   // SM clock cycles per phase: selection, link, multipliers, power, scale, dinkelbach, total, pad
};

// Largest shapes of a launch; they size the per-warp shared buffers.
struct KDims {
  int Upmax;    // max slot stride
  int Mmax;     // max RRHs
  int NPmax;    // max pairs per (m, n)
  int NPPmax;   // max pair stride per subcarrier (doubles)
  int KSmax;    // max streaming users
  int staged;   // 1: per-subcarrier state double-buffered in shared memory by bulk copies
  int resident; // 1: the dual loop keeps the CTA's subcarrier state in shared memory
  int res_floats;  // resident region (floats), the largest instance of the launch
  int teams;    // > 0: the sweeps run on this many teams of kWarps / teams warps, one
                // subcarrier per team at a time, each team double-buffering its
                // subcarriers' state by bulk copies (needs staged = 1)
};
// per-warp working buffers (floats)
HCRAN_HD int warp_work_floats(const KDims &k) {
  return 4 * k.Upmax + 6 * k.Mmax + 2 * k.Mmax * (k.NPmax > 0 ? k.NPmax : 1) + 32 +
         2 * (k.KSmax > 0 ? k.KSmax : 1);
}
// one staging buffer (floats, 16-byte multiple): SIC multipliers (doubles),
// slab rows, then the slot arrays k, p, Aden, Bnum, Cnum, alpha, beta, plin,
// own gain and its reciprocal, priority weight w_{m,k} of the slot's link
constexpr int kStagedArrays = 11;
HCRAN_HD int stage_buf_floats(const KDims &k) {
  return 2 * k.NPPmax + k.Mmax * k.Upmax + kStagedArrays * k.Upmax;
}
HCRAN_HD int warp_buf_floats(const KDims &k) {
  return int(al4(warp_work_floats(k))) + (k.staged ? 2 * stage_buf_floats(k) : 0);
}
// Team sweeps: a team of kWarps / teams warps works on one subcarrier at a
// time.  Per team: the two staging buffers; slot arrays p, pi, X, k [Upmax];
// a compact list of the nonzero SIC multipliers (two weights, two slots)
// [Mmax * NPmax]; per-RRH totals, price sums, SIC+, SIC-, power partials
// [Mmax]; the SIC multipliers of the subcarrier [Mmax * NPmax]; three partial
// sums per thread; the streaming rate and alpha partials [KSmax]; a counter.
HCRAN_HD int team_threads(const KDims &k) { return (kWarps / (k.teams > 0 ? k.teams : 1)) * 32; }
HCRAN_HD int team_work_floats(const KDims &k) {
  const int np = k.NPmax > 0 ? k.NPmax : 1;
  return int(al4(4 * k.Upmax + 5 * k.Mmax + 5 * k.Mmax * np + 3 * team_threads(k) +
                 2 * (k.KSmax > 0 ? k.KSmax : 1) + 4));
}
HCRAN_HD int team_stride(const KDims &k) { return team_work_floats(k) + 2 * stage_buf_floats(k); }
// Resident dual loop: shared-memory state of Nc subcarriers (structure of
// arrays): slab [Nc][M][Rs] (row stride Rs = Up, or Up + 4 when Up / 4 is
// even, so that lanes reading consecutive rows as float4 hit distinct banks);
// slot arrays k, p, pi, g_own, 1/g_own, w*alpha, alpha, w*beta, p_lin, X
// [Nc][Up]; per-RRH totals, price sums, SIC+ and SIC- [Nc][M]; SIC
// multipliers as (hi, lo) float pairs in two generations [Nc][M*npair]; the
// nonzero-multiplier bit masks [Nc][ceil(M*npair/32)]; the streaming rate and
// alpha contributions [Nc][Ks].
HCRAN_HD int res_row_stride(int M, int l) {
  const int Up = slot_stride(M, l);
  return ((Up / 4) & 1) ? Up : Up + 4;
}
constexpr int kResSlotArrays = 10;
HCRAN_HD int64_t res_floats(int M, int l, int Ks, int Nc) {
  const int64_t Up = slot_stride(M, l), Mi = int64_t(M) * (l * (l - 1) / 2);
  const int64_t NW = (Mi + 31) / 32;
  return int64_t(Nc) * M * res_row_stride(M, l) + kResSlotArrays * int64_t(Nc) * Up +
         4 * al4(int64_t(Nc) * M) + 4 * al4(int64_t(Nc) * Mi) + al4(int64_t(Nc) * NW) +
         2 * al4(int64_t(Nc) * Ks);
}
// resident scratch: the CTA's residual vector (two parities, read by the
// other CTAs of its cluster), the multipliers xi', zeta' of the CTA as FP32
// pairs, and the constants of their steps (pmax_m, 1 / (ln2 mask_m pmax_m),
// Psi_k)
HCRAN_HD int res_xch_floats(const KDims &k) {
  return int(al4(k.Mmax + 2 * (k.KSmax > 0 ? k.KSmax : 1) + 2));
}
HCRAN_HD int res_scratch_floats(const KDims &k) {
  const int m4 = int(al4(k.Mmax)), s4 = int(al4(k.KSmax > 0 ? k.KSmax : 1));
  return 2 * res_xch_floats(k) + 2 * m4 + 2 * s4 + 2 * m4 + s4;
}
// Dynamic shared memory: streaming multipliers zeta' (FP32), the resident
// scratch, then one region that holds either the per-warp buffers of the
// other phases or, during a dual loop, the resident state.
HCRAN_HD int64_t dyn_head_floats(const KDims &k) {
  return al4(k.KSmax > 0 ? k.KSmax : 1) + (k.resident ? res_scratch_floats(k) : 0);
}
HCRAN_HD int warp_stride(const KDims &k) { return warp_buf_floats(k); }
HCRAN_HD int64_t dyn_smem_bytes(const KDims &k) {
  const int64_t w = k.teams > 0 ? int64_t(k.teams) * team_stride(k) : int64_t(kWarps) * warp_stride(k);
  const int64_t r = k.resident ? int64_t(k.res_floats) : 0;
  return 4 * (dyn_head_floats(k) + (w > r ? w : r));
}

// Schedule of a launch: the resident dual loop when the largest instance's
// state fits shared memory; else bulk-copy staging of each subcarrier, by
// every warp when its double buffers fit, else by as many teams of warps
// (4, 3, 2, 1) as fit; else global reads.  Returns nonzero when even the
// per-warp buffers do not fit.
inline int plan_kdims(KDims &k, int64_t res_need) {
  k.staged = 0;
  k.teams = 0;
  k.resident = 1;
  k.res_floats = int(res_need < (int64_t(1) << 30) ? res_need : (int64_t(1) << 30));
  if (dyn_smem_bytes(k) <= kMaxDynSmem) return 0;
  k.resident = 0;
  k.res_floats = 0;
  k.staged = 1;
  if (dyn_smem_bytes(k) <= kMaxDynSmem) return 0;
  for (int t = 4; t >= 1; t--) {
    k.teams = t;
    if (dyn_smem_bytes(k) <= kMaxDynSmem) return 0;
  }
  k.teams = 0;
  k.staged = 0;
  return dyn_smem_bytes(k) <= kMaxDynSmem ? 0 : 1;
}

// Launch dimensions for one instance of shape (M, l, Ks, N) solved with the
// resident dual loop by clusters of C CTAs (each CTA holds ceil(N / C)
// subcarriers).
inline KDims resident_kdims(int M, int l, int Ks, int N, int C) {
  KDims k;
  k.Upmax = slot_stride(M, l);
  k.Mmax = M;
  k.NPmax = l * (l - 1) / 2;
  k.NPPmax = pair_stride(M, l);
  k.KSmax = Ks;
  k.staged = 0;
  k.teams = 0;
  k.resident = 1;
  const int64_t r = res_floats(M, l, Ks, (N + C - 1) / C);
  k.res_floats = int(r < (int64_t(1) << 30) ? r : (int64_t(1) << 30));
  return k;
}
// dimensions of a launch that holds the instances of a and of b
inline void kdims_merge(KDims &a, const KDims &b) {
  a.Upmax = a.Upmax > b.Upmax ? a.Upmax : b.Upmax;
  a.Mmax = a.Mmax > b.Mmax ? a.Mmax : b.Mmax;
  a.NPmax = a.NPmax > b.NPmax ? a.NPmax : b.NPmax;
  a.NPPmax = a.NPPmax > b.NPPmax ? a.NPPmax : b.NPPmax;
  a.KSmax = a.KSmax > b.KSmax ? a.KSmax : b.KSmax;
  a.res_floats = a.res_floats > b.res_floats ? a.res_floats : b.res_floats;
}
// Launch classes: class k < kMaxCluster holds the instances solved by
// clusters of kMaxCluster - k CTAs (largest first); class kNumClasses - 1 is
// the streamed schedule (one CTA, subcarrier state staged from global memory)
// for instances whose resident state fits no cluster.
constexpr int kMaxCluster = 8;  // portable cluster size limit
constexpr int kNumClasses = kMaxCluster + 1;
HCRAN_HD int class_csize(int cls) { return cls < kMaxCluster ? kMaxCluster - cls : 1; }
HCRAN_HD int class_of(int C) { return kMaxCluster - C; }
// margin kept free for the per-launch maxima of the other instances of a class
constexpr int kClassMargin = 4096;
// SM cycles of one resident dual iteration on a CTA that holds g (n, m)
// groups, measured on GB300 over the uneven batch: about 7000 + 6 g while
// every thread holds at most one group (the stages are bound by the latency
// of a group's chain, not by the number of groups), and about 3400 more for
// each further group per thread.
inline double res_iter_cycles(int64_t g) {
  const int64_t per = (g + kThreads - 1) / kThreads;
  return 7000.0 + 6.0 * double(g < kThreads ? g : kThreads) + 3400.0 * double(per > 1 ? per - 1 : 0);
}
// launch class of one instance: among the cluster sizes whose resident state
// fits, the one with the fewest SM cycles per dual iteration, C times the
// cycles of a CTA holding ceil(N / C) M groups (ties: the smaller cluster);
// the streamed class when none fits
inline int pick_class(int M, int l, int Ks, int N) {
  int best = kNumClasses - 1;
  double best_cost = 0.0;
  for (int C = 1; C <= kMaxCluster && C <= N; C++) {
    if (dyn_smem_bytes(resident_kdims(M, l, Ks, N, C)) > kMaxDynSmem - kClassMargin) continue;
    const double cost = C * res_iter_cycles(int64_t((N + C - 1) / C) * M);
    if (best == kNumClasses - 1 || cost < best_cost) {
      best = class_of(C);
      best_cost = cost;
    }
  }
  return best;
}
// candidate-utility chunks of an instance solved by clusters of C CTAs: a
// multiple of C, so that every CTA sums chunks of its own subcarriers
HCRAN_HD int class_nchunk(int N, int K, int C) {
  int per = nchunk_for(N, K) / C;
  if (per < 1) per = 1;
  return per * C;
}

// What a launch does with each instance: the whole solve from the cold
// initial point, only the initial selection and the warm-start features of
// its slots, or the whole solve from the network's warm start.
enum SolveMode { kModeCold = 0, kModeFeatures = 1, kModeWarm = 2 };

struct Tol {
  double tol_dinkelbach, tol_scale, tol_dual;
  int32_t max_dinkelbach, max_scale, max_dual;
  float tie_eps;
  double q_init;
  int32_t mode;  // SolveMode
  int64_t spin_limit;      // tries of every bounded mbarrier wait (<= 0: the default)
  int32_t stall_instance;  // instance whose solve first waits on a barrier nothing completes (-1: none)
};

// warm-start rows (one per slot: row s_off + n * Up + u): the features the
// features mode writes ([rows][16] BF16) and the network outputs the warm mode
// reads ([rows][16] FP32)
struct WarmIO {
  const float *out;
  void *feat;
};

// region offsets (bytes) inside the workspace
struct WsLayout {
  uint64_t descs, order, counter, outs, darena, farena, iarena, staging, total;
};

}  // namespace hcran
