/*
 * hcran.h -- C ABI of the GB300 (sm_103a) solver for energy-efficient
 * resource allocation in PD-NOMA H-CRANs (arXiv 1803.07772).
 *
 * One call solves a batch of independent channel realisations ("instances")
 * of problem (eq7): maximise the elastic users' energy efficiency
 * E = R(p)/P(p) over RRH selection, subcarrier/NOMA selection and transmit
 * powers, subject to the power budgets (C12), spectral masks (C4), the
 * delay-derived minimum rates of the streaming users (C9/C13) and SIC
 * feasibility (C14).  The method is the paper's: the Dinkelbach iteration of
 * Sec. III (Theorem 1, Prop. 1) around Algorithm 1 of Sec. IV-A (SCALE lower
 * bound of eq. scale_approximation, log-power change of variable, closed-form
 * KKT powers of eq. (653)/(683), projected subgradient multipliers).
 *
 * Conventions
 *  - Every function returns an hcran_status code; nothing aborts or prints.
 *  - Gains are float32 Gamma[n][m][k] = |h_{m,k}^{(n)}|^2 (k fastest), one
 *    slab per instance, inside one device buffer.  Instance b starts at
 *    element gain_offsets[b] (given at create time, must be a multiple of 4).
 *  - All device memory is owned by the caller: the solver works inside one
 *    workspace buffer of hcran_workspace_size() bytes (256-byte aligned),
 *    which the caller allocates (e.g. with PyTorch) and keeps alive while any
 *    call that uses it is in flight.  The library allocates no device memory.
 *  - Calls that take a stream only enqueue work on it; hcran_get* synchronise
 *    that stream before copying results to the caller's host arrays.
 *  - Arithmetic: SINR, power, prices and subgradient residuals in FP32;
 *    the multipliers accumulate their subgradient steps as unevaluated
 *    float pairs (about 48 significant bits) and are stored in FP64;
 *    Dinkelbach ratio q = R/P and the F(q) test in FP64.
 */
#ifndef HCRAN_H
#define HCRAN_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HCRAN_OK = 0,
  HCRAN_EINVAL = 1,    /* bad argument (sizes, NULL, NaN/negative constants, misaligned offset) */
  HCRAN_ENOMEM = 2,    /* host allocation failed or workspace too small */
  HCRAN_ECUDA = 3,     /* a CUDA runtime call failed (launch, copy, sync) */
  HCRAN_ETIMEDOUT = 4, /* a bounded device wait gave up (hcran_get, hcran_solve_host) */
  HCRAN_ENUMERIC = 5,  /* a non-finite or negative gain, or NaN/Inf in the Dinkelbach ratio */
  HCRAN_E2BIG = 6      /* the instance does not fit the fixed scratch of hcran_solve_noalloc */
} hcran_status;

/* per-instance result status bits */
#define HCRAN_ST_NOT_CONVERGED 1   /* Dinkelbach cap reached before F(q) <= tol * R */
#define HCRAN_ST_STREAMING_UNMET 2 /* some streaming user ends below Psi_k (relative slack < -1e-3) */
#define HCRAN_ST_EE_DECREASED 4    /* the output's EE is below an earlier Dinkelbach iterate's (kept for C13) */
#define HCRAN_ST_NUMERIC 8         /* non-finite or negative gain, or non-finite R/P; outputs not valid */
#define HCRAN_ST_TIMEOUT 16        /* a bounded wait for a shared-memory copy gave up; outputs not valid */

typedef struct hcran_s *hcran_t;

/* One instance: the system model of Sec. II-A and the traffic of C7/C9.
 * Copied at create time; the caller keeps ownership of every pointer. */
typedef struct {
  int32_t M;                 /* RRHs, index 0 = HPN (1..64) */
  int32_t N;                 /* subcarriers (>= 1) */
  int32_t K;                 /* users (>= 1); 0..K-Ks-1 elastic, K-Ks..K-1 streaming */
  int32_t Ks;                /* streaming users (0..K) */
  int32_t l;                 /* NOMA users per subcarrier and RRH, C1 (1..8); M*l <= 256 */
  const double *pmax;        /* [M] W, per-RRH budget (C12); mask = pmax/N (C4) */
  const double *eta;         /* [M] power-amplifier factor (> 0) */
  const double *Pc;          /* [M] W circuit power (>= 0) */
  const double *Pf;          /* [M] W fronthaul power (>= 0) */
  double Bn_hz;              /* subcarrier bandwidth (> 0) */
  double N0_w_per_hz;        /* noise PSD (> 0); sigma = N0 * Bn */
  const double *T_s;         /* [Ks] delay targets (> 0) */
  const double *lambda_pps;  /* [Ks] Poisson arrival rates (> 0) */
  double zbar_bits;          /* packet size (> 0) */
  const double *w;           /* [M*K] priority weights w_{m,k} in [0,1], or NULL (= 1) */
} hcran_config;

/* Stopping rules of Sec. III and Algorithm 1. */
typedef struct {
  double tol_dinkelbach;     /* stop when F(q) <= tol * R */
  double tol_scale;          /* varpi_2: max |p^s - p^{s-1}| / mask */
  double tol_dual;           /* varpi_1: max |p^v - p^{v-1}| / mask */
  int32_t max_dinkelbach, max_scale, max_dual;
  double tie_eps;            /* relative margin under which a selection decision is flagged */
  double q_init;             /* > 0: use this E^1 instead of R(p^0)/P(p^0) (0 = the method's start) */
} hcran_tol;

/* Result of one instance.  Array members are caller-allocated host arrays
 * (NULL = skip); scalars are always written. */
typedef struct {
  int32_t *A;                /* [K] serving RRH per user, -1 = unserved */
  int32_t *S;                /* [N*M*l] users per (n,m) in SIC order (strongest first), -1 = empty */
  float *p;                  /* [N*M*l] W */
  float *alpha, *beta;       /* [N*M*l] SCALE coefficients at the returned point */
  double *xi;                /* [M]  power-budget multipliers */
  double *zeta;              /* [Ks] rate multipliers */
  double *zeta_sic;          /* [N*M*l(l-1)/2] SIC multipliers per (n,m,pair) */
  double ee, R, P;           /* EE = R/P (bits/s/Hz/W), R (bits/s/Hz), P (W) */
  int32_t iters[3];          /* Dinkelbach iterations, SCALE passes, dual iterations */
  int32_t status;            /* HCRAN_ST_* bits */
  double slack_power_min;    /* min_m (pmax - sum p)/pmax */
  double slack_rate_min;     /* min_k (r_k - Psi_k)/Psi_k, exact rates */
  double slack_sic_max;      /* max over selected pairs of Omega_bar/mask (<= 0 feasible) */
  double min_margin;         /* smallest relative margin of a selection decision */
  int32_t n_ties;            /* decisions with margin < tie_eps */
} hcran_result;

/* Plan a batch of n independent instances (host only, no device work).
 * Returns HCRAN_EINVAL for a bad config, or when the largest instance's
 * per-warp shared working buffers (about 4 * (5 M l + 7 M + M l(l-1)/2 + 2 Ks)
 * bytes per warp, 16 warps) exceed 220 KB.  When the per-warp double staging
 * buffers of one subcarrier's state (about 8 * (M*l*(M + 8) + M l(l-1)) bytes
 * per warp) also fit, the dual loop streams that state through shared memory
 * with bulk copies; otherwise it reads it from global memory.
 * gain_offsets[b]: element offset of instance b's gains in the buffer later
 * given to hcran_solve (NULL = packed back to back, each rounded up to 4). */
int hcran_create(hcran_t *out, const hcran_config *cfgs, int32_t n, const int64_t *gain_offsets);

/* Bytes of device workspace the plan needs (constants, state, scratch, results). */
int hcran_workspace_size(hcran_t h, uint64_t *bytes);

/* Total float32 elements the gain buffer must hold. */
int hcran_gain_elems(hcran_t h, int64_t *elems);

/* Upload the plan's constants into the workspace (a host-to-device copy
 * enqueued on `stream`); required once per workspace before hcran_solve. */
int hcran_prepare(hcran_t h, void *workspace_dev, void *stream);

/* Solve every instance: enqueue the persistent solver launch on `stream`.
 * Issues only device work (memset + kernel), so it may be captured in a CUDA
 * graph.  gains_dev and workspace_dev must stay valid until it completes. */
int hcran_solve(hcran_t h, const float *gains_dev, const hcran_tol *tol, void *workspace_dev,
                void *stream);

/* End-to-end form: copies gains from host memory (pinned for overlap) into
 * the workspace's staging area, solves, and copies the per-instance summary
 * (ee, status) back into the caller's host arrays (either may be NULL).
 * Returns after the stream has finished. */
int hcran_solve_host(hcran_t h, const float *gains_host, const hcran_tol *tol, void *workspace_dev,
                     void *stream, double *ee_host, int32_t *status_host);

/* Results.  Both synchronise the stream of the last solve.  hcran_get fills
 * `out` and returns HCRAN_ETIMEDOUT when the instance's status carries
 * HCRAN_ST_TIMEOUT, HCRAN_ENUMERIC when it carries HCRAN_ST_NUMERIC (the
 * other instances of the batch are unaffected); hcran_solve_host returns the
 * same codes when any instance carries them. */
int hcran_get(hcran_t h, int32_t index, hcran_result *out);
int hcran_get_summary(hcran_t h, double *ee, double *R, double *P, int32_t *status,
                      int32_t *iters3, double *min_margin, int32_t *n_ties);

/* Bound of every device wait, and a test of the path that reports a wait
 * that gave up.  The solver's waits on shared-memory copies (mbarrier
 * try-waits) give up after max_tries tries (0 = the default, 2^22), and the
 * instance then ends with HCRAN_ST_TIMEOUT.  stall_instance >= 0 makes the
 * solve of that instance first wait on a barrier that nothing completes (no
 * copy in flight), so that this wait gives up and the instance reports the
 * timeout while the others solve normally; -1 turns it off.  Applies to the
 * following solves of h.  HCRAN_EINVAL for max_tries < 0 or an index out of
 * range. */
int hcran_set_wait_limit(hcran_t h, int64_t max_tries, int32_t stall_instance);

/* Start point of instance `index` for the next hcran_solve / hcran_solve_host
 * (Sec. III: iteration i of the Dinkelbach method starts from p^{i-1} and its
 * multipliers; the outer iteration eq. outer_iterative_algorithm carries them
 * from one iteration to the next).  The next solve starts that instance from
 * `state` (the allocation A, S, p of a hcran_result, as hcran_get returns it,
 * with E^1 = R(p)/P(p)) instead of the cold initial point; the other
 * instances start cold.  Exporting the state of a solve stopped by its
 * Dinkelbach cap (hcran_get) and importing it here continues that solve:
 * the continued solve takes the same steps as an uninterrupted one.
 *  - workspace_dev: the workspace the next solve will use.
 *  - state: host arrays read during the call only; A, S and p are required;
 *    alpha, beta (default 1, 0), xi (0), zeta (1) and zeta_sic (0) may be NULL.
 *  - The state must be an allocation: A_k in [-1, M); on every (n, m) at
 *    most l distinct users, each with A_k = m, packed at the front (-1
 *    after them), in SIC order; powers in [0, pmax_m / N]; xi, zeta_sic >= 0
 *    and zeta in [1e-6, 1e6], all finite.  Otherwise HCRAN_EINVAL and
 *    nothing is written.
 *  - The copies are enqueued on `stream` (pageable sources, staged before
 *    the call returns).  The state applies to one solve; hcran_solve_graph
 *    and hcran_autotune return HCRAN_EINVAL while a state is pending.
 *  - HCRAN_ECUDA if a copy fails. */
int hcran_set_state(hcran_t h, void *workspace_dev, int32_t index, const hcran_result *state, void *stream);

/* Per-instance SM clock cycles spent in each phase of the last solve
 * (cycles[8*b + i]: 0 selection, 1 interference/SINR/prices, 2 multiplier
 * steps, 3 KKT power update, 4 SCALE coefficient update, 5 projection and
 * Dinkelbach update, 6 whole instance, 7 reserved), read by the CTA's first
 * thread with clock64().  Synchronises the stream of the last solve. */
int hcran_get_phase_cycles(hcran_t h, int64_t *cycles);

/* Kernel launches issued by the last hcran_solve (for accounting). */
int hcran_last_launch_count(hcran_t h, int32_t *launches);

/* Schedule chosen at hcran_create for every instance (no device access):
 * cluster_size[b] = number of CTAs (a thread-block cluster of 1 to 8) that
 * solve instance b with the dual-loop state resident in their shared memory,
 * or 0 when that state does not fit even 8 CTAs and the instance is solved by
 * one CTA streaming each subcarrier's state from global memory.  Among the
 * sizes whose state fits, the planner takes the one with the fewest SM
 * cycles per dual iteration under a cost model measured on GB300 (a CTA's
 * iteration costs about the same whether it holds a few or up to 512 (n, m)
 * groups, so fewer, fuller CTAs win).  Instances of one cluster size share one
 * persistent launch.  cluster_size:
 * caller-owned host array of n int32.  Returns HCRAN_EINVAL on a NULL
 * argument. */
int hcran_get_schedule(hcran_t h, int32_t *cluster_size);

/* Replace the schedule: cluster_size[b] in 1 .. 8 (a cluster of that
 * many CTAs with the dual-loop state resident in their shared memory; at
 * least one subcarrier per CTA, and the state must fit), 0 (one CTA
 * streaming each subcarrier's state from global memory, staged as the
 * planner sees fit) or -T, T in 1 .. 4 (the same, with the CTA's warps in T
 * teams that each stage one subcarrier at a time: the planner's choice when
 * the double buffers of every warp do not fit; every negative entry must
 * give the same T, and the teams' buffers must fit).  An instance whose
 * class would exceed shared memory moves on to a larger cluster
 * (hcran_get_schedule reports the result, 0 for every streamed instance).
 * The next solve uploads the new plan to its workspace.  Returns
 * HCRAN_EINVAL (schedule unchanged) on a NULL argument or an infeasible
 * size. */
int hcran_set_schedule(hcran_t h, const int32_t *cluster_size);

/* Autotuner of the schedule.  For each cluster size C < 8 in use it times
 * that class's launch against clusters of min(2 C, 8) CTAs on the class's first
 * S instances in launch order (S = the class size, at most eight waves of the
 * current schedule), with one Dinkelbach iteration, one SCALE pass and
 * exactly max(max_dual_probe / 4, 1) and that plus max_dual_probe dual
 * iterations, and keeps the schedule whose extra max_dual_probe dual
 * iterations take less time (the dual loop is almost all of a full solve);
 * every probe is timed twice and the shorter time kept.
 * When the streamed class runs team sweeps, it times the same probe on the
 * class's first wave (at most one instance per SM) for every team count from
 * 1 to the planner's (all of whose buffers fit) and keeps the fastest, as if
 * set by hcran_set_schedule's -T.
 * Probes overwrite the solution state in the workspace (a later solve starts
 * afresh).  Synchronises the stream.  gains_dev and workspace as for
 * hcran_solve; tol supplies tie_eps and q_init.  Returns HCRAN_EINVAL on bad
 * arguments, HCRAN_ECUDA on a CUDA error. */
int hcran_autotune(hcran_t h, const float *gains_dev, const hcran_tol *tol, void *workspace_dev, void *stream,
                   int32_t max_dual_probe);

/* Teams of warps the streamed class's sweeps run (0 when the class is empty
 * or its warps stage their own subcarriers); see hcran_set_schedule and
 * hcran_autotune.  Host only.  HCRAN_EINVAL on a NULL argument. */
int hcran_get_stream_teams(hcran_t h, int32_t *teams);

/* hcran_solve through a CUDA graph: the launch sequence (one persistent
 * launch per cluster size) is captured on the first call for a given
 * (gains_dev, workspace, tol) and replayed by later calls with the same
 * arguments; any change, or a new schedule, re-captures.  stream must be a
 * created stream (not the legacy default stream, which cannot be captured).
 * Same results as hcran_solve. */
int hcran_solve_graph(hcran_t h, const float *gains_dev, const hcran_tol *tol, void *workspace_dev, void *stream);

/* ---- learned warm start ----
 * The network (include/hcran_mlp.h) reads one row of features per slot of
 * the cold initial selection (A_k = argmax_m sum_n Gamma, the l strongest
 * users of A_k's RRH on every subcarrier) and returns one row of outputs per
 * slot; instance b owns rows [s_off_b, s_off_b + N_b * Up_b), slot (n, u) is
 * row s_off_b + n * Up_b + u, Up_b = M_b * l_b rounded up to a multiple of 4,
 * and the instances follow one another in creation order.
 *   features (BF16, 16 columns, the first four used): (log10 Gamma + 11) / 3,
 *     rank of Gamma among the K users on (m, n) / K, streaming (0 / 1),
 *     delay target / 0.1 s; empty slots are all zero;
 *   outputs (FP32, 16 columns, the first three used): y0 = log(p / mask_m),
 *     y1 with xi'_m = max(mean of e^y1 over RRH m's slots - 1e-3, 0) /
 *     (ln2 mask_m), y2 with zeta'_k = mean of e^y2 over user k's slots
 *     (clipped to [1e-6, 1e6]).
 * *rows = the number of rows (sum over instances of N * Up). */
int hcran_warm_rows(hcran_t h, int64_t *rows);

/* Writes the features of every row into features_dev ([rows][16] BF16,
 * device, 16-byte aligned).  Also leaves the initial selection (A, S) and
 * its powers in the workspace, where hcran_get reads them (its scalar
 * results are not updated).  Asynchronous on stream. */
int hcran_warm_features(hcran_t h, const float *gains_dev, void *workspace_dev, void *stream, void *features_dev);

/* hcran_solve started from the network's outputs (net_out_dev: [rows][16]
 * FP32, device) instead of the cold point: the same initial selection, p^0
 * = mask_m e^y0 clipped to [1e-9 mask_m, mask_m], xi' and zeta' as above,
 * then the C12 projection; E^1 = R(p^0) / P(p^0). */
int hcran_solve_warm(hcran_t h, const float *gains_dev, const hcran_tol *tol, void *workspace_dev, void *stream,
                     const float *net_out_dev);

void hcran_destroy(hcran_t h);

/* ---- global-optimum comparator -----------------------------------------
 * The paper compares its method with the optimum found by monotonic
 * optimisation (Sec. IV-B).  For small instances this computes that optimum's
 * stand-in by enumeration on the GPU: the best EE = R/P over every
 * assignment and over the powers.
 *  - Assignments: every RRH choice A_k in {-1 .. M-1} (A as a number in base
 *    M+1, user 0 the fastest digit, digit d meaning A_k = d - 1) and, on every
 *    (n, m) in (n, m) order with n slowest, every subset of the users of m of
 *    at most l members (listed by size, then lexicographically; the last
 *    (n, m) varies fastest), keeping those where every user with A_k >= 0 has
 *    at least one link.  best_index counts in that order.
 *  - Powers: coordinate golden-section search in [1e-6 mask, mask] from three
 *    starts p = f mask (f = 0.1, 0.4, 1), 8 sweeps over the links, 40 steps
 *    per link; a point breaking C12 or C14 (pairs of one (m, n) in SIC order)
 *    is infeasible.  FP64.
 *  - cfgs: n instances of one shape (M <= 8, K <= 6, l <= 3, N*M*l <= 16),
 *    elastic users only (Ks = 0); host memory read during the call.
 *  - gains_dev: float32 Gamma[n][m][k], instance b at element
 *    b * ((N*M*K + 3) / 4 * 4), device memory, 16-byte aligned.
 *  - workspace_dev: hcran_bf_workspace_size() bytes, 256-byte aligned,
 *    owned by the caller; the library allocates nothing.
 *  - Enqueues on `stream`, synchronises it, and writes best_ee[n] (0 when no
 *    assignment is feasible) and best_index[n] (-1 then; may be NULL) to host
 *    memory.  HCRAN_EINVAL for a bad or mixed shape, HCRAN_ECUDA on a CUDA
 *    error. */
int hcran_bf_workspace_size(const hcran_config *cfgs, int32_t n, uint64_t *bytes, int64_t *n_assign);
int hcran_bruteforce(const hcran_config *cfgs, int32_t n, const float *gains_dev, void *workspace_dev,
                     void *stream, double *best_ee, int64_t *best_index);

/* ---- penalty form of the selection constraints --------------------------
 * Sec. IV-A relaxes the binary RRH and subcarrier assignment into C10
 * (p_{m,k}^{(n)} p_{m',k}^{(n')} <= rho_1, m != m') and C11 (the product of the
 * powers of any l + 1 users on (m, n) <= rho_2), priced by the multipliers
 * theta, theta' in eq. (653).  hcran_solve takes the rho -> 0 limit as an
 * explicit selection; this call solves the penalty form itself, to compare
 * the two on small instances.  Every (m, k, n) link carries a power; the
 * iteration is hcran_solve's (Dinkelbach loop around Algorithm 1, same stop
 * rules) with theta, theta' stepped by
 *   theta  += delta_v clip((p p' - rho_1)/rho_1, -1, 1) / (ln2 mask_m mask_m'),
 *   theta' += delta_v clip((prod - rho_2)/rho_2, -1, 1) / (ln2 mask_m^(l+1)),
 * both projected on >= 0, rho_1 = rho_rel^2 mask_m mask_m',
 * rho_2 = (rho_rel mask_m)^(l+1); p starts at mask_m / K on every link.  C14
 * is not enforced.  FP64 arithmetic.
 *  - cfgs: n instances of one shape, M <= 4, N <= 4, K <= 8, l <= 3,
 *    N*M*K <= 128, elastic users only (Ks = 0), unit weights; host memory
 *    read during the call.
 *  - gains_dev: float32 Gamma[n][m][k], instance b at element
 *    b * ((N*M*K + 3) / 4 * 4), device memory, 16-byte aligned.
 *  - tol: tolerances and caps as for hcran_solve (tie_eps unused).
 *  - rho_rel in (0, 1).
 *  - workspace_dev: hcran_penalty_workspace_size() bytes, 256-byte aligned,
 *    owned by the caller; the library allocates no device memory.
 *  - Enqueues one kernel (one CTA per instance) on `stream`, synchronises it
 *    and writes to host memory ee[n], and when not NULL p[n*N*M*K] (W, the
 *    gain array's order), iters[3*n] (Dinkelbach, SCALE, dual), c10_max[n]
 *    and c11_max[n] (the largest C10 / C11 product over rho_1 / rho_2).
 *  - HCRAN_EINVAL for a bad or mixed shape or argument, HCRAN_ECUDA on a
 *    CUDA error. */
int hcran_penalty_workspace_size(const hcran_config *cfgs, int32_t n, uint64_t *bytes);
int hcran_penalty_solve(const hcran_config *cfgs, int32_t n, const float *gains_dev, const hcran_tol *tol,
                        double rho_rel, void *workspace_dev, void *stream, double *ee, double *p,
                        int32_t *iters, double *c10_max, double *c11_max);

/* ---- allocation-free single-instance solve ----------------------------
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory (a process whose device memory belongs to
 * another framework's pool or is locked after start-up, or a real-time loop
 * that must not call the allocator because an allocation can stall on a
 * device-wide synchronisation).  It solves one instance with the same solver
 * kernel, using as workspace a file-scope device array of
 * HCRAN_NOALLOC_SCRATCH_BYTES that every GPU loading this library holds
 * until the process exits.  It calls no cudaMalloc, cudaFree or other
 * allocating routine.
 *  - cfg: the instance (host memory, read during the call only).
 *  - gains_dev: float32 Gamma[n][m][k], device memory, 16-byte aligned.
 *  - out: caller-allocated host arrays as in hcran_result (NULL skips one).
 *  - Enqueues on `stream`, then synchronises it and copies the results; the
 *    call returns when they are in `out`.  Because it synchronises and
 *    copies synchronously, it cannot run inside a stream capture.
 *  - Every call looks up the array's address on the current device.
 *  - Every call on a device reuses the same array and leaves the previous
 *    call's contents behind; the call initialises everything it reads.  Two
 *    calls whose work overlaps on one GPU (different streams or threads)
 *    race on the array: serialise them.
 *  - Returns HCRAN_E2BIG, without touching the GPU, when the instance's
 *    workspace exceeds the array (about 4*N*M*M*l + 92*N*M*l + 20*N*K +
 *    12*N*M*l*(l-1) bytes must stay under 16 MiB); HCRAN_EINVAL for a bad
 *    config or tolerance. */
#define HCRAN_NOALLOC_SCRATCH_BYTES (16u << 20)
int hcran_solve_noalloc(const hcran_config *cfg, const float *gains_dev, const hcran_tol *tol, void *stream,
                        hcran_result *out);

#ifdef __cplusplus
}
#endif
#endif
