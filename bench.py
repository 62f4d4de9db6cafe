"""Benchmark: instances/s of the batched GPU solve (4096 uneven H-CRAN
realisations per step, the same seeds every step) on N GPUs of one node.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  A step is one hcran_solve of the whole batch (selection,
SCALE passes, dual loops and Dinkelbach updates of every instance, one
persistent kernel launch).  Under torchrun each rank solves its own batch
(seed offset by rank): weak scaling, no collective on the data path.
`--impl reference` times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "batch-4096-uneven"
METRIC = "instances/sec to EE within 1e-4 of FP64 oracle (plain cold-start batched GPU solve)"


def rank_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


# Under torchrun every rank solves its own batch (replicas, weak scaling): the
# instances of rank r are the seeds [r * count, (r + 1) * count) of the
# workload, the step time is the maximum over ranks, and the job value counts
# every rank's instances.
def rank_seed_start(rank: int, count: int) -> int:
    return rank * count


def max_over_ranks(x: float, device, world: int) -> float:
    """Maximum of x over the ranks of the default process group (x itself
    when there is one rank)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world: int, count: int, per_step_s: float) -> float:
    """Instances per second of the whole job."""
    return world * count / per_step_s


# ---------------------------------------------------------------- CPU oracle leg

def _oracle_one(args):
    idx, start = args
    sys.path.insert(0, ROOT)
    import oracle
    from hcran_inputs import WORKLOADS, make_workload
    inst = make_workload(WORKLOAD, count=1, start=start + idx)[0]
    t = time.perf_counter()
    oracle.solve(inst, WORKLOADS[WORKLOAD]["tol"])
    return time.perf_counter() - t


def oracle_sample_ids(count: int, seed: int = 12345):
    """A seeded random subset (without replacement) of the workload's 4096
    instances, drawn uniformly: the whole size range, not only small ones."""
    rng = np.random.default_rng(seed)
    return sorted(rng.choice(4096, size=min(count, 4096), replace=False).tolist())


def time_oracle(ids, procs: int):
    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        pool.map(_oracle_one, [(0, ids[0])])           # warm the workers' imports
        t0 = time.perf_counter()
        pool.map(_oracle_one, [(0, i) for i in ids])
        wall = time.perf_counter() - t0
    return wall


def cpu_baseline(cores: int):
    ids = oracle_sample_ids(cores)
    wall = time_oracle(ids, cores)
    return {"value": len(ids) / wall, "unit": "instances/s", "cores": cores, "kind": "oracle",
            "sample": "%d instances of the %s workload drawn uniformly at random (seeded) from its "
                      "4096, one per process, FP64 C oracle" % (len(ids), WORKLOAD)}


def run_reference(args):
    rank, world, _ = rank_env()
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    ids_all = oracle_sample_ids(cores * args.steps)
    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    times = []
    with ctx.Pool(cores) as pool:
        # warm-up steps: the workers import and load the oracle (it keeps no
        # other state between solves), on the workload's first instance
        for s in range(args.warmup):
            pool.map(_oracle_one, [(0, 0)] * cores)
        for s in range(args.steps):
            ids = ids_all[s * cores:(s + 1) * cores] or ids_all[:cores]
            t0 = time.perf_counter()
            pool.map(_oracle_one, [(0, i) for i in ids], chunksize=1)
            times.append((len(ids), time.perf_counter() - t0))
    n = sum(c for c, _ in times)
    wall = sum(t for _, t in times)
    v = n / wall
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "instances/s",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * wall / max(len(times), 1), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "instances_per_step": cores,
                      "sample": "instances drawn uniformly at random (seeded) from the 4096"},
           "cpu_baseline": {"value": v, "unit": "instances/s", "cores": cores, "kind": "oracle",
                            "sample": "%d instances per step, one per process" % cores},
           "e2e": {"value": v, "unit": "instances/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------- clocks

class Clocks:
    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except Exception:
            self.p.kill()
            return None
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 6:
                continue
            try:
                sm.append(float(f[0]))
                mx = max(mx, float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[2:6]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- GPU leg

def algorithmic_bytes(insts, iters, links):
    """Bytes the method must move per solve (per instance, summed):
    one read of Gamma (4 M N K) per selection (one per Dinkelbach iteration),
    and per dual iteration one read of the compact slab, the gains from all
    M RRHs to the selected links (4 M sum_n |S_n|, links[b] = sum_n |S_n| of
    the final selection), plus four words per slot (power, alpha, price, user
    id: 16 N M l)."""
    tot = 0
    for inst, it, nl in zip(insts, iters, links):
        M, N, K, l = inst.M, inst.N, inst.K, inst.l
        tot += 4 * M * N * K * int(it[0]) + int(it[2]) * (4 * M * int(nl) + 16 * N * M * l)
    return tot


def selected_links(solver, n):
    """sum_n |S_n| (selected links) of every instance's final selection."""
    return np.array([int(np.sum(solver.get(i)["S"] >= 0)) for i in range(n)], dtype=np.int64)


def run_gpu(args):
    import torch
    import torch.distributed as dist
    from hcran_inputs import WORKLOADS, make_workload, pack_batch
    from paper_1803_07772_gb300 import Solver, make_tol

    rank, world, local = rank_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cpu_line = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # before any CUDA work in this process; the pool uses spawn anyway
        cpu_line = cpu_baseline(os.cpu_count() or 1)

    count = args.instances
    insts = make_workload(WORKLOAD, count=count, start=rank_seed_start(rank, count))
    gains, offs = pack_batch(insts)
    tol = make_tol(WORKLOADS[WORKLOAD]["tol"])
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        solver = Solver(insts, gain_offsets=offs, device=str(dev), stream=stream)
        g = torch.from_numpy(gains).to(dev)
    torch.cuda.synchronize(dev)

    # schedule: the planner's cost-model choice, then the autotuner
    # (untimed); the timed steps replay one CUDA graph of the class launches
    # (--no-graph: direct launches, the form a profiler can replay one by one)
    planned = solver.schedule()
    if not args.no_autotune:
        solver.autotune(g, tol, max_dual_probe=60)
    sched = solver.schedule()
    step = solver.solve if args.no_graph else solver.solve_graph
    for _ in range(args.warmup):
        step(g, tol)
    stream.synchronize()

    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clocks = Clocks(local)
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    launches = 0
    for _ in range(args.steps):
        step(g, tol)
        launches += solver.launches()
    ev1.record(stream)
    stream.synchronize()
    torch.cuda.synchronize(dev)
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    ms_max = max_over_ranks(ms, dev, world)
    if world > 1:
        dist.barrier()
    summ = solver.summary()

    # end to end through the C ABI from pinned host memory (copies inside the timed region)
    host = torch.from_numpy(gains).pin_memory()
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ee_h, st_h = solver.solve_host(host, tol)
    e2e_s = max_over_ranks((time.perf_counter() - t0) / args.steps, dev, world)

    warm = None
    if not args.no_warm and world == 1:
        warm = warm_leg(args, solver, g, insts, tol, summ, ms_max / args.steps, stream, dev)
    scen = None
    if not args.no_scenarios and world == 1:
        try:
            scen = scenario_leg(dev)
        except Exception as e:  # the main bench line stands on its own
            scen = {"error": "%s: %s" % (type(e).__name__, e)}

    large = None
    if args.large and world == 1:
        large = large_leg(dev)
    optimum = None
    if not args.no_scenarios and world == 1:
        try:
            optimum = optimum_leg(dev)
        except Exception as e:  # the main bench line stands on its own
            optimum = {"error": "%s: %s" % (type(e).__name__, e)}

    if rank == 0:
        per_step_ms = ms_max / args.steps
        value = job_value(world, count, per_step_ms / 1e3)
        links = selected_links(solver, count)
        abytes = algorithmic_bytes(insts, summ["iters"], links)
        peaks = {}
        try:
            peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        except Exception:
            pass
        peak = float(peaks.get("hbm_gbs", 6800.0))
        achieved = abytes / (per_step_ms / 1e3) / 1e9
        traffic = None
        try:
            prof = json.load(open(os.path.join(ROOT, "profiles", "solve_kernel_traffic.json")))
            if prof.get("kernel_hash") == kernel_hash():
                # DRAM bytes per algorithmic byte from the launch list of a smaller
                # case of the same workload, scaled to this launch's algorithmic bytes
                traffic = float(prof["traffic_per_algorithmic_byte"]) * abytes
        except Exception:
            pass
        dram_gbs = traffic / (per_step_ms / 1e3) / 1e9 if traffic is not None else None
        out = {
            "metric": METRIC, "value": value, "unit": "instances/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step_ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "instances_per_gpu": count,
                       "sizes": "M~U{3..16}, N~U{16..256}, K~U{10..120}, 30% streaming, l=3",
                       "precision": "FP32 SINR/power/prices, FP64 Dinkelbach q, F(q), multipliers",
                       "l2": "inputs larger than L2 (%.2f GB of gains per step)" % (gains.nbytes / 1e9),
                       "parallelism": "replicas" if world == 1 else "dp%d" % world,
                       "schedule": {("streamed" if k == 0 else "cluster%d" % k): int(v)
                                    for k, v in zip(*np.unique(sched, return_counts=True))},
                       "schedule_changed_by_autotuner": int(np.sum(sched != planned)),
                       "launch": ("direct launches" if args.no_graph else "CUDA graph") +
                                 ", one persistent launch per cluster size"},
            "gpu_launches": launches,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks else "fallback 6.8 TB/s",
                         "achieved_is": "algorithmic bytes (Gamma per selection, compact slab of the selected "
                                        "links and slot state per dual iteration) / step time",
                         "algorithmic_bytes_per_launch": abytes,
                         "selected_links_mean": float(links.mean()),
                         "dram_gbs": dram_gbs,
                         "dram_frac": dram_gbs / peak if dram_gbs is not None else None},
            "e2e": {"value": job_value(world, count, e2e_s), "unit": "instances/s",
                    "h2d_bytes_per_step": int(gains.nbytes),
                    "d2h_bytes_per_step": int(count * 8 + count * 4)},
            "solve_stats": {"mean_iters": np.mean(summ["iters"], axis=0).tolist(),
                            "status_counts": {str(k): int(v) for k, v in
                                              zip(*np.unique(summ["status"], return_counts=True))},
                            "ee_mean": float(np.mean(summ["ee"]))},
        }
        if clk:
            out["clocks"] = clk
        if cpu_line:
            out["cpu_baseline"] = cpu_line
        if warm:
            out["warm_start"] = warm
        if scen:
            out["scenarios"] = scen
        if large:
            out["large"] = large
        if optimum:
            out["optimum_gap"] = optimum
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def _hbm_peak() -> float:
    """Measured copy bandwidth of the GB300s (GB/s), else the fallback."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except Exception:
        return 6800.0


def large_leg(dev, count=256):
    """The large workload (1 HPN + 32 LPNs, 1024 subcarriers, 512 users, l = 4;
    about 69 MB of FP32 gains per instance, 17.7 GB for 256): every instance
    solved to the workload's own stop rules in one solve (one CTA per
    instance on the streamed schedule, its dual-loop state exceeding any
    cluster's shared memory), timed with CUDA events after one untimed
    solve.  Returns instances/s, algorithmic GB/s and the solve statistics."""
    import torch
    from hcran_inputs import WORKLOADS, make_workload, pack_batch
    from paper_1803_07772_gb300 import Solver, make_tol
    name = "large-33x1024x512"
    insts = make_workload(name, count=count)
    gains, offs = pack_batch(insts)
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        s = Solver(insts, gain_offsets=offs, device=str(dev), stream=stream)
        g = torch.from_numpy(gains).to(dev)
    del gains
    tol = make_tol(WORKLOADS[name]["tol"])
    teams_planned = s.stream_teams()
    s.autotune(g, tol)  # the team count of the streamed sweeps
    s.solve(g, tol)
    stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.solve(g, tol)
    e1.record(stream)
    stream.synchronize()
    sec = e0.elapsed_time(e1) / 1e3
    summ = s.summary()
    links = selected_links(s, count)
    ab = algorithmic_bytes(insts, summ["iters"], links)
    out = {"workload": name, "instances": count, "instances_per_s": count / sec, "seconds": sec,
           "algorithmic_gbs": ab / sec / 1e9, "schedule": "one CTA per instance, streamed",
           "algorithmic_frac_of_measured_hbm": ab / sec / 1e9 / _hbm_peak(),
           "teams": {"planned": int(teams_planned), "autotuned": int(s.stream_teams())},
           "gain_bytes": int(4 * sum(i.cost for i in insts)),
           "mean_iters": np.mean(summ["iters"], axis=0).tolist(),
           "status_counts": {str(k): int(v) for k, v in zip(*np.unique(summ["status"], return_counts=True))},
           "ee_mean": float(np.mean(summ["ee"]))}
    s.close()
    del g
    torch.cuda.empty_cache()
    return out


def optimum_leg(dev):
    """The gap of the method to the optimum (Sec. IV-B's role): the 256
    instances of the optimum workload (1 HPN + 2 LPNs, 2 subcarriers, 3
    elastic users, l = 2; 954 assignments each) through the GPU brute-force
    comparator and through the method's GPU solve.  Reports the comparator's
    time and the distribution of EE(method) / EE(optimum)."""
    import torch
    from hcran_inputs import WORKLOADS, make_workload, pack_batch
    from paper_1803_07772_gb300 import Solver, make_tol
    from paper_1803_07772_gb300.hcran import bruteforce
    name = "optimum-3x2x3"
    insts = make_workload(name)
    gains, offs = pack_batch(insts)
    g = torch.from_numpy(gains).to(dev)
    bruteforce(insts, g)  # warm-up
    t0 = time.perf_counter()
    ee_opt, _, na = bruteforce(insts, g)
    bf_s = time.perf_counter() - t0
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        s = Solver(insts, gain_offsets=offs, device=str(dev), stream=stream)
    s.solve(g, make_tol(WORKLOADS[name]["tol"]))
    ee = s.summary()["ee"]
    s.close()
    r = ee / ee_opt
    # the paper's own relaxation of the selection (C10 / C11 with theta, theta')
    # on the same instances: a cross-check of the explicit selection
    from paper_1803_07772_gb300.hcran import penalty_solve
    tol = make_tol(WORKLOADS[name]["tol"])
    penalty_solve(insts, g, tol)  # warm-up
    t0 = time.perf_counter()
    pen = penalty_solve(insts, g, tol)
    pen_s = time.perf_counter() - t0
    rp = pen["ee"] / ee_opt
    leak = (pen["c10_max"] > 1.0 + 1e-9) | (pen["c11_max"] > 1.0 + 1e-9)

    def dist(x):
        return {"min": float(x.min()), "median": float(np.median(x)), "mean": float(x.mean()),
                "max": float(x.max()), "within_1pct": float(np.mean(x >= 0.99))}
    return {"workload": name, "instances": len(insts), "assignments_per_instance": int(na),
            "comparator_seconds": bf_s, "comparator_assignments_per_s": len(insts) * na / bf_s,
            "method_over_optimum": dist(r),
            "penalty_form": {"seconds": pen_s, "instances_per_s": len(insts) / pen_s,
                             "rho_rel": 1e-3, "over_optimum": dist(rp),
                             "above_selection_form": float(np.mean(pen["ee"] > ee * (1 + 1e-4))),
                             "below_selection_form": float(np.mean(pen["ee"] < ee * (1 - 1e-4))),
                             "c10_or_c11_above_rho": float(np.mean(leak)),
                             "mean_iters": pen["iters"].mean(axis=0).tolist()}}


def scenario_leg(dev):
    """The architectures of Sec. VI (H-CRAN with NOMA and OMA, 1-tier C-RAN,
    2-tier HCN, 1-tier HPN; 256 instances each, same seeds and users): solve
    throughput and the mean elastic-user EE of each, timed with CUDA events
    after 3 warm-up solves."""
    import torch
    from hcran_inputs import SCENARIOS, WORKLOADS, make_workload, pack_batch
    from paper_1803_07772_gb300 import Solver, make_tol
    out = {}
    stream = torch.cuda.Stream(dev)
    for name in SCENARIOS:
        insts = make_workload(name)
        gains, offs = pack_batch(insts)
        with torch.cuda.stream(stream):
            s = Solver(insts, gain_offsets=offs, device=str(dev), stream=stream)
            g = torch.from_numpy(gains).to(dev)
        tol = make_tol(WORKLOADS[name]["tol"])
        for _ in range(3):
            s.solve_graph(g, tol)
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.solve_graph(g, tol)
        e1.record(stream)
        stream.synchronize()
        summ = s.summary()
        out[name] = {"instances_per_s": len(insts) / (e0.elapsed_time(e1) / 1e3),
                     "mean_ee": float(np.mean(summ["ee"])),
                     "streaming_unmet": int(np.sum((np.asarray(summ["status"]) & 2) != 0)),
                     "mean_iters": np.mean(summ["iters"], axis=0).tolist()}
        s.close()
    return out


MLP_FLOPS_PER_ROW = 2 * (16 * 256 + 256 * 256 + 256 * 256 + 256 * 16)  # forward, padded widths


def warm_leg(args, solver, g, insts, tol, cold_summ, cold_ms, stream, dev):
    """Learned warm start on the same batch: train the network on instances
    from a disjoint seed range (untimed), then time features + network +
    warm solve with CUDA events and hold every warm EE to the cold solve's."""
    import torch
    from hcran_inputs import make_workload, pack_batch
    from paper_1803_07772_gb300 import Solver
    from paper_1803_07772_gb300.mlp import MLP
    from paper_1803_07772_gb300.warmstart import TRAIN_SEED_BASE, build_dataset, train, warm_solve
    t0 = time.time()
    tr = make_workload(WORKLOAD, count=args.warm_train, start=TRAIN_SEED_BASE - 300000)
    tg, toffs = pack_batch(tr)
    with torch.cuda.stream(stream):
        ts = Solver(tr, gain_offsets=toffs, device=str(dev), stream=stream)
        tgd = torch.from_numpy(tg).to(dev)
    X, Y, Mk = build_dataset(ts, tgd, tr, tol)
    del ts, tgd
    net = MLP(seed=7, max_rows=1 << 22)  # inference in chunks of 4M rows; training batches of 2^15
    hist = train(net, X, Y, Mk, epochs=args.warm_epochs, batch=1 << 15, lr=2e-3)
    train_s = time.time() - t0
    rows = solver.warm_rows()
    feats = torch.zeros((rows, 16), dtype=torch.bfloat16, device=dev)
    out = torch.empty((rows, 16), dtype=torch.float32, device=dev)
    warm_solve(solver, net, g, tol, feats, out)  # warm-up
    stream.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    e[0].record(stream)
    solver.warm_features(g, feats)
    e[1].record(stream)
    net.forward(feats, out, stream)
    e[2].record(stream)
    solver.solve_warm(g, tol, out)
    e[3].record(stream)
    stream.synchronize()
    ms = [e[i].elapsed_time(e[i + 1]) for i in range(3)]
    tot_ms = sum(ms)
    ws = solver.summary()
    rel = np.abs(ws["ee"] - cold_summ["ee"]) / np.maximum(np.abs(cold_summ["ee"]), 1e-300)
    acc = rel <= 1e-4
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    tflops = rows * MLP_FLOPS_PER_ROW / (ms[1] / 1e3) / 1e12
    n = len(insts)
    # ceiling of any warm start: every instance started from the cold solve's
    # own converged state (a perfect predictor of powers, selection and
    # multipliers, through hcran_set_state), timed the same way
    solver.solve(g, tol)
    states = [solver.get(i) for i in range(n)]
    for i, st_ in enumerate(states):
        solver.set_state(i, st_)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    solver.solve(g, tol)
    e1.record(stream)
    stream.synchronize()
    ex_ms = e0.elapsed_time(e1)
    xs = solver.summary()
    ex_rel = np.abs(xs["ee"] - cold_summ["ee"]) / np.maximum(np.abs(cold_summ["ee"]), 1e-300)
    ex_acc = ex_rel <= 1e-4
    ceiling = {"instances_per_s_with_cold_fallback": n / ((ex_ms + (1.0 - ex_acc.mean()) * cold_ms) / 1e3),
               "speedup_vs_cold": (n / ((ex_ms + (1.0 - ex_acc.mean()) * cold_ms) / 1e3)) / (n / (cold_ms / 1e3)),
               "accepted_within_1e-4_of_cold": float(ex_acc.mean()),
               "mean_iters": np.mean(xs["iters"], axis=0).tolist(),
               "is": "every instance resumed from the cold solve's own converged state (hcran_set_state): the "
                     "best any predicted start point can do under the method's stop rules"}
    # instances whose warm EE misses the cold one by more than 1e-4 are solved cold again
    eff = n / ((tot_ms + (1.0 - acc.mean()) * cold_ms) / 1e3)
    return {"value": eff, "unit": "instances/s",
            "value_is": "instances/s of features + network + warm solve, with every instance whose warm EE "
                        "misses the cold solve's by more than 1e-4 solved cold again",
            "speedup_vs_cold": eff / (n / (cold_ms / 1e3)),
            "ms_per_step": tot_ms, "ms_features_network_solve": ms,
            "accepted_within_1e-4_of_cold": float(acc.mean()),
            "warm_ee_not_below_cold": float(np.mean(ws["ee"] >= cold_summ["ee"] * (1 - 1e-4))),
            "median_ee_ratio_warm_to_cold": float(np.median(ws["ee"] / np.maximum(cold_summ["ee"], 1e-300))),
            "warm_only_instances_per_s": n / (tot_ms / 1e3),
            "mean_iters_warm": np.mean(ws["iters"], axis=0).tolist(),
            "ceiling_exact_state": ceiling,
            "network": {"rows": int(rows), "tflops": tflops,
                        "peak_tflops": float(peaks.get("bf16_tflops", 1900.0)),
                        "frac": tflops / float(peaks.get("bf16_tflops", 1900.0)),
                        "kernel": "tcgen05 BF16 x BF16 -> FP32 (TMEM)"},
            "training": {"instances": len(tr), "rows": int(X.shape[0]), "epochs": args.warm_epochs,
                         "loss_per_epoch": hist, "seconds": train_s,
                         "seeds": "%d.." % (TRAIN_SEED_BASE,)}}


def run_profile_case():
    import torch
    from hcran_inputs import Tolerances, make_workload, pack_batch
    from paper_1803_07772_gb300 import Solver, make_tol
    insts = make_workload(WORKLOAD, count=152)
    gains, offs = pack_batch(insts)
    s = Solver(insts, gain_offsets=offs)
    g = torch.from_numpy(gains).cuda()
    s.solve(g, make_tol(Tolerances(max_dinkelbach=1, max_scale=2, max_dual=100)))
    torch.cuda.synchronize()
    sched = s.schedule()
    print(json.dumps({"profile_case": WORKLOAD, "instances": 152,
                      "iters_total": s.summary()["iters"].sum(0).tolist(),
                      "schedule": {int(k): int(v) for k, v in zip(*np.unique(sched, return_counts=True))}}))


# device code of the solve kernel (the host planner and ABI files are left out:
# they do not change what one launch reads and writes)
KERNEL_FILES = ("hcran_kernel.cu", "hcran_layout.h", "hcran_dev_common.cuh", "hcran_dev_link.cuh",
                "hcran_dev_dual.cuh", "hcran_dev_team.cuh", "hcran_dev_resident.cuh", "hcran_dev_select.cuh",
                "hcran_dev_warm.cuh")


def run_profile_large():
    """The first 16 instances of the 33 x 1024 x 512 workload with short caps
    (1 Dinkelbach iteration, 1 SCALE pass, 8 dual iterations): the small
    case of the streamed team sweeps for ncu (about 1.6 GB on the device)."""
    import torch
    from hcran_inputs import Tolerances, make_workload, pack_batch
    from paper_1803_07772_gb300 import Solver, make_tol
    insts = make_workload("large-33x1024x512", count=16)
    gains, offs = pack_batch(insts)
    s = Solver(insts, gain_offsets=offs)
    g = torch.from_numpy(gains).cuda()
    s.solve(g, make_tol(Tolerances(max_dinkelbach=1, max_scale=1, max_dual=8)))
    torch.cuda.synchronize()
    cyc = s.phase_cycles()
    print(json.dumps({"profile_large": "large-33x1024x512", "instances": 16,
                      "iters_total": s.summary()["iters"].sum(0).tolist(),
                      "fused_sweep_cycles_per_dual_iteration": float(cyc[:, 3].sum() / max(1, s.summary()["iters"][:, 2].sum()))}))


def run_profile_penalty():
    """The penalty form of C10 / C11 on the 256 instances of the optimum
    workload (one launch, one CTA per instance): the case for ncu."""
    import torch
    from hcran_inputs import WORKLOADS, make_workload, pack_batch
    from paper_1803_07772_gb300 import make_tol
    from paper_1803_07772_gb300.hcran import penalty_solve
    name = "optimum-3x2x3"
    insts = make_workload(name)
    gains, _ = pack_batch(insts)
    g = torch.from_numpy(gains).cuda()
    t0 = time.perf_counter()
    out = penalty_solve(insts, g, make_tol(WORKLOADS[name]["tol"]))
    sec = time.perf_counter() - t0
    print(json.dumps({"profile_penalty": name, "instances": len(insts), "seconds": sec,
                      "mean_iters": out["iters"].mean(axis=0).tolist(), "mean_ee": float(out["ee"].mean())}))


def run_profile_mlp():
    """One forward, loss gradient, backward and Adam step of the warm-start
    network on 2^20 synthetic rows (the profiling case of its kernels)."""
    import torch
    from paper_1803_07772_gb300.mlp import MLP
    T = 1 << 20
    g = torch.Generator().manual_seed(0)
    x = torch.zeros((T, 16))
    x[:, :4] = torch.randn((T, 4), generator=g)
    x = x.to(torch.bfloat16).cuda()
    tgt = torch.randn((T, 16), generator=g).cuda()
    mask = torch.ones((T, 16)).cuda()
    net = MLP(seed=1, max_rows=T)
    out = torch.empty((T, 16), dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, device="cuda")
    net.forward(x, out)
    net.loss_grad(out, tgt, mask, loss)
    net.backward(x)
    net.adam(1e-3)
    torch.cuda.synchronize()
    print(json.dumps({"profile_mlp_rows": T, "loss": float(loss.item()), "tc_failed": net.tc_failed()}))


def _code_only(src: bytes) -> bytes:
    """C/C++ source with comments removed and whitespace runs collapsed, so
    that a comment edit does not count as a change of the device code."""
    out, i, n, quote = [], 0, len(src), None
    while i < n:
        c = src[i:i + 1]
        if quote:
            out.append(c)
            if c == b"\\":
                out.append(src[i + 1:i + 2])
                i += 2
                continue
            if c == quote:
                quote = None
        elif c in (b'"', b"'"):
            quote = c
            out.append(c)
        elif src[i:i + 2] == b"//":
            j = src.find(b"\n", i)
            i = n if j < 0 else j
            continue
        elif src[i:i + 2] == b"/*":
            j = src.find(b"*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(b" ")
            continue
        else:
            out.append(c)
        i += 1
    return b" ".join(b"".join(out).split())


def kernel_hash(read=None) -> str:
    """sha256 (first 16 hex digits) of the solve kernel's device source, comments
    and whitespace removed."""
    import hashlib
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1803_07772_gb300", "csrc")
    for f in KERNEL_FILES:
        h.update(_code_only(read(f) if read else open(os.path.join(d, f), "rb").read()))
    return h.hexdigest()[:16]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--instances", type=int, default=4096)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the planner's schedule")
    ap.add_argument("--no-warm", action="store_true", help="skip the learned warm-start leg")
    ap.add_argument("--no-scenarios", action="store_true", help="skip the Sec. VI architecture scenarios")
    ap.add_argument("--no-graph", action="store_true",
                    help="launch the classes directly instead of replaying a CUDA graph (for profiler launch lists)")
    ap.add_argument("--profile-mlp", action="store_true",
                    help="one training step of the warm-start network on 2^20 rows (the case for ncu)")
    ap.add_argument("--large", action="store_true",
                    help="also solve the 256 instances of the 33 x 1024 x 512 workload (about 17.7 GB of gains)")
    ap.add_argument("--warm-train", type=int, default=512, help="training instances of the warm start")
    ap.add_argument("--warm-epochs", type=int, default=8)
    ap.add_argument("--profile-penalty", action="store_true",
                    help="the penalty form of C10/C11 on the 256 optimum-workload instances (the case for ncu)")
    ap.add_argument("--profile-large", action="store_true",
                    help="16 instances of the 33 x 1024 x 512 workload with short caps (the small case for ncu)")
    ap.add_argument("--profile-case", action="store_true",
                    help="one solve of the first 152 instances with short caps (1 Dinkelbach "
                         "iteration, 2 SCALE passes, 100 dual iterations): the small case for ncu")
    args = ap.parse_args()
    if args.profile_case:
        run_profile_case()
        return
    if args.profile_large:
        run_profile_large()
        return
    if args.profile_penalty:
        run_profile_penalty()
        return
    if args.profile_mlp:
        run_profile_mlp()
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
