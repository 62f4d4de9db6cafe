"""The 4096-instance batch at full size, in the benchmark's launch
configuration (the planner's schedule, one CUDA graph of the class launches),
held to the oracle on a sample spread over every cluster size and over the
size range within it.  Named to run last: it is the slowest GPU test (the
whole batch plus 64 oracle solves)."""
import multiprocessing as mp
import os

import numpy as np
import pytest

from hcran_inputs import WORKLOADS, make_workload, pack_batch
from tests.parity import TIE_BAND

pytestmark = pytest.mark.gpu

PER_CLASS = 8


def _orc(args):
    import oracle
    inst, tol = args
    return oracle.solve(inst, tol, tie_eps=TIE_BAND)


def _sample(insts, sched):
    """Up to PER_CLASS instances of every cluster size (0 = streamed), evenly
    spaced over the class's cost order: its cheapest, its most expensive and
    the sizes between."""
    out = []
    for c in range(0, 9):
        idx = sorted((i for i in range(len(insts)) if sched[i] == c), key=lambda i: insts[i].cost)
        if not idx:
            continue
        k = min(PER_CLASS, len(idx))
        out += [idx[int(round(j * (len(idx) - 1) / max(k - 1, 1)))] for j in range(k)]
    return sorted(set(out))


def test_full_batch_in_bench_configuration_matches_oracle_on_a_sample():
    import oracle
    oracle.build()
    name = "batch-4096-uneven"
    insts = make_workload(name)
    tol = WORKLOADS[name]["tol"]
    # the oracle pool starts before the first CUDA call (spawn, as required
    # once a CUDA context exists)
    pool = mp.get_context("spawn").Pool(max(1, min(16, os.cpu_count() or 1)))
    try:
        import torch
        from paper_1803_07772_gb300 import Solver, make_tol
        from tests.oracle_ensemble import ensemble
        from tests.parity import classify
        gains, offs = pack_batch(insts)
        st = torch.cuda.Stream(device="cuda:0")
        s = Solver(insts, gain_offsets=offs, device="cuda:0", stream=st)
        g = torch.from_numpy(gains).to("cuda:0")
        sched = s.schedule()
        sample = _sample(insts, sched)
        assert len(sample) >= 64, len(sample)
        pending = pool.map_async(_orc, [(insts[b], tol) for b in sample], chunksize=1)
        s.solve_graph(g, make_tol(tol, tie_eps=TIE_BAND))
        summ = s.summary()
        u, cnt = np.unique(summ["status"], return_counts=True)
        print("status counts over the batch", dict(zip(u.tolist(), cnt.tolist())))
        assert np.all(np.isfinite(summ["ee"]))
        assert (summ["status"] == 0).mean() >= 0.95
        orcs = pending.get()
    finally:
        pool.close()
    tiers = {}
    errs = []
    for b, o in zip(sample, orcs):
        inst = insts[b]
        label = "batch instance %d (cluster of %d, M%d N%d K%d)" % (b, sched[b], inst.M, inst.N, inst.K)
        tier, rep = classify(inst, s.get(b), o, tol, label, ensemble_fn=ensemble)
        print("parity", tier, rep)
        tiers[tier] = tiers.get(tier, 0) + 1
        errs.append(rep["ee_rel"])
    print("tiers", tiers, "EE error vs plain oracle: median %.2e max %.2e" % (np.median(errs), max(errs)))
    assert tiers.get("fail", 0) == 0, tiers
    assert tiers.get("plain", 0) >= 0.9 * len(sample), tiers
