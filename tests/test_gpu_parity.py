"""CUDA solver vs FP64 oracle on the same seeded inputs, through the C ABI.

The bar is tests.parity's: the plain oracle, element by element (selection
up to vanishing links, EE within 1e-4, powers within 1e-3), else a tie
flagged below 1e-9 on either side or an instance whose oracle end point is
itself rounding-sensitive, each held to the validity checks.  Every report
prints the error against the plain oracle.  With the stop tests switched off
(fixed iteration counts on both sides) the bar is the plain one and the
iteration counts must agree.
"""
import copy

import numpy as np
import pytest

import oracle
from tests.oracle_ensemble import ensemble
from tests.parity import EE_RTOL, TIE_BAND, check, classify, validity
from hcran_inputs import Instance, Tolerances, WORKLOADS, make_instance, make_workload, pack_batch

pytestmark = pytest.mark.gpu


def gpu_solve(insts, tol, **tolkw):
    import torch
    from paper_1803_07772_gb300 import Solver, make_tol
    gains, offs = pack_batch(insts)
    s = Solver(insts, gain_offsets=offs, device="cuda:0")
    g = torch.from_numpy(gains).to("cuda:0")
    s.solve(g, make_tol(tol, tie_eps=TIE_BAND, **tolkw))
    out = [s.get(i) for i in range(len(insts))]
    assert s.launches() >= 1
    return out


def compare(inst, g, o, label="", p_abs=1e-6):
    """Assert the plain bar against one oracle result; return the report.
    p_abs: the absolute power allowance in mask units (1e-6 at fixed
    iteration counts; the dual loop's tolerance under the stop rules)."""
    rep = check(inst, g, o, label, p_abs=p_abs)
    print("parity", rep)
    assert rep["ok"], rep
    validity(inst, g, label, ref=o)
    return rep


def hold(inst, g, tol, label="", **kw):
    """Tier of one result under the workload's own stop rules (tests.parity)."""
    o = oracle.solve(inst, tol, tie_eps=TIE_BAND, **kw)
    tier, rep = classify(inst, g, o, tol, label, ensemble_fn=ensemble, **kw)
    print("parity", tier, rep)
    assert tier != "fail", rep
    return tier, rep


@pytest.mark.parametrize("name", ["small-3x8x6", "medium-9x64x48"])
def test_config_matches_plain_oracle(name):
    """The small and medium configurations under their own stop rules, held to
    the plain oracle."""
    inst = make_workload(name)[0]
    tol = WORKLOADS[name]["tol"]
    g = gpu_solve([inst], tol)[0]
    o = oracle.solve(inst, tol, tie_eps=TIE_BAND)
    compare(inst, g, o, name, p_abs=tol.tol_dual)
    assert g["status"] == o.status == 0


@pytest.mark.parametrize("v", [1, 5, 60, 200])
def test_dual_steps_match_at_fixed_E(v):
    """One selection then exactly v dual iterations of one SCALE pass at a
    fixed E: isolates the KKT power and subgradient arithmetic."""
    name = "medium-9x64x48"
    inst = make_workload(name)[0]
    tol = Tolerances(tol_dinkelbach=0.0, tol_scale=0.0, tol_dual=0.0,
                     max_dinkelbach=1, max_scale=1, max_dual=v)
    g = gpu_solve([inst], tol, q_init=40.0)[0]
    o = oracle.solve(inst, tol, q_init=40.0)
    assert np.array_equal(g["S"], o.S) and np.array_equal(g["A"], o.A)
    sel = o.S >= 0
    rel = np.abs(g["p"][sel] - o.p[sel]) / o.p[sel]
    print("dual steps", v, "max p rel", rel.max(), "xi", np.abs(g["xi"] - o.xi).max(),
          "zeta rel", np.max(np.abs(g["zeta"] - o.zeta) / o.zeta))
    assert rel.max() < 1e-4
    assert np.allclose(g["zeta"], o.zeta, rtol=1e-4)
    assert np.allclose(g["xi"], o.xi, rtol=1e-4, atol=1e-6 * max(1.0, float(np.max(np.abs(o.xi)))))


def test_algorithm1_matches_at_fixed_E():
    name = "medium-9x64x48"
    inst = make_workload(name)[0]
    tol = copy.copy(WORKLOADS[name]["tol"])
    tol.max_dinkelbach = 1
    g = gpu_solve([inst], tol, q_init=60.0)[0]
    compare(inst, g, oracle.solve(inst, tol, q_init=60.0, tie_eps=TIE_BAND), "alg1@E=60", p_abs=tol.tol_dual)


@pytest.mark.parametrize("name", ["medium-9x64x48", "batch"])
def test_fixed_iteration_counts_match_everywhere(name):
    """Stop tests off (every loop runs to its cap): both sides take the same
    steps, so every selected power must agree to 1e-3 relative."""
    tol = Tolerances(tol_dinkelbach=0.0, tol_scale=0.0, tol_dual=0.0,
                     max_dinkelbach=2, max_scale=6, max_dual=60)
    insts = make_workload(name)[:1] if name != "batch" else _batch_subset(count=2)
    gs = gpu_solve(insts, tol)
    for inst, g in zip(insts, gs):
        o = oracle.solve(inst, tol)
        assert g["iters"] == o.iters
        compare(inst, g, o, "fixed-count " + name)


def _batch_subset(count=4, max_cost=40000):
    out = []
    i = 0
    while len(out) < count:
        inst = make_workload("batch-4096-uneven", count=1, start=i)[0]
        if inst.cost <= max_cost:
            out.append(inst)
        i += 1
    return out


def test_uneven_batch_in_one_launch_matches_oracle():
    insts = _batch_subset(count=6)
    tol = WORKLOADS["batch-4096-uneven"]["tol"]
    gs = gpu_solve(insts, tol)
    tiers = [hold(inst, g, tol, "seed%d M%d N%d K%d" % (inst.seed, inst.M, inst.N, inst.K))[0]
             for inst, g in zip(insts, gs)]
    print("uneven batch tiers", tiers)
    assert tiers.count("plain") >= len(tiers) - 1


def test_repeat_runs_are_bitwise_identical():
    insts = _batch_subset(count=3)
    tol = WORKLOADS["batch-4096-uneven"]["tol"]
    a = gpu_solve(insts, tol)
    b = gpu_solve(insts, tol)
    for x, y in zip(a, b):
        assert x["ee"] == y["ee"]
        assert np.array_equal(x["p"], y["p"]) and np.array_equal(x["S"], y["S"])


@pytest.mark.parametrize("shape", [
    dict(M=1, N=4, K=3, Ks=0, l=1),      # one RRH, OMA
    dict(M=2, N=1, K=1, Ks=0, l=1),      # one user, one subcarrier
    dict(M=3, N=5, K=4, Ks=4, l=2),      # streaming only: R = 0, EE = 0
    dict(M=4, N=3, K=9, Ks=0, l=3),      # elastic only
    dict(M=64, N=2, K=80, Ks=10, l=4),   # largest RRH count, M*l at the 256-slot cap
    dict(M=16, N=3, K=40, Ks=5, l=8),    # largest NOMA cap
])
def test_edge_shapes_match_oracle(shape):
    inst = make_instance(4242, **shape)
    tol = Tolerances()
    g = gpu_solve([inst], tol)[0]
    if shape["Ks"] == shape["K"]:
        o = oracle.solve(inst, tol)
        assert g["ee"] == 0.0 and o.ee == 0.0
        assert np.array_equal(g["S"], o.S)
        return
    hold(inst, g, tol, str(shape))


def _solver(insts):
    import torch
    from paper_1803_07772_gb300 import Solver
    gains, offs = pack_batch(insts)
    st = torch.cuda.Stream(device="cuda:0")
    s = Solver(insts, gain_offsets=offs, device="cuda:0", stream=st)
    return s, torch.from_numpy(gains).to("cuda:0")


def test_graph_replay_matches_direct_launches():
    from paper_1803_07772_gb300 import make_tol
    insts = _batch_subset(count=6)
    s, g = _solver(insts)
    tol = make_tol(WORKLOADS["batch-4096-uneven"]["tol"], max_dinkelbach=2, max_scale=4)
    s.solve(g, tol)
    direct = [s.get(i) for i in range(len(insts))]
    for _ in range(2):  # capture, then replay
        s.solve_graph(g, tol)
        for i, d in enumerate(direct):
            r = s.get(i)
            assert r["ee"] == d["ee"] and np.array_equal(r["p"], d["p"]) and np.array_equal(r["S"], d["S"])
    tol2 = make_tol(WORKLOADS["batch-4096-uneven"]["tol"], max_dinkelbach=1, max_scale=3)
    s.solve_graph(g, tol2)  # new arguments: re-capture
    got = [s.get(i)["ee"] for i in range(len(insts))]
    s.solve(g, tol2)
    assert got == [s.get(i)["ee"] for i in range(len(insts))]


def test_every_cluster_size_matches_oracle_at_fixed_counts():
    """The same instances forced onto clusters of 1 to 8 CTAs (where
    the state fits and N allows) and onto the streamed schedule: fixed
    iteration counts, every selected power held to the strict bar."""
    insts = _batch_subset(count=3)
    tol = Tolerances(tol_dinkelbach=0.0, tol_scale=0.0, tol_dual=0.0,
                     max_dinkelbach=2, max_scale=3, max_dual=40)
    orcs = [oracle.solve(i, tol) for i in insts]
    from paper_1803_07772_gb300 import make_tol
    s, g = _solver(insts)
    base = s.schedule()
    for want in [0, 1, 2, 3, 4, 5, 6, 7, 8]:
        sched = np.array([want if (want == 0 or (want >= b and i.N >= want)) else b
                          for i, b in zip(insts, base)], np.int32)
        s.set_schedule(sched)
        s.solve(g, make_tol(tol, tie_eps=TIE_BAND))
        for i, (inst, o) in enumerate(zip(insts, orcs)):
            r = s.get(i)
            assert r["iters"] == o.iters
            compare(inst, r, o, "schedule %d (got %d)" % (want, s.schedule()[i]))


def test_team_sweeps_match_oracle_at_fixed_counts():
    """The streamed schedule with its warps in 1 to 4 teams that each stage
    one subcarrier at a time (the planner's choice for instances whose warp
    buffers do not fit, such as the 33 x 1024 x 512 shape), forced on batch
    instances and the medium configuration: fixed iteration counts, every
    selected power held to the strict bar."""
    insts = _batch_subset(count=3) + make_workload("medium-9x64x48")
    tol = Tolerances(tol_dinkelbach=0.0, tol_scale=0.0, tol_dual=0.0,
                     max_dinkelbach=2, max_scale=3, max_dual=40)
    orcs = [oracle.solve(i, tol) for i in insts]
    from paper_1803_07772_gb300 import make_tol
    s, g = _solver(insts)
    for teams in [1, 2, 3, 4]:
        s.set_schedule(np.full(len(insts), -teams, np.int32))
        s.solve(g, make_tol(tol, tie_eps=TIE_BAND))
        for i, (inst, o) in enumerate(zip(insts, orcs)):
            r = s.get(i)
            assert r["iters"] == o.iters
            compare(inst, r, o, "%d teams" % teams)


def test_autotune_picks_a_team_count_for_the_streamed_class():
    """Instances on the streamed schedule with team sweeps: the autotuner
    times every team count that fits and keeps one; the solve then still
    matches the oracle at fixed counts."""
    from paper_1803_07772_gb300 import make_tol
    insts = _batch_subset(count=3)
    tol = Tolerances(tol_dinkelbach=0.0, tol_scale=0.0, tol_dual=0.0,
                     max_dinkelbach=2, max_scale=3, max_dual=40)
    s, g = _solver(insts)
    s.set_schedule(np.full(len(insts), -4, np.int32))
    assert s.stream_teams() == 4
    s.autotune(g, make_tol(tol, tie_eps=TIE_BAND), max_dual_probe=20)
    t = s.stream_teams()
    print("team count after autotune", t)
    assert 1 <= t <= 4
    s.solve(g, make_tol(tol, tie_eps=TIE_BAND))
    for i, inst in enumerate(insts):
        r = s.get(i)
        o = oracle.solve(inst, tol)
        assert r["iters"] == o.iters
        compare(inst, r, o, "%d teams (autotuned)" % t)


def test_autotuned_schedule_is_valid_and_matches_oracle():
    from paper_1803_07772_gb300 import make_tol
    insts = _batch_subset(count=4)
    s, g = _solver(insts)
    tol = Tolerances(tol_dinkelbach=0.0, tol_scale=0.0, tol_dual=0.0,
                     max_dinkelbach=2, max_scale=3, max_dual=40)
    before = s.schedule()
    after = s.autotune(g, make_tol(tol, tie_eps=TIE_BAND), max_dual_probe=20)
    print("schedule before", before, "after autotune", after)
    assert np.all((after == 0) | (after >= before))
    s.solve(g, make_tol(tol, tie_eps=TIE_BAND))
    for i, inst in enumerate(insts):
        compare(inst, s.get(i), oracle.solve(inst, tol), "autotuned")


def test_large_instance_matches_oracle_at_fixed_counts():
    """The 33 x 1024 x 512 shape (l = 4): its dual-loop state (about 24 MB)
    fits no cluster, so it runs the streamed single-CTA schedule; one
    Dinkelbach iteration, two SCALE passes of 10 dual iterations, every
    selected power held to the strict bar."""
    inst = make_workload("large-33x1024x512", count=1)[0]
    tol = Tolerances(tol_dinkelbach=0.0, tol_scale=0.0, tol_dual=0.0,
                     max_dinkelbach=1, max_scale=2, max_dual=10)
    g = gpu_solve([inst], tol)[0]
    o = oracle.solve(inst, tol)
    assert g["iters"] == o.iters
    compare(inst, g, o, "large fixed-count")



def test_large_instance_first_dinkelbach_iteration_under_its_stop_rules():
    """The 33 x 1024 x 512 shape through one whole Dinkelbach iteration with
    the workload's own SCALE and dual stop rules (varpi_1, varpi_2, S = 50,
    V = 200): the plain bar, with the tiers of tests.parity."""
    inst = make_workload("large-33x1024x512", count=1)[0]
    tol = copy.copy(WORKLOADS["large-33x1024x512"]["tol"])
    tol.max_dinkelbach = 1
    g = gpu_solve([inst], tol)[0]
    tier, rep = hold(inst, g, tol, "large, one Dinkelbach iteration")
    assert tier in ("plain", "tie", "stop"), rep
