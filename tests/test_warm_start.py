"""Learned warm start through the C ABI: the features of the initial
selection, a warm start that encodes the cold point (it must reproduce the
cold solve), and a trained network (valid solves; iterations and EE against
the cold solve reported)."""
import math

import numpy as np
import pytest

import oracle
from hcran_inputs import Tolerances, WORKLOADS, make_workload, pack_batch

pytestmark = pytest.mark.gpu


def _solver(insts):
    import torch
    from paper_1803_07772_gb300 import Solver
    gains, offs = pack_batch(insts)
    st = torch.cuda.Stream(device="cuda:0")
    s = Solver(insts, gain_offsets=offs, device="cuda:0", stream=st)
    return s, torch.from_numpy(gains).to("cuda:0")


def _subset(count, max_cost=40000, start=0):
    out, i = [], start
    while len(out) < count:
        inst = make_workload("batch-4096-uneven", count=1, start=i)[0]
        if inst.cost <= max_cost:
            out.append(inst)
        i += 1
    return out


def test_features_follow_their_definition():
    from paper_1803_07772_gb300.warmstart import row_offsets
    insts = _subset(3)
    s, g = _solver(insts)
    F = s.warm_features(g).float().cpu().numpy()
    offs, rows = row_offsets(insts)
    assert F.shape == (rows, 16) and s.warm_rows() == rows
    for b, inst in enumerate(insts):
        S0 = s.get(b)["S"]
        Up = (inst.M * inst.l + 3) // 4 * 4
        Ke = inst.K - inst.Ks
        for n in range(inst.N):
            for u in range(Up):
                row = F[offs[b] + n * Up + u]
                m, sl = divmod(u, inst.l)
                k = S0[n, m, sl] if u < inst.M * inst.l else -1
                if k < 0:
                    assert np.all(row == 0.0)
                    continue
                g_ = inst.G[n, m]
                want = [(math.log10(g_[k]) + 11.0) / 3.0, np.sum(g_ > g_[k]) / inst.K,
                        1.0 if k >= Ke else 0.0, (inst.T_s[k - Ke] / 0.1) if k >= Ke else 0.0]
                assert np.allclose(row[:4], want, rtol=2 ** -7, atol=2 ** -8), (b, n, u, row[:4], want)
                assert np.all(row[4:] == 0.0)


def test_cold_encoded_warm_start_reproduces_cold_solve():
    import torch
    from paper_1803_07772_gb300 import make_tol
    from paper_1803_07772_gb300.warmstart import cold_point_outputs
    insts = _subset(4)
    tol = Tolerances(tol_dinkelbach=0.0, tol_scale=0.0, tol_dual=0.0, max_dinkelbach=2, max_scale=3, max_dual=40)
    s, g = _solver(insts)
    s.solve(g, make_tol(tol))
    cold = [s.get(i) for i in range(len(insts))]
    y = torch.from_numpy(cold_point_outputs(insts)).to("cuda:0")
    s.solve_warm(g, make_tol(tol), y)
    warm = [s.get(i) for i in range(len(insts))]
    for inst, c, w in zip(insts, cold, warm):
        o = oracle.solve(inst, tol)
        assert np.array_equal(w["S"], c["S"]) and np.array_equal(w["S"], o.S)
        assert abs(w["ee"] - c["ee"]) <= 1e-6 * c["ee"]
        assert abs(w["ee"] - o.ee) <= 1e-4 * o.ee
        sel = o.S >= 0
        assert np.max(np.abs(w["p"][sel] - o.p[sel]) / o.p[sel]) <= 1e-3


def test_trained_warm_start_gives_valid_solves():
    import torch
    from paper_1803_07772_gb300 import make_tol
    from paper_1803_07772_gb300.mlp import MLP
    from paper_1803_07772_gb300.warmstart import TRAIN_SEED_BASE, build_dataset, train, warm_solve
    tol = make_tol(WORKLOADS["batch-4096-uneven"]["tol"])
    train_insts = make_workload("batch-4096-uneven", count=24, start=TRAIN_SEED_BASE - 300000)
    s, g = _solver(train_insts)
    X, Y, Mk = build_dataset(s, g, train_insts, tol)
    net = MLP(seed=5, max_rows=8192)
    hist = train(net, X, Y, Mk, epochs=6, batch=4096, lr=2e-3)
    print("train rows", X.shape[0], "loss per epoch", hist)
    assert not net.tc_failed()
    assert hist[-1] < hist[0]
    ev = _subset(6)
    se, ge = _solver(ev)
    se.solve(ge, tol)
    cold = [se.get(i) for i in range(len(ev))]
    warm_solve(se, net, ge, tol)
    warm = [se.get(i) for i in range(len(ev))]
    for c, w in zip(cold, warm):
        print("cold ee %.4f iters %s | warm ee %.4f iters %s" % (c["ee"], c["iters"], w["ee"], w["iters"]))
        assert np.isfinite(w["ee"]) and w["ee"] >= 0.0
        assert w["slack_power_min"] >= -1e-5


def test_warm_start_gain_against_the_exact_state_ceiling():
    """What the trained network gains over the cold solve under the acceptance
    rule (a warm result counts when its EE is within 1e-4 of the cold one,
    otherwise the instance is solved cold again), measured in dual iterations,
    the solver's unit of work; and the ceiling of any warm start: every
    instance resumed from the cold solve's own converged state."""
    from paper_1803_07772_gb300 import make_tol
    from paper_1803_07772_gb300.mlp import MLP
    from paper_1803_07772_gb300.warmstart import TRAIN_SEED_BASE, build_dataset, train, warm_solve
    tol = make_tol(WORKLOADS["batch-4096-uneven"]["tol"])
    train_insts = make_workload("batch-4096-uneven", count=48, start=TRAIN_SEED_BASE - 300000)
    s, g = _solver(train_insts)
    X, Y, Mk = build_dataset(s, g, train_insts, tol)
    net = MLP(seed=5, max_rows=8192)
    train(net, X, Y, Mk, epochs=6, batch=4096, lr=2e-3)
    ev = _subset(16)
    se, ge = _solver(ev)
    se.solve(ge, tol)
    cold = [se.get(i) for i in range(len(ev))]
    warm_solve(se, net, ge, tol)
    warm = [se.get(i) for i in range(len(ev))]
    for i, c in enumerate(cold):
        se.set_state(i, c)
    se.solve(ge, tol)
    exact = [se.get(i) for i in range(len(ev))]

    def gain(res):
        work_cold = sum(c["iters"][2] for c in cold)
        acc = [abs(r["ee"] - c["ee"]) <= 1e-4 * c["ee"] for r, c in zip(res, cold)]
        work = sum(r["iters"][2] for r in res) + sum(c["iters"][2] for c, a in zip(cold, acc) if not a)
        return work_cold / work, float(np.mean(acc))
    g_net, a_net = gain(warm)
    g_ex, a_ex = gain(exact)
    print("network: gain %.3f, accepted %.2f | exact state: gain %.3f, accepted %.2f" % (g_net, a_net, g_ex, a_ex))
    assert a_ex >= 0.9                      # the converged state is (nearly) a fixed point of the solve
    assert g_ex > 1.5                       # and resuming from it saves most of the work
    assert 0.0 < g_net <= g_ex * 1.05       # no predicted start does better than the exact one
