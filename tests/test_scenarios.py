"""The architectures compared in Sec. VI as workloads: H-CRAN with PD-NOMA
and with OMA (at most one user per subcarrier of an RRH), 1-tier C-RAN (three
LPN RRHs), 2-tier HCN (one macro and two pico BSs) and 1-tier HPN (two macro
BSs).  The same kernels run them with other constants; the oracle is held to
the constraints of problem (eq7) on them, and the GPU path to the oracle."""
import numpy as np
import pytest

import oracle
from hcran_inputs import Tolerances, WORKLOADS, make_workload
from hcran_inputs.gen import SCENARIOS


def test_scenarios_carry_the_paper_constants():
    by = {n: make_workload(n, count=1)[0] for n in SCENARIOS}
    for inst in by.values():
        assert (inst.N, inst.K, inst.Ks) == (32, 12, 6)
        assert np.all(inst.lambda_pps == 125.0) and np.all(inst.T_s == 0.2)
    assert by["scenario-hcran-noma"].M == 3 and by["scenario-hcran-noma"].l == 3
    assert by["scenario-hcran-oma"].l == 1
    assert np.array_equal(by["scenario-hcran-oma"].G, by["scenario-hcran-noma"].G)
    cran = by["scenario-cran-1tier"]
    assert cran.M == 3 and np.all(cran.pmax == 1.0) and np.all(cran.Pc == 1.0)
    hcn = by["scenario-hcn-2tier"]
    assert list(hcn.Pc) == [10.0, 6.8, 6.8] and np.all(hcn.eta == 4.0) and np.all(hcn.Pf == 0.0)
    hpn = by["scenario-hpn-1tier"]
    assert hpn.M == 2 and np.all(hpn.pmax == 40.0) and np.all(hpn.Pc == 10.0) and np.all(hpn.eta == 4.0)


@pytest.mark.parametrize("name", SCENARIOS)
def test_oracle_solution_meets_the_constraints(name):
    """C1 (at most l users per RRH and subcarrier; one under OMA), C5 (a user
    is served by its one chosen RRH), C4 (spectral mask), C12 (power budget),
    and a positive finite EE, on two instances of each scenario."""
    for inst in make_workload(name, count=2):
        o = oracle.solve(inst, WORKLOADS[name]["tol"])
        S, p = np.asarray(o.S), np.asarray(o.p)
        assert S.shape == (inst.N, inst.M, inst.l)
        sel = S >= 0
        assert np.all(sel.sum(axis=2) <= inst.l)
        for n in range(inst.N):
            for m in range(inst.M):
                ks = S[n, m][S[n, m] >= 0]
                assert len(set(ks.tolist())) == len(ks)
                for k in ks:
                    assert o.A[k] == m  # C5: served only by its chosen RRH
        mask = inst.pmax / inst.N
        assert np.all(p[sel] <= mask[None, :, None].repeat(inst.N, 0).repeat(inst.l, 2)[sel] * (1 + 1e-9))
        tot = np.where(sel, p, 0.0).sum(axis=(0, 2))
        assert np.all(tot <= inst.pmax * (1 + 1e-9))
        assert np.isfinite(o.ee) and o.ee > 0.0


@pytest.mark.gpu
def test_scenarios_match_oracle_at_fixed_counts():
    """Stop tests off (every loop runs to its cap): the plain bar, with the
    same iteration counts on both sides, on three instances of every
    architecture."""
    from tests.test_gpu_parity import compare, gpu_solve
    tol = Tolerances(tol_dinkelbach=0.0, tol_scale=0.0, tol_dual=0.0, max_dinkelbach=2, max_scale=3, max_dual=40)
    for name in SCENARIOS:
        insts = make_workload(name, count=3)
        for inst, g in zip(insts, gpu_solve(insts, tol)):
            o = oracle.solve(inst, tol)
            assert g["iters"] == o.iters
            compare(inst, g, o, "fixed-count %s seed %d" % (name, inst.seed))


@pytest.mark.gpu
def test_scenarios_match_oracle_under_their_stop_rules():
    """With the workloads' own stop rules, three instances of every
    architecture held to the tiers of tests.parity; at least 85 % of them on
    the plain bar (measured: 13 of 15, the other two OMA instances, one whose
    oracle end point is itself rounding-sensitive and one whose stop test
    fired one SCALE pass apart)."""
    from tests.test_gpu_parity import gpu_solve, hold
    tiers = []
    for name in SCENARIOS:
        tol = WORKLOADS[name]["tol"]
        insts = make_workload(name, count=3)
        for inst, g in zip(insts, gpu_solve(insts, tol)):
            tiers.append(hold(inst, g, tol, "%s seed %d" % (name, inst.seed))[0])
    print("scenario tiers", tiers)
    assert tiers.count("plain") >= 0.85 * len(tiers), tiers
