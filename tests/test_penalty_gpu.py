"""Penalty form of C10 / C11 on the GPU (hcran_penalty_solve) against the
penalty-form oracle (oracle/hcran_penalty.c), through the C ABI.

Both sides compute in FP64 without FMA contraction and sum in the order the
definitions list, so the bar is tight: powers within 1e-9 relative plus
1e-12 of the mask, EE within 1e-9, equal iteration counts."""
import numpy as np
import pytest

import oracle.oracle as oo
from hcran_inputs import Tolerances, WORKLOADS, make_instance, make_workload, pack_batch

pytestmark = pytest.mark.gpu


def _gpu(insts, tol, rho_rel=1e-3):
    import torch
    from paper_1803_07772_gb300 import make_tol
    from paper_1803_07772_gb300.hcran import penalty_solve
    gains, _ = pack_batch(insts)
    g = torch.from_numpy(gains).to("cuda:0")
    return penalty_solve(insts, g, make_tol(tol), rho_rel=rho_rel)


def _compare(insts, tol, rho_rel=1e-3, label=""):
    out = _gpu(insts, tol, rho_rel)
    worst = 0.0
    for b, inst in enumerate(insts):
        o = oo.penalty_solve(inst, tol, rho_rel=rho_rel)
        mask = np.asarray(inst.pmax)[None, :, None] / inst.N
        err = np.abs(out["p"][b] - o.p) - 1e-9 * o.p - 1e-12 * mask
        rel = abs(out["ee"][b] - o.ee) / o.ee
        worst = max(worst, rel)
        print(label, b, "ee gpu %.12g oracle %.12g rel %.2e iters %s %s" % (out["ee"][b], o.ee, rel,
                                                                          tuple(out["iters"][b]), o.iters))
        assert tuple(out["iters"][b]) == o.iters
        assert np.all(err <= 0.0), np.max(err)
        assert rel <= 1e-9
        assert out["c10_max"][b] == pytest.approx(o.c10_max, rel=1e-6, abs=1e-12)
        assert out["c11_max"][b] == pytest.approx(o.c11_max, rel=1e-6, abs=1e-12)
    return worst


def test_penalty_form_matches_oracle_at_fixed_counts():
    tol = Tolerances(tol_dinkelbach=0.0, tol_scale=0.0, tol_dual=0.0,
                     max_dinkelbach=2, max_scale=3, max_dual=50)
    _compare(make_workload("optimum-3x2x3", count=6), tol, label="3x2x3 fixed")


@pytest.mark.parametrize("shape", [dict(M=2, N=2, K=6, Ks=0, l=2), dict(M=4, N=4, K=8, Ks=0, l=3),
                                   dict(M=1, N=3, K=4, Ks=0, l=1)])
def test_penalty_form_shapes_match_oracle(shape):
    """Other shapes, the largest the call takes (128 links) included, under
    the workloads' stop rules."""
    insts = [make_instance(900000 + i, **shape) for i in range(3)]
    _compare(insts, Tolerances(), label=str(shape))


def test_penalty_form_matches_oracle_under_stop_rules():
    name = "optimum-3x2x3"
    _compare(make_workload(name, count=16), WORKLOADS[name]["tol"], label=name)
