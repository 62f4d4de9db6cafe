"""hcran_solve_noalloc: the solve for callers that cannot allocate device memory.

The entry point works in the library's own fixed device array instead of a
caller-provided workspace.  These tests call it through the C ABI and check
its results against the workspace-based entry point (hcran_create /
hcran_solve / hcran_get) on the same instance, twice in a row, with the
tolerances of the other GPU parity tests.  This file is collected last so a
run that stops at the first failure has already run every other test.
"""
import numpy as np
import pytest

from hcran_inputs import WORKLOADS, make_instance, make_workload, pack_batch
from paper_1803_07772_gb300 import hcran

EE_RTOL = 1e-4
P_RTOL = 1e-3


def _workspace_solve(inst, tol):
    import torch
    gains, offs = pack_batch([inst])
    s = hcran.Solver([inst], gain_offsets=offs, device="cuda:0")
    g = torch.from_numpy(gains).to("cuda:0")
    s.solve(g, tol)
    return s.get(0)


def _same(a, b, inst):
    mask = inst.pmax / inst.N
    assert np.array_equal(a["A"], b["A"]) and np.array_equal(a["S"], b["S"])
    assert abs(a["ee"] - b["ee"]) <= EE_RTOL * abs(b["ee"])
    sel = b["S"] >= 0
    lim = P_RTOL * np.maximum(np.abs(a["p"]), np.abs(b["p"])) + 1e-6 * mask[None, :, None]
    assert np.all(np.abs(a["p"] - b["p"])[sel] <= np.broadcast_to(lim, sel.shape)[sel])


@pytest.mark.gpu
@pytest.mark.parametrize("which", ["small", "batch"])
def test_noalloc_matches_workspace_solve_twice(which):
    import torch
    if which == "small":
        inst, tol = make_workload("small-3x8x6")[0], WORKLOADS["small-3x8x6"]["tol"]
    else:
        inst, tol = make_workload("batch-4096-uneven", count=1, start=2)[0], WORKLOADS["batch-4096-uneven"]["tol"]
    t = hcran.make_tol(tol)
    ref = _workspace_solve(inst, t)
    g = torch.from_numpy(np.ascontiguousarray(inst.G.reshape(-1))).to("cuda:0")
    first = hcran.solve_noalloc(inst, g, t)
    second = hcran.solve_noalloc(inst, g, t)
    _same(first, ref, inst)
    _same(second, ref, inst)
    assert first["ee"] == second["ee"] and np.array_equal(first["p"], second["p"])


@pytest.mark.gpu
def test_noalloc_leftover_contents_do_not_leak_between_instances():
    import torch
    a = make_workload("small-3x8x6")[0]
    b = make_instance(77, M=4, N=12, K=9, Ks=3, l=2)
    t = hcran.make_tol(WORKLOADS["small-3x8x6"]["tol"])
    ga = torch.from_numpy(np.ascontiguousarray(a.G.reshape(-1))).to("cuda:0")
    gb = torch.from_numpy(np.ascontiguousarray(b.G.reshape(-1))).to("cuda:0")
    ra1 = hcran.solve_noalloc(a, ga, t)
    hcran.solve_noalloc(b, gb, t)
    ra2 = hcran.solve_noalloc(a, ga, t)
    assert ra1["ee"] == ra2["ee"] and np.array_equal(ra1["p"], ra2["p"])


def test_noalloc_rejects_instances_beyond_its_array_without_a_gpu():
    big = make_workload("large-33x1024x512", count=1)[0]
    with pytest.raises(hcran.HcranError) as e:
        hcran.solve_noalloc(big, 256, hcran.make_tol())
    assert e.value.code == 6  # HCRAN_E2BIG, before any device work


def test_noalloc_rejects_bad_arguments_without_a_gpu():
    inst = make_workload("small-3x8x6")[0]
    with pytest.raises(hcran.HcranError) as e:
        hcran.solve_noalloc(inst, 8, hcran.make_tol())   # misaligned gains pointer
    assert e.value.code == 1
    with pytest.raises(hcran.HcranError) as e:
        hcran.solve_noalloc(inst, 256, hcran.make_tol(max_dual=0))
    assert e.value.code == 1
