"""hcran_set_state: a solve stopped by its Dinkelbach cap, exported with
hcran_get and imported again, continues exactly where the uninterrupted solve
would be (Sec. III carries p^{i-1} and its multipliers into iteration i)."""
import numpy as np
import pytest

from hcran_inputs import WORKLOADS, make_workload, pack_batch
from tests.test_gpu_parity import _batch_subset

pytestmark = pytest.mark.gpu


def _solver(insts):
    import torch
    from paper_1803_07772_gb300 import Solver
    gains, offs = pack_batch(insts)
    st = torch.cuda.Stream(device="cuda:0")
    s = Solver(insts, gain_offsets=offs, device="cuda:0", stream=st)
    return s, torch.from_numpy(gains).to("cuda:0")


def test_resumed_solve_equals_the_uninterrupted_one():
    from paper_1803_07772_gb300 import make_tol
    insts = make_workload("medium-9x64x48") + _batch_subset(count=4)
    tol = WORKLOADS["batch-4096-uneven"]["tol"]
    s, g = _solver(insts)
    s.solve(g, make_tol(tol, max_dinkelbach=6))
    whole = [s.get(i) for i in range(len(insts))]
    s.solve(g, make_tol(tol, max_dinkelbach=2))
    first = [s.get(i) for i in range(len(insts))]
    for i, r in enumerate(first):
        s.set_state(i, r)
    s.solve(g, make_tol(tol, max_dinkelbach=4))
    rest = [s.get(i) for i in range(len(insts))]
    resumed = 0
    for i, (a, b, c) in enumerate(zip(whole, first, rest)):
        if not (b["status"] & 1):  # converged within two iterations: nothing to resume
            continue
        resumed += 1
        assert np.array_equal(c["S"], a["S"]) and np.array_equal(c["A"], a["A"]), i
        assert np.array_equal(c["p"], a["p"]), i
        assert c["ee"] == a["ee"], (i, c["ee"], a["ee"])
        assert np.array_equal(c["xi"], a["xi"]) and np.array_equal(c["zeta"], a["zeta"]), i
        assert [x + y for x, y in zip(b["iters"], c["iters"])] == list(a["iters"]), (i, b["iters"], c["iters"], a["iters"])
    assert resumed >= 3
    # the state applied to one solve only: the next solve starts cold again
    s.solve(g, make_tol(tol, max_dinkelbach=6))
    again = [s.get(i) for i in range(len(insts))]
    for a, b in zip(whole, again):
        assert a["ee"] == b["ee"] and np.array_equal(a["p"], b["p"])


def test_graph_and_autotune_refuse_a_pending_state():
    from paper_1803_07772_gb300 import make_tol
    from paper_1803_07772_gb300.hcran import HcranError
    insts = _batch_subset(count=2)
    s, g = _solver(insts)
    tol = make_tol(WORKLOADS["batch-4096-uneven"]["tol"], max_dinkelbach=1, max_scale=2)
    s.solve(g, tol)
    s.set_state(0, s.get(0))
    with pytest.raises(HcranError) as e:
        s.solve_graph(g, tol)
    assert e.value.code == 1
    with pytest.raises(HcranError):
        s.autotune(g, tol, max_dual_probe=8)
    s.solve(g, tol)          # consumes the state
    s.solve_graph(g, tol)    # then the graph path is open again
