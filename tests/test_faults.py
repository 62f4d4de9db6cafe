"""Failure paths, exercised without faulting the GPU: a bounded device wait
that gives up (a barrier nothing completes, no copy in flight) and gains that
are not finite or negative.  Each affects its own instance only."""
import numpy as np
import pytest

from hcran_inputs import WORKLOADS, pack_batch
from tests.test_gpu_parity import _batch_subset

pytestmark = pytest.mark.gpu

ST_NUMERIC, ST_TIMEOUT = 8, 16
ETIMEDOUT, ENUMERIC = 4, 5


def _run(insts, gains_np, stall=-1, tries=0):
    import torch
    from paper_1803_07772_gb300 import Solver, make_tol
    _, offs = pack_batch(insts)
    s = Solver(insts, gain_offsets=offs, device="cuda:0")
    s.set_wait_limit(tries, stall)
    g = torch.from_numpy(gains_np).to("cuda:0")
    tol = make_tol(WORKLOADS["batch-4096-uneven"]["tol"], max_dinkelbach=2, max_scale=4)
    s.solve(g, tol)
    out = [s.get(i) for i in range(len(insts))]
    host = s.solve_host(torch.from_numpy(gains_np).pin_memory(), tol)
    return out, host


def _same(a, b):
    return a["ee"] == b["ee"] and np.array_equal(a["p"], b["p"]) and np.array_equal(a["S"], b["S"])


def test_a_wait_that_gives_up_reports_a_timeout_on_its_instance_only():
    insts = _batch_subset(count=3)
    gains, _ = pack_batch(insts)
    clean, _ = _run(insts, gains)
    got, (ee_h, st_h) = _run(insts, gains, stall=1, tries=1000)
    assert got[1]["rc"] == ETIMEDOUT and got[1]["status"] & ST_TIMEOUT
    assert st_h[1] & ST_TIMEOUT
    for i in (0, 2):
        assert got[i]["rc"] == 0 and not (got[i]["status"] & ST_TIMEOUT)
        assert _same(got[i], clean[i]), i
        assert ee_h[i] == clean[i]["ee"]
    # the context is still usable: a clean solve afterwards matches
    again, _ = _run(insts, gains)
    assert all(_same(a, b) for a, b in zip(again, clean))


@pytest.mark.parametrize("bad", [np.nan, np.inf, -1e-12])
def test_a_bad_gain_flags_its_instance_only(bad):
    insts = _batch_subset(count=3)
    gains, offs = pack_batch(insts)
    clean, _ = _run(insts, gains)
    dirty = gains.copy()
    dirty[offs[1] + 7] = bad
    got, (ee_h, st_h) = _run(insts, dirty)
    assert got[1]["rc"] == ENUMERIC and got[1]["status"] & ST_NUMERIC
    assert st_h[1] & ST_NUMERIC
    for i in (0, 2):
        assert got[i]["rc"] == 0 and _same(got[i], clean[i]), i
