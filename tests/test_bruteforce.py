"""The global-optimum comparator on the GPU (hcran_bruteforce) against the
oracle's (orc_bruteforce), and the gap of the method to that optimum."""
import numpy as np
import pytest

import oracle
from hcran_inputs import WORKLOADS, make_instance, make_workload, pack_batch

pytestmark = pytest.mark.gpu


def _gpu_bf(insts):
    import torch
    from paper_1803_07772_gb300.hcran import bruteforce
    gains, _ = pack_batch(insts)
    return bruteforce(insts, torch.from_numpy(gains).to("cuda:0"))


@pytest.mark.parametrize("shape", [(2, 1, 3, 2), (1, 2, 3, 2), (3, 2, 3, 2), (2, 2, 3, 1)])
def test_gpu_comparator_matches_the_oracle(shape):
    M, N, K, l = shape
    insts = [make_instance(810000 + i, M=M, N=N, K=K, Ks=0, l=l) for i in range(6)]
    ee, idx, na = _gpu_bf(insts)
    for inst, e, i in zip(insts, ee, idx):
        oe, ona, oi = oracle.bruteforce(inst)
        print(shape, inst.seed, "gpu %.12g (#%d) oracle %.12g (#%d)" % (e, i, oe, oi))
        assert na == ona
        assert e == pytest.approx(oe, rel=1e-9)
        assert i == oi


def test_method_gap_to_the_optimum():
    """The CUDA solve of the method on 64 instances of the optimum workload
    never beats the comparator's optimum and stays close to it; the paper
    calls its solution close to the optimal one (Sec. VI)."""
    import torch
    from paper_1803_07772_gb300 import Solver, make_tol
    name = "optimum-3x2x3"
    insts = make_workload(name, count=64)
    ee_opt, _, _ = _gpu_bf(insts)
    gains, offs = pack_batch(insts)
    s = Solver(insts, gain_offsets=offs, device="cuda:0")
    s.solve(torch.from_numpy(gains).to("cuda:0"), make_tol(WORKLOADS[name]["tol"]))
    ee = s.summary()["ee"]
    ratio = ee / ee_opt
    print("method / optimum: min %.4f median %.4f mean %.4f, within 1 %%: %.2f" % (
        ratio.min(), np.median(ratio), ratio.mean(), np.mean(ratio >= 0.99)))
    assert np.all(ratio <= 1 + 1e-6)
    assert np.median(ratio) >= 0.99
