"""The bench's multi-rank path on CPU: two gloo ranks (no GPU), the same
helpers a torchrun launch uses: disjoint per-rank instance seeds, the step
time as the maximum over ranks, and the job value over every rank."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    import bench
    from hcran_inputs import make_workload
    r, w, local = bench.rank_env()
    dist.init_process_group("gloo", rank=r, world_size=w)
    count = 3
    insts = make_workload(bench.WORKLOAD, count=count, start=bench.rank_seed_start(r, count))
    seeds = [int(i.seed) for i in insts]
    step_s = 0.5 + r  # a rank-dependent step time
    slowest = bench.max_over_ranks(step_s, "cpu", w)
    gathered = [None] * w
    dist.all_gather_object(gathered, seeds)
    out.put((r, local, seeds, slowest, gathered, bench.job_value(w, count, slowest)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_disjoint_batches_and_the_slowest_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=240) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    all_seeds = [s for r in res for s in r[2]]
    assert len(set(all_seeds)) == len(all_seeds) == 6  # disjoint batches
    for r, local, seeds, slowest, gathered, value in res:
        assert local == r
        assert slowest == pytest.approx(1.5)  # the maximum over ranks
        assert gathered == [res[0][2], res[1][2]]
        assert value == pytest.approx(2 * 3 / 1.5)  # every rank's instances over the slowest time
