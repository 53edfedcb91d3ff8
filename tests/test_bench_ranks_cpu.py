"""The N > 1 path of bench.py (independent replicas, no data-path collective):
two gloo ranks on the CPU time different steps, and the whole-job rate uses
the slowest rank's step time and the units of both ranks."""
import os
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    r, w, _ = bench.dist_env()
    assert (r, w) == (rank, world)
    dist.barrier()
    ms_max, value = bench.whole_job_rate(1.0 + rank, 10.0, dist)
    out[rank] = (ms_max, value)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_take_the_slowest_step():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(90)
        assert p.exitcode == 0
    for r in range(2):
        ms_max, value = out[r]
        assert ms_max == 2.0
        assert value == pytest.approx(2 * 10.0 / 2e-3)
