"""bench.py's replica aggregation across ranks (gloo, world size 2, CPU)."""
import os
import sys

import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r solved 10 problems in (100 + 50 r) ms
    rate, ms = bench.job_rate(10, 100.0 + 50.0 * rank, world)
    q.put((rank, rate, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_job_rate_sums_units_over_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, rate, ms in out:
        assert ms == 150.0
        assert abs(rate - 20 / 0.150) < 1e-9
