"""The multi-GPU form is replicas: each rank factors its own batch (seed
3 + 1000 * rank) and the step time is the max over ranks.  Checked here with
two gloo ranks on CPU (no GPU involved)."""
import os
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    insts = bench.workload("cfg3", rank, 4)
    t = bench.max_over_ranks(10.0 + rank, world)
    q.put((rank, [tuple(i.coeffs) for i in insts], t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_distinct_work_and_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29731
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    (_, polys0, t0), (_, polys1, t1) = out
    assert t0 == t1 == 11.0                      # both ranks see the slowest replica's time
    assert not set(polys0) & set(polys1)         # replicas factor different polynomials
    assert all(len(p) == 101 for p in polys0 + polys1)
