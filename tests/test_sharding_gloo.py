"""Key-range sharding: the exchange of verified divisor sets between shards.
Two gloo ranks on CPU run sharding.torch_gather (the all-gather a sharded
batch calls between verification and the atoms); threads check the
in-process exchange.  No GPU involved."""
import os
import sys
import threading

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2410_15880_b300.sharding import torch_gather
    g = torch_gather()
    mine = [(0, 1 << (60 + rank), 0), (3, rank, 1 << 63)] if rank == 0 else [(1, (1 << 64) - 1, 5)]
    first = g(mine)
    second = g([])                                  # a shard with nothing to send still takes part
    q.put((rank, first, second))
    dist.barrier()
    dist.destroy_process_group()


def test_torch_gather_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, 29741, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    want = [(0, 1 << 60, 0), (3, 0, 1 << 63), (1, (1 << 64) - 1, 5)]   # rank order, 64-bit values intact
    assert out[0][1] == out[1][1] == want
    assert out[0][2] == out[1][2] == []


def test_thread_exchange():
    from paper_2410_15880_b300.sharding import ThreadExchange
    ex = ThreadExchange(3, timeout=30)
    res = [None] * 3

    def run(s):
        res[s] = ex.gather_for(s)([(s, s, s)] * s)
    th = [threading.Thread(target=run, args=(s,)) for s in range(3)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert res[0] == res[1] == res[2] == [(1, 1, 1), (2, 2, 2), (2, 2, 2)]


class _FakeShardContext:
    """Stands in for Context on CPU: shard s "verifies" the items i with
    i % nshards == s, exchanges them through gather, and answers every item
    with the shards that reported it, so a result depends on the exchange."""

    def factor_batch_sharded(self, polys, shard, nshards, gather):
        from paper_2410_15880_b300._native import Result
        mine = [(i, shard, 7) for i in range(len(polys)) if i % nshards == shard]
        everyone = gather(mine)
        return [Result(status=0, factors=[[t[1] for t in everyone if t[0] == i]]) for i in range(len(polys))]


def _bench_rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2410_15880_b300.sharding import torch_gather
    polys = [[1, 0, 1]] * 5
    golden = [[[i % world]] for i in range(5)]
    ms, res, ok = bench.sharded_leg(_FakeShardContext(), polys, rank, world, steps=3, warmup=1,
                                    gather=torch_gather(), golden=golden, barrier=dist.barrier)
    q.put((rank, ms, [r.factors for r in res], ok))
    dist.barrier()
    dist.destroy_process_group()


def test_bench_sharded_leg_two_ranks():
    """The bench's --shard wiring: both ranks factor the same batch, the
    all-gather makes their results whole and equal, and the step time is the
    max over the ranks."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_bench_rank_main, args=(r, 2, 29751, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, ms0, f0, ok0), (_, ms1, f1, ok1) = out
    assert ok0 and ok1 and f0 == f1 == [[[i % 2]] for i in range(5)]
    assert ms0 == ms1 > 0
