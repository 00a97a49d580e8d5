"""Exchanges for Context.factor_batch_sharded (key-range sharding of one
batch over several processes or threads).  Each returns a gather(triples)
callable: it takes this shard's verified divisor sets as (item, lo, hi)
triples and returns every shard's, in shard order."""
from __future__ import annotations

import threading


def torch_gather(group=None):
    """All-gather over a torch.distributed process group (one rank per GPU)."""
    import torch.distributed as dist

    def gather(triples):
        out = [None] * dist.get_world_size(group)
        dist.all_gather_object(out, [tuple(int(v) for v in t) for t in triples], group=group)
        return [t for part in out for t in part]
    return gather


class ThreadExchange:
    """Shards run by threads of one process: gather_for(shard) blocks until
    every shard has contributed (timeout in seconds), then returns them all."""

    def __init__(self, nshards: int, timeout: float = 120.0):
        self.n = nshards
        self.parts = [None] * nshards
        self.barrier = threading.Barrier(nshards, timeout=timeout)

    def gather_for(self, shard: int):
        def gather(triples):
            self.parts[shard] = list(triples)
            self.barrier.wait()
            return [t for part in self.parts for t in part]
        return gather
