"""Sharding of independent search queries over processes (one process per GPU).

Pairs and queries are independent units of the search (Sec. 3: each pair is searched on its
own), so N processes take every N-th query and gather their found windows at the end; the
data path needs no collective.  The distributed design of the paper (Sec. 7.2, Spark map /
collect over overlapping chunks) is not reproduced: a GPU holds a whole pair.
"""
from __future__ import annotations


def shard(items, rank: int, world: int):
    """The items this rank handles: every world-th item starting at rank (keeps the global
    order within the shard and balances long and short queries)."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad rank / world size")
    return list(items[rank::world])


def shard_indices(n: int, rank: int, world: int):
    return list(range(rank, n, world))


def gather(local_results, rank: int, world: int, n: int, group=None):
    """Collect every rank's results into global order on rank 0 (None elsewhere)."""
    if world == 1:
        return list(local_results)
    import torch.distributed as dist
    payload = list(zip(shard_indices(n, rank, world), local_results))
    gathered = [None] * world if rank == 0 else None
    dist.gather_object(payload, gathered, dst=0, group=group)
    if rank != 0:
        return None
    out = [None] * n
    for part in gathered:
        for i, r in part:
            out[i] = r
    return out


def sharded_map(fn, queries, rank: int, world: int, group=None):
    """Run fn on this rank's queries and gather the results in query order on rank 0."""
    local = [fn(q) for q in shard(queries, rank, world)]
    return gather(local, rank, world, len(queries), group=group)
