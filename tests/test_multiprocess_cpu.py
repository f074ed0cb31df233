"""The N > 1 path on CPU: queries sharded over 2 gloo processes, gathered on rank 0, equal
to a single-process run (the per-rank search is the CPU oracle here: no GPU is needed to
test the sharding and gathering)."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2204_09131_gb300 import shard, synth


def _queries():
    x, y = synth.planted_small_pair(1200)
    qs = []
    for lo, hi, mode in ((0, 1200, 0), (100, 900, 1), (300, 1200, 0), (0, 600, 1), (250, 1000, 0)):
        qs.append((lo, hi, mode))
    return x, y, qs


def _run_query(q):
    from oracle import oracle as O
    x, y, _ = _queries()
    lo, hi, mode = q
    fn = O.search_td if mode == 0 else O.search_bu
    wins, _ = fn(x, y, t_begin=lo, t_end=hi, k=4, s_min=32, s_max=128, pruning=1, seed=5)
    return [(a, b) for a, b, _, _ in wins]


def _worker(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        _, _, qs = _queries()
        res = shard.sharded_map(_run_query, qs, rank, world)
        if rank == 0:
            import json
            with open(out_path, "w") as f:
                json.dump(res, f)
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_shard_covers_every_query_once():
    for world in (1, 2, 3, 5):
        seen = []
        for r in range(world):
            seen += shard.shard_indices(11, r, world)
        assert sorted(seen) == list(range(11))
    with pytest.raises(ValueError):
        shard.shard([1, 2], 2, 2)


def test_two_gloo_ranks_match_one_process(tmp_path):
    import json
    out = tmp_path / "res.json"
    mp.spawn(_worker, args=(2, _free_port(), str(out)), nprocs=2, join=True)
    got = [[tuple(w) for w in r] for r in json.load(open(out))]
    _, _, qs = _queries()
    ref = [_run_query(q) for q in qs]
    assert got == ref
    assert any(len(r) > 0 for r in ref)
