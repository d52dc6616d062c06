"""Multi-rank host logic on CPU: instance shards and the max-over-ranks time (gloo, world size 2)."""
import os
import socket

import pytest

from paper_1702_02207_gb300 import shard


def test_shard_bounds_partition():
    for n in (0, 1, 7, 65536, 65537):
        for world in (1, 2, 3, 8):
            spans = [shard.shard_bounds(n, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            for (a, b), (c, d) in zip(spans, spans[1:]):
                assert b == c
            sizes = [b - a for a, b in spans]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.shard_bounds(10, 2, 2)
    assert shard.rank_seed(1703, 0) != shard.rank_seed(1703, 1)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    lo, hi = shard.shard_bounds(1001, rank, world)
    t = shard.max_over_ranks(0.5 + rank, dist)
    q.put((rank, lo, hi, t))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got[0][1:3] == (0, 501) and got[1][1:3] == (501, 1001)
    assert got[0][3] == 1.5 and got[1][3] == 1.5
    assert shard.max_over_ranks(2.5) == 2.5
