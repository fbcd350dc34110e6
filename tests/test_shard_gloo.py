"""The multi-rank host path (sample ranges, max-over-ranks timing) with two
gloo ranks on CPU."""

import os
import socket

import pytest

from paper_2212_04352_gb300 import shard


def test_ranges_partition():
    for world in (1, 2, 3, 8):
        got = [shard.sample_range(r, world, 5) for r in range(world)]
        assert got == [(5 * r, 5) for r in range(world)]
        for total in (0, 1, 7, 100):
            parts = [shard.split_range(r, world, total) for r in range(world)]
            assert sum(c for _, c in parts) == total
            pos = 0
            for first, count in parts:
                assert first == pos
                pos += count
    with pytest.raises(ValueError):
        shard.sample_range(2, 2, 1)


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        first, count = shard.sample_range(rank, world, 4)
        m = shard.max_over_ranks(10.0 + rank, world)
        q.put((rank, first, count, m))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, 0, 4, 11.0), (1, 4, 4, 11.0)]
