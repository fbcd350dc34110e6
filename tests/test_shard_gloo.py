"""The multi-rank host path (sample ranges, max-over-ranks timing, the
all-reduce of the estimators) with two gloo ranks on CPU."""

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


def _combine_worker(rank, world, port, q):
    import numpy as np
    import torch
    import torch.distributed as dist
    import oracle
    import workloads as W
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        lat = W.periodic_honeycomb()
        nu, nd = W.neel_state(lat)
        first, count = shard.split_range(rank, world, 301)          # uneven halves: 151 + 150
        snap, _ = oracle.run(lat, 1.6, nu, nd, 9, first, count, 0.01, 60, 20)
        occ, conn, _ = oracle.moments(snap, want_g2=False)
        M, o, c, g = shard.combine_moments(count, torch.from_numpy(occ), torch.from_numpy(conn), world)
        q.put((rank, M, o.numpy(), c.numpy(), g.numpy()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_combine_moments():
    """Two ranks with uneven sample ranges combine their estimators into the
    oracle's estimators over all 301 samples (Eqs. 5 and 10) to rounding."""
    import multiprocessing as mp
    import numpy as np
    import oracle
    import workloads as W
    ctx = mp.get_context("spawn")
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    q = ctx.Queue()
    procs = [ctx.Process(target=_combine_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=180) for _ in range(2)), key=lambda r: r[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    lat = W.periodic_honeycomb()
    nu, nd = W.neel_state(lat)
    snap, _ = oracle.run(lat, 1.6, nu, nd, 9, 0, 301, 0.01, 60, 20)
    occ, conn, g2 = oracle.moments(snap)
    for rank, M, o, c, g in res:
        assert M == 301
        np.testing.assert_allclose(o, occ, rtol=0, atol=1e-14)
        np.testing.assert_allclose(c, conn, rtol=0, atol=1e-14)
        ok = ~np.isnan(g2)
        assert np.array_equal(np.isnan(g), np.isnan(g2))
        np.testing.assert_allclose(g[ok], g2[ok], rtol=1e-12)
    # both ranks hold the same combined result
    assert np.array_equal(res[0][3], res[1][3])
