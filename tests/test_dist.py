"""Multi-process host logic with the gloo backend on CPU (world size 2)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2603_26691_gb300.dist import max_over_ranks, reduce_sources_rank_order, shard


def test_shard_covers_every_particle_once():
    for n in (0, 1, 7, 1000, 10**9 + 3):
        for world in (1, 2, 3, 8):
            ranges = [shard(n, r, world) for r in range(world)]
            assert ranges[0][0] == 0
            for (f0, c0), (f1, _) in zip(ranges, ranges[1:]):
                assert f0 + c0 == f1
            assert sum(c for _, c in ranges) == n
            assert max(c for _, c in ranges) - min(c for _, c in ranges) <= 1
    with pytest.raises(ValueError):
        shard(10, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    g = torch.Generator().manual_seed(100 + rank)
    src = torch.randn(3, 64, generator=g, dtype=torch.float64) * 10.0 ** (rank * 8)
    tot = reduce_sources_rank_order(src)
    t = max_over_ranks(1.5 + rank)
    out.put((rank, tot.numpy().tobytes(), t))
    dist.destroy_process_group()


def test_rank_order_reduction_and_max_with_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    # every rank holds the same bits, equal to the sum taken in rank order
    want = None
    for r in range(world):
        g = torch.Generator().manual_seed(100 + r)
        s = torch.randn(3, 64, generator=g, dtype=torch.float64) * 10.0 ** (r * 8)
        want = s.clone() if want is None else want + s
    for _, tot, t in res:
        assert tot == want.numpy().tobytes()
        assert t == 1.5 + world - 1
