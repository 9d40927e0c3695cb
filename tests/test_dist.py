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


def _words_of(values, E):
    """Normalised fixed-point words (digits below a signed top word) of integers round(v 2^E), by plain
    integer arithmetic."""
    import numpy as np

    w = np.zeros((len(values), 4), dtype=np.int64)
    for i, v in enumerate(values):
        m = int(v)
        w[i] = [m & 0xFFFFFFFF, (m >> 32) & 0xFFFFFFFF, (m >> 64) & 0xFFFFFFFF, m >> 96]
    return w


def _exact_values(rank):
    """Rank r's integers and exponent: huge values that cancel between the ranks plus small ones."""
    import random

    rnd = random.Random(7)
    big = [rnd.randrange(-(1 << 120), 1 << 120) for _ in range(24)]
    rs = random.Random(100 + rank)
    small = [rs.randrange(-(1 << 40), 1 << 40) for _ in range(24)]
    E = (40, 73)[rank]
    # rank 0 holds +big, rank 1 holds -big at a scale 2^33 finer (the same real values)
    vals = [(b if rank == 0 else -(b << 33)) + s for b, s in zip(big, small)]
    return vals, E


def _exact_worker(rank, world, port, out):
    import numpy as np

    from paper_2603_26691_gb300.dist import reduce_sources_exact

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    vals, E = _exact_values(rank)
    w = torch.as_tensor(_words_of(vals, E)).reshape(3, 8, 4)
    tot = reduce_sources_exact(w, E)
    out.put((rank, np.ascontiguousarray(tot.numpy()).tobytes()))
    dist.destroy_process_group()


def test_exact_fixed_point_reduction_with_gloo():
    """Two ranks' fixed-point sources at different exponents whose large parts cancel: the integer sum
    keeps the small remainder exactly (an FP64 sum of the ranks' values would lose it), and both ranks get
    the same bits."""
    from fractions import Fraction

    import numpy as np

    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_exact_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0][1] == res[1][1]
    got = np.frombuffer(res[0][1], dtype=np.float64)
    want = []
    for i in range(24):
        tot = Fraction(0)
        for r in range(world):
            vals, E = _exact_values(r)
            tot += Fraction(vals[i], 2 ** E)
        want.append(float(tot))
    want = np.array(want)
    assert np.all(np.abs(got - want) <= 2 * np.spacing(np.abs(want)))
    # the naive route: each rank's value rounded to FP64, then added, keeps nothing of the remainder
    naive = sum(np.array([float(Fraction(v, 2 ** E)) for v in _exact_values(r)[0]]) for r in range(world)
                for E in [_exact_values(r)[1]])
    assert np.all(np.abs(naive - want) >= 0.5 * np.abs(want))
