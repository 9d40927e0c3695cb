"""Chunked particle sets (Sec. 2.2: chunks computed one after another, each chunk's transfer hidden
behind the next one's computation): the same particles stepped as chunks streamed from pinned host
memory and stepped resident give bit-identical positions and velocities, and sources that agree to
the rounding of the run sums (FP32) or bit for bit up to the summation order (FP64)."""
import numpy as np
import pytest

from paper_2603_26691_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Sim():
    import torch

    assert torch.cuda.is_available()
    from paper_2603_26691_gb300.sim import Sim

    return Sim


def _by_id(pos, vel, d, ids):
    o = np.argsort(ids.astype(np.int64))
    return pos[:, o], vel[:, o], d[o]


@pytest.mark.parametrize("prec,chunk", [("mixed_f32", 64_000), ("mixed_bf16", 100_000), ("fp64", 70_000)])
def test_chunks_match_the_resident_run(Sim, prec, chunk):
    N, n, dt = 32, 300_007, 5e-4
    U = inputs.random_fourier(N, seed=8) * 8.0
    pos, vel, d, _ = inputs.particles(61, 0, n, vmax=0.5)
    Uin = U.astype(np.float32) if prec != "fp64" else U
    res = Sim(N, precision=prec)
    res.set_params(reorder_every=5)
    res.set_fluid(Uin)
    res.add_particles(pos, d, vel)
    res.step(12, dt)
    a = _by_id(*res.particles())
    sa = res.sources(host=True)
    res.close()
    ch = Sim(N, precision=prec)
    ch.set_params(reorder_every=5)
    ch.set_fluid(Uin)
    ch.chunks_create(chunk)
    ch.chunks_add(pos, d, vel)
    assert ch.chunks_count() == (n, -(-n // (-(-chunk // 64) * 64)))
    t1 = ch.chunks_step(7, dt)
    t2 = ch.chunks_step(5, dt)
    b = _by_id(*ch.chunks_particles())
    sb = ch.sources(host=True)
    ch.close()
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    tol = 1e-6 if prec != "fp64" else 1e-13
    assert np.linalg.norm(sa - sb) <= tol * np.linalg.norm(sa)
    for t in (t1, t2):
        assert t["wall_ms"] > 0 and t["compute_ms"] > 0 and t["h2d_ms"] > 0 and t["d2h_ms"] > 0


def test_chunk_calls_refuse_misuse(Sim):
    from paper_2603_26691_gb300._lib import StError

    N = 16
    pos, vel, d, _ = inputs.particles(62, 0, 1000)
    sim = Sim(N, precision="mixed_f32")
    sim.set_fluid(inputs.taylor_green(N).astype(np.float32))
    with pytest.raises(StError):
        sim.chunks_step(1, 1e-3)  # no chunks yet
    sim.add_particles(pos, d, vel)
    with pytest.raises(StError):
        sim.chunks_create(512)  # resident particles held
    sim.clear_particles()
    sim.chunks_create(512)
    sim.chunks_add(pos, d, vel)
    with pytest.raises(StError):
        sim.add_particles(pos, d, vel)  # resident adds refused while chunks are held
    with pytest.raises(StError):
        sim.reserve(10_000)  # the buffers are the chunks' device slots
    with pytest.raises(StError):
        sim.set_microphysics(True)  # chunks carry no particle temperatures
    sim.chunks_step(2, 1e-3)
    assert sim.n == 0 and sim.chunks_count() == (1000, 2)
    sim.close()


def test_chunk_reads_check_their_range(Sim):
    from paper_2603_26691_gb300._lib import StError

    N = 16
    pos, vel, d, _ = inputs.particles(63, 0, 1500)
    sim = Sim(N, precision="mixed_f32")
    sim.set_fluid(inputs.taylor_green(N).astype(np.float32))
    sim.chunks_create(640)
    sim.chunks_add(pos, d, vel)
    assert sim.chunks_count() == (1500, 3)
    p, v, dd, ids = sim.chunks_particles(1400, 100)  # across the last chunk's end
    assert np.array_equal(ids, np.arange(1400, 1500, dtype=np.uint32))
    with pytest.raises(StError):
        sim.chunks_particles(1400, 101)
    with pytest.raises(StError):
        sim.chunks_create(640)  # once per handle
    sim.close()
