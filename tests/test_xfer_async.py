"""Asynchronous field uploads and source downloads (st_set_fluid_async, st_get_sources_async): a loop
of field in, step, sources out gives the same bits through the asynchronous calls as through the
synchronous ones, and a field holding NaN is refused at the next call with the previous field kept."""
import numpy as np
import pytest

from paper_2603_26691_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_mod():
    import torch

    assert torch.cuda.is_available()
    return torch


def _sim(prec, N, U0, seed=91, n=50_003):
    from paper_2603_26691_gb300.sim import Sim

    pos, vel, d, _ = inputs.particles(seed, 0, n, vmax=0.3)
    sim = Sim(N, precision=prec)
    sim.set_params(reorder_every=3)
    sim.set_fluid(U0)
    sim.add_particles(pos, d, vel)
    return sim


@pytest.mark.parametrize("prec,field", [("mixed_f32", "f32"), ("fp64", "f64"), ("mixed_bf16", "f64")])
def test_async_loop_equals_sync_loop(torch_mod, prec, field):
    torch = torch_mod
    N, steps, dt = 32, 7, 5e-4
    base = inputs.random_fourier(N, seed=21) * 8.0
    dtype = np.float32 if field == "f32" else np.float64
    fields = [(base * (1.0 + 0.1 * s)).astype(dtype) for s in range(steps)]
    sync = _sim(prec, N, fields[0])
    want = []
    for s in range(steps):
        sync.set_fluid(fields[s])
        sync.step(1, dt)
        want.append(sync.sources(reset=True, host=True))
    wp = sync.particles()
    sync.close()
    asy = _sim(prec, N, fields[0])
    hf = [torch.from_numpy(f).pin_memory() for f in fields]
    outs = [torch.empty((3, N ** 3), dtype=torch.float64).pin_memory() for _ in range(steps)]
    for s in range(steps):
        asy.set_fluid_async(hf[s])
        asy.step(1, dt)
        asy.sources_async(outs[s], reset=True)
    asy.synchronize()
    got = [o.numpy() for o in outs]
    gp = asy.particles()
    asy.close()
    for a, b in zip(want, got):
        assert np.array_equal(a, b)
    for a, b in zip(wp, gp):
        assert np.array_equal(a, b)


def test_nonfinite_field_is_refused_and_the_previous_one_kept(torch_mod):
    from paper_2603_26691_gb300._lib import StError

    torch = torch_mod
    N, dt = 16, 5e-4
    U = (inputs.random_fourier(N, seed=22) * 8.0).astype(np.float32)
    ref = _sim("mixed_f32", N, U, n=20_001)
    ref.step(3, dt)
    want = ref.sources(host=True)
    ref.close()
    sim = _sim("mixed_f32", N, U, n=20_001)
    sim.step(1, dt)
    bad = U.copy()
    bad[3, 4, 5, 1] = np.nan
    sim.set_fluid_async(torch.from_numpy(bad).pin_memory())
    with pytest.raises(StError):
        sim.step(1, dt)  # reads the upload's scan: refused, nothing stepped
    sim.step(2, dt)
    got = sim.sources(host=True)
    sim.close()
    assert np.array_equal(want, got)


def test_async_reads_without_reset_and_a_synchronous_field_after_an_async_one(torch_mod):
    """Sources read asynchronously without a reset hold the running sum (as the synchronous read does),
    and a synchronous st_set_fluid issued after an asynchronous one is the field the next step uses."""
    torch = torch_mod
    N, dt = 16, 5e-4
    U1 = (inputs.random_fourier(N, seed=23) * 8.0).astype(np.float32)
    U2 = (U1 * 1.5).astype(np.float32)
    ref = _sim("mixed_f32", N, U1, n=30_001)
    ref.step(2, dt)
    r1 = ref.sources(host=True)
    ref.set_fluid(U2)
    ref.step(2, dt)
    r2 = ref.sources(host=True)
    ref.close()
    sim = _sim("mixed_f32", N, U1, n=30_001)
    o1 = torch.empty((3, N ** 3), dtype=torch.float64).pin_memory()
    o2 = torch.empty((3, N ** 3), dtype=torch.float64).pin_memory()
    sim.step(2, dt)
    sim.sources_async(o1)
    sim.set_fluid_async(torch.from_numpy(U1 * 3.0).pin_memory())
    sim.set_fluid(U2)  # waits for the upload above and replaces it
    sim.step(2, dt)
    sim.sources_async(o2)
    sim.synchronize()
    sim.close()
    assert np.array_equal(o1.numpy(), r1)
    assert np.array_equal(o2.numpy(), r2)
