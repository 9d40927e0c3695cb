"""The library's kernel timers (st_timers_*): CUDA events around its own launches, per kind."""
import numpy as np
import pytest

from paper_2603_26691_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_timers_count_and_time_the_launches():
    import torch

    assert torch.cuda.is_available()
    from paper_2603_26691_gb300.sim import Sim

    N = 16
    sim = Sim(N, precision="fp64")
    sim.set_params(reorder_every=3)
    sim.set_fluid(inputs.taylor_green(N))
    pos, vel, d, _ = inputs.particles(3, 0, 5000)
    sim.add_particles(pos, d, vel)
    sim.step(2, 1e-3)  # not timed
    sim.timers(True)
    sim.step(7, 1e-3)  # sorts before steps 3 and 6 of the handle's count (steps_since_sort 3)
    t = sim.timers()
    assert t["step"][1] == 7 and t["step"][0] > 0.0
    assert t["sort"][1] == 2 and t["sort"][0] > 0.0
    assert t["adjoint"] == (0.0, 0) and t["fluid"] == (0.0, 0)
    sim.adjoint_forward(6, 1e-3, 4)
    sim.adjoint_backward(np.ones((3, N ** 3)))
    t = sim.timers(reset=True)
    assert t["adjoint"][1] == 6
    assert t["step"][1] == 7 + 6 + 4  # the forward's six steps, then 3 + 1 recomputed in two segments
    assert sim.timers()["step"] == (0.0, 0)
    sim.timers(False)
    sim.step(1, 1e-3)
    assert sim.timers()["step"] == (0.0, 0)
    sim.close()


def test_source_density_is_impulse_over_volume_and_time():
    import torch

    from paper_2603_26691_gb300.sim import Sim

    N, steps, dt = (8, 6, 4), 5, 1e-3
    sim = Sim(N, box=(1.0, 0.5, 2.0), precision="fp64")
    sim.set_fluid(np.zeros((4, 6, 8, 3)))
    pos, vel, d, _ = inputs.particles(9, 0, 2000, L=(1.0, 0.5, 2.0), vmax=1.0)
    sim.add_particles(pos, d, vel)
    sim.step(steps, dt)
    J = sim.sources(host=True)
    S = sim.source_density(steps * dt, host=True)
    V = (1.0 / 8) * (0.5 / 6) * (2.0 / 4)
    assert np.array_equal(S, J / (V * steps * dt))
    sim.close()


def test_timers_count_the_coupled_fluid_updates():
    from paper_2603_26691_gb300.sim import Sim

    N = 16
    sim = Sim(N, precision="mixed_f32")
    sim.set_params(reorder_every=4)
    sim.set_fluid(inputs.taylor_green(N).astype(np.float32))
    pos, vel, d, _ = inputs.particles(4, 0, 20_000)
    sim.add_particles(pos, d, vel)
    sim.couple_params(steps_per_interval=3)
    sim.timers(True)
    sim.couple_run(5, 1e-3)
    t = sim.timers()
    assert t["fluid"][1] == 5 and t["fluid"][0] > 0.0
    assert t["step"][1] == 15
    assert t["sort"][1] == 4  # before steps 0, 4, 8, 12 of the handle's count
    sim.close()


def test_fma_probe_rates_are_plausible():
    from paper_2603_26691_gb300.sim import Sim

    sim = Sim(8, precision="fp64")
    f64, f32 = sim.probe_fma()
    sim.close()
    # GB300: dense FP64 about 1.25 TFLOP/s, FP32 FMA tens of TFLOP/s; the ratio is what matters here
    assert 100.0 < f64 < 1e5 and f32 > 10.0 * f64, (f64, f32)
