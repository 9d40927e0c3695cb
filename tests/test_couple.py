"""Asynchronous two-way coupling on the GPU (the fluid update from lagged sources with the
extrapolator-corrector estimate, between the particle intervals) against the FP64 oracle's orc_couple, and the global
momentum budget (particles + fluid + pending sources - gravity impulse) at small and full size."""
import numpy as np
import pytest

import oracle
from paper_2603_26691_gb300 import inputs
from tests.helpers import min_image

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Sim():
    import torch

    assert torch.cuda.is_available()
    from paper_2603_26691_gb300.sim import Sim

    return Sim


def _run(Sim, prec, N, U, pos, vel, d, nint, K, dt, rho_f, nu, sweeps, extrap, chunk_edge=8, reorder_every=10):
    sim = Sim(N, precision=prec, chunk_edge=chunk_edge)
    sim.set_params(reorder_every=reorder_every)
    sim.set_fluid(U if prec == "fp64" else U.astype(np.float32))
    sim.add_particles(pos, d, vel)
    sim.couple_params(rho_f=rho_f, nu=nu, sweeps=sweeps, steps_per_interval=K, extrapolator=extrap)
    inv0 = sim.invariants()
    sim.couple_run(nint, dt)
    out = dict(U=sim.fluid(), pend=sim.pending_sources(), inv0=inv0, inv1=sim.invariants())
    out["pos"], out["vel"], out["d"], out["ids"] = sim.particles()
    sim.close()
    return out


def _budget(g, N, rho_f, steps, dt, U0):
    """Relative residual of: particle momentum + fluid momentum + pending - gravity impulse."""
    V = (1.0 / N) ** 3
    gv = np.array([0.0, 0.0, -9.81])
    P0 = g["inv0"][1:4] + rho_f * V * U0.reshape(-1, 3).sum(0)
    P1 = g["inv1"][1:4] + rho_f * V * g["U"].reshape(-1, 3).sum(0) + g["pend"].sum(1)
    grav = g["inv1"][7] * gv * steps * dt
    scale = np.abs(P0).max() + np.abs(grav).max() + np.abs(g["pend"]).sum(1).max()
    return np.abs(P1 - P0 - grav).max() / scale


CASE = dict(N=16, n=3001, nint=6, K=3, dt=1e-3, rho_f=1.2e-6, nu=1e-3, sweeps=10)


@pytest.mark.parametrize("extrap", ["zero", "const", "lin"])
def test_fp64_coupled_run_matches_oracle(Sim, extrap):
    c = CASE
    N = c["N"]
    U = inputs.taylor_green(N) * 0.5
    pos, vel, d, _ = inputs.particles(21, 0, c["n"], vmax=0.2)
    g = _run(Sim, "fp64", N, U, pos, vel, d, c["nint"], c["K"], c["dt"], c["rho_f"], c["nu"], c["sweeps"], extrap)
    Uo, po, vo, pend = oracle.couple(oracle.make_grid(N), U, pos, vel, d, c["nint"], c["K"], c["dt"], c["rho_f"],
                                     c["nu"], c["sweeps"], extrap)
    order = g["ids"].astype(np.int64)
    assert np.abs(g["U"] - Uo).max() <= 1e-10 * np.abs(Uo).max()
    assert np.abs(Uo - U).max() > 1e-3  # the exchange moved the fluid
    assert np.abs(min_image(g["pos"], po[:, order])).max() <= 1e-10
    assert (np.abs(g["vel"] - vo[:, order]) / np.maximum(np.abs(vo[:, order]), 1.0)).max() <= 1e-10
    assert np.abs(g["pend"] - pend).max() <= 1e-10 * np.abs(pend).max()
    assert _budget(g, N, c["rho_f"], c["nint"] * c["K"], c["dt"], U) <= 1e-10


@pytest.mark.parametrize("prec", ["mixed_f32", "mixed_bf16"])
def test_mixed_coupled_run_within_bounds(Sim, prec):
    c = CASE
    N = c["N"]
    U = (inputs.taylor_green(N) * 0.5).astype(np.float32).astype(np.float64)
    pos, vel, d, _ = inputs.particles(22, 0, c["n"], vmax=0.2)
    g = _run(Sim, prec, N, U, pos, vel, d, c["nint"], c["K"], c["dt"], c["rho_f"], c["nu"], c["sweeps"], "const")
    Uo, po, vo, pend = oracle.couple(oracle.make_grid(N), U, pos, vel, d, c["nint"], c["K"], c["dt"], c["rho_f"],
                                     c["nu"], c["sweeps"], "const")
    order = g["ids"].astype(np.int64)
    steps = c["nint"] * c["K"]
    if prec == "mixed_f32":
        # FP32 field, state and fluid update: position 1e-5 h, velocity 1e-5 (|v| + 1), field 1e-5 max|u|
        assert np.abs(g["U"] - Uo).max() <= 1e-5 * np.abs(Uo).max()
        assert np.abs(min_image(g["pos"], po[:, order])).max() * N <= 1e-5
        assert (np.abs(g["vel"] - vo[:, order]) / (np.abs(vo[:, order]) + 1.0)).max() <= 1e-5
        assert np.linalg.norm(g["pend"] - pend) <= 1e-5 * np.linalg.norm(pend)
        assert _budget(g, N, c["rho_f"], steps, c["dt"], U) <= 1e-6
    else:
        # BF16 velocity storage: the bounds of the uncoupled BF16 step (steps 2^-8 relative)
        bound = steps * 2.0 ** -8
        vmax = np.abs(vo).max()
        assert np.abs(g["vel"] - vo[:, order]).max() <= bound * (vmax + 1.0)
        assert np.abs(g["U"] - Uo).max() <= bound * np.abs(Uo).max()
        assert _budget(g, N, c["rho_f"], steps, c["dt"], U) <= 1e-6


def test_coupled_fourier256_2e9_momentum_budget(Sim):
    """The coupled workload: 256^3 FP32 Fourier field, 2e9 mixed-precision particles in 32^3-cell
    chunks, fluid update every 5 steps from lagged sources (nu = 1e-3, 10 Jacobi sweeps,
    rho_f = 1.2), 50 steps of 5e-4; the FP64 global momentum budget."""
    import torch

    w = inputs.WORKLOADS["fourier256_coupled_2e9"]
    N = w.grid
    U = w.make_field()
    sim = Sim(N, precision="mixed_f32", chunk_edge=w.chunk_edge)
    sim.set_params(reorder_every=10)
    sim.set_fluid(U.astype(np.float32))
    q = inputs.lognormal_qtable()
    sim.reserve(w.n)
    for first in range(0, w.n, 50_000_000):
        cnt = min(50_000_000, w.n - first)
        p, v, dd, ids = sim.gen_particles(w.seed, first, cnt, q)
        sim.add_particles(p, dd, v, ids)
        del p, v, dd, ids
    K = w.extra["fluid_every"]
    sim.couple_params(rho_f=1.2, nu=w.extra["nu"], sweeps=10, steps_per_interval=K, extrapolator="zero")
    U0 = sim.fluid()
    inv0 = sim.invariants()
    sim.couple_run(w.steps // K, w.dt)
    g = dict(U=sim.fluid(), pend=sim.pending_sources(), inv0=inv0, inv1=sim.invariants())
    sim.close()
    torch.cuda.empty_cache()
    assert g["inv1"][0] == w.n
    assert _budget(g, N, 1.2, w.steps, w.dt, U0) <= 1e-6
