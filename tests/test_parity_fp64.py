"""Parity of the plain FP64 CUDA path with the FP64 CPU oracle (through the C ABI)."""
import math

import numpy as np
import pytest

import oracle
from paper_2603_26691_gb300 import inputs
from tests.helpers import face_distance, linear_cells, min_image

pytestmark = pytest.mark.gpu

FLOAT_TOL = 1e-10   # relative, FP64 path against the FP64 oracle
FACE_BAND = 1e-9    # cells are compared bit-exactly outside this band (cell units)


@pytest.fixture(scope="module")
def Sim():
    import torch

    assert torch.cuda.is_available()
    from paper_2603_26691_gb300.sim import Sim

    return Sim


def _run_gpu(Sim, N, U, pos, vel, d, steps, dt, reorder_every=10, chunk_edge=8, **params):
    sim = Sim(N, precision="fp64", chunk_edge=chunk_edge)
    sim.set_params(reorder_every=reorder_every, **params)
    sim.set_fluid(U)
    sim.add_particles(pos, d, vel)
    sim.step(steps, dt)
    out = dict(src=sim.sources(host=True), inv=sim.invariants())
    out["pos"], out["vel"], out["d"], out["ids"] = sim.particles()
    out["cells"] = sim.cells()
    sim.close()
    return out


def _compare(g, opos, ovel, osrc, N, L=1.0):
    order = g["ids"].astype(np.int64)
    dx = min_image(g["pos"], opos[:, order], L)
    assert np.abs(dx).max() <= FLOAT_TOL * L
    vscale = np.maximum(np.abs(ovel[:, order]), 1.0)
    assert (np.abs(g["vel"] - ovel[:, order]) / vscale).max() <= FLOAT_TOL
    smax = np.abs(osrc).max()
    if smax > 0:
        assert np.abs(g["src"] - osrc).max() <= FLOAT_TOL * smax
    else:
        assert np.abs(g["src"]).max() == 0.0
    # cells bit-exact away from faces
    ocell = linear_cells(opos[:, order], (N, N, N))
    far = face_distance(opos[:, order], (N, N, N)) > FACE_BAND
    assert np.array_equal(g["cells"][far], ocell[far])


def test_taylor_green_32_1e5_particles_100_steps(Sim):
    """The smallest workload: 32^3 Taylor-Green (U0 = 1), 1e5 particles at rest, 100 steps of 1e-3."""
    N, n, steps, dt = 32, 100_000, 100, 1e-3
    U = inputs.taylor_green(N)
    pos, vel, d, _ = inputs.particles(12345, 0, n)
    g = _run_gpu(Sim, N, U, pos, vel, d, steps, dt)
    G = oracle.make_grid(N)
    opos, ovel, osrc, _ = oracle.run(G, U, pos, vel, d, steps, dt)
    _compare(g, opos, ovel, osrc, N)
    # momentum balance of the GPU's own results
    m = np.array([oracle.mass(G, x) for x in g["d"]])
    P0 = np.zeros(3)
    gvec = np.array([0.0, 0.0, -9.81])
    bal = g["inv"][1:4] - P0 - m.sum() * gvec * steps * dt + g["inv"][4:7]
    scale = (m * (np.abs(g["vel"]).sum(0) + 9.81 * steps * dt)).sum()
    assert np.abs(bal).max() <= 1e-12 * scale
    assert g["inv"][0] == n


@pytest.mark.parametrize("n", [1, 31, 33, 4097, 100_003])
def test_ragged_sizes_fourier_field(Sim, n):
    N, steps, dt = 24, 17, 7e-4
    U = inputs.random_fourier(N, seed=5)
    pos, vel, d, _ = inputs.particles(777, 10, n, vmax=0.8)
    g = _run_gpu(Sim, N, U, pos, vel, d, steps, dt, reorder_every=4, chunk_edge=4)
    opos, ovel, osrc, _ = oracle.run(oracle.make_grid(N, chunk_edge=4), U, pos, vel, d, steps, dt)
    _compare(g, opos, ovel, osrc, N)


def test_uniform_flow_closed_form_subcase(Sim):
    """Uniform u = (0.3, -0.2, 0.1), random initial velocities: every particle follows the closed form."""
    N, n, steps, dt = 32, 20_000, 50, 5e-4
    u = np.array([0.3, -0.2, 0.1])
    U = inputs.uniform_field(N, u)
    pos, vel, d, _ = inputs.particles(99, 0, n, vmax=1.0)
    g = _run_gpu(Sim, N, U, pos, vel, d, steps, dt)
    order = g["ids"].astype(np.int64)
    gv = np.array([0.0, 0.0, -9.81])
    a = 18 * 1.8e-5 / (1000.0 * d[order] ** 2)
    T = steps * dt
    vinf = u[:, None] + gv[:, None] / a
    v0 = vel[:, order]
    vT = vinf + (v0 - vinf) * np.exp(-a * T)
    xT = pos[:, order] + vinf * T + (v0 - vinf) * (-np.expm1(-a * T)) / a
    assert np.abs(min_image(g["pos"], xT)).max() <= 1e-10
    assert (np.abs(g["vel"] - vT) / np.maximum(np.abs(vT), 1.0)).max() <= 1e-10


def test_edge_cases_zero_and_degenerate(Sim):
    N = 8
    sim = Sim(N, precision="fp64")
    sim.set_fluid(np.zeros((N, N, N, 3)))
    sim.step(3, 1e-3)  # no particles: nothing happens
    assert np.all(sim.sources(host=True) == 0.0)
    assert sim.invariants()[0] == 0
    # particles exactly on faces and corners, tiny and large diameters
    pos = np.array([[0.0, 0.125, 0.5, 0.999999999999], [0.0, 0.25, 0.5, 0.0], [0.0, 0.375, 0.875, 0.5]])
    d = np.array([1e-8, 2e-5, 1e-3, 5e-5])
    vel = np.array([[0.0, 1.0, -2.0, 0.5], [0.0, 0.0, 3.0, 0.0], [0.0, -1.0, 0.0, 0.0]])
    sim.add_particles(pos, d, vel)
    sim.step(5, 1e-3)
    g = {"src": sim.sources(host=True), "inv": sim.invariants()}
    g["pos"], g["vel"], g["d"], g["ids"] = sim.particles()
    g["cells"] = sim.cells()
    sim.close()
    opos, ovel, osrc, _ = oracle.run(oracle.make_grid(N), np.zeros((N, N, N, 3)), pos, vel, d, 5, 1e-3)
    _compare(g, opos, ovel, osrc, N)


def test_errors_are_reported(Sim):
    from paper_2603_26691_gb300._lib import ST_ERR_INVALID_ARG, ST_ERR_NONFINITE, StError

    N = 8
    sim = Sim(N, precision="fp64")
    bad = np.zeros((N, N, N, 3))
    bad[1, 2, 3, 1] = np.nan
    with pytest.raises(StError) as e:
        sim.set_fluid(bad)
    assert e.value.status == ST_ERR_NONFINITE
    with pytest.raises(StError) as e:
        sim.step(1, -1.0)
    assert e.value.status == ST_ERR_INVALID_ARG
    with pytest.raises(StError) as e:
        sim.add_particles(np.zeros((3, 2)), np.array([1e-5, 0.0]))
    assert e.value.status == ST_ERR_INVALID_ARG
    with pytest.raises(StError) as e:
        sim.add_particles(np.array([[np.inf], [0.0], [0.0]]), np.array([1e-5]))
    assert e.value.status == ST_ERR_NONFINITE
    with pytest.raises(StError) as e:
        sim.set_params(rho_p=-1.0)
    assert e.value.status == ST_ERR_INVALID_ARG
    sim.close()


def test_deterministic_and_order_independent_particles(Sim):
    """Bit-identical sources on a rerun; per-particle results do not depend on the sort cadence."""
    N, n, steps, dt = 32, 50_000, 30, 1e-3
    U = inputs.random_fourier(N, seed=8)
    pos, vel, d, _ = inputs.particles(5, 0, n)
    a = _run_gpu(Sim, N, U, pos, vel, d, steps, dt, reorder_every=10)
    b = _run_gpu(Sim, N, U, pos, vel, d, steps, dt, reorder_every=10)
    assert np.array_equal(a["src"], b["src"]) and np.array_equal(a["ids"], b["ids"])
    c = _run_gpu(Sim, N, U, pos, vel, d, steps, dt, reorder_every=1)
    oa, oc = np.argsort(a["ids"]), np.argsort(c["ids"])
    assert np.array_equal(a["pos"][:, oa], c["pos"][:, oc])
    assert np.array_equal(a["vel"][:, oa], c["vel"][:, oc])
    assert np.abs(a["src"] - c["src"]).max() <= 1e-13 * np.abs(a["src"]).max()
