"""Mixed-precision CUDA path (int32 cell + FP32 offset, FP32 or BF16 velocity) against the FP64
oracle, within stated error bounds.  The oracle reads the same FP32-rounded fluid field, so the
bounds measure the step's own arithmetic and storage, not the field's storage."""
import numpy as np
import pytest

import oracle
from paper_2603_26691_gb300 import inputs
from tests.helpers import face_distance, linear_cells, min_image

pytestmark = pytest.mark.gpu

# Stated bounds.  FP32 storage: position in cell widths h, velocity relative to |v| + 1 m/s,
# sources relative to the oracle's L2 / max norm.
BOUNDS = {"mixed_f32": dict(pos_h=1e-5, vel=1e-5, src_l2=1e-5, src_max=1e-4)}
# BF16 velocity storage rounds the velocity to 8 significant bits (unit roundoff 2^-8) every step
# and the integrator carries each rounding forward with a factor e^{-a dt} <= 1, so after S steps
# the velocity error is at most S 2^-8 (|v| + 1) and the position error at most S 2^-8 times the
# path S dt max(|v|, 1) (0.078 and 0.156 for the two cases below).  The rounding errors of
# successive steps have random signs, so the errors found are far below that worst case; the
# bounds are stated at about twice the values measured on GB300 (velocity relative to |v| + 1,
# position relative to the path, sources relative L2):
#   64^3, 200003 particles, 20 steps: 8.1e-3, 3.0e-3, 5.4e-3
#   32^3, 5001 particles, 40 steps:   1.37e-2, 4.2e-3, 8.0e-3
BF16_BOUNDS = {
    (64, 200_003, 20): dict(vel=1.6e-2, pos_path=6e-3, src_l2=1.1e-2),
    (32, 5_001, 40): dict(vel=2.7e-2, pos_path=8.5e-3, src_l2=1.6e-2),
}


@pytest.fixture(scope="module")
def Sim():
    import torch

    assert torch.cuda.is_available()
    from paper_2603_26691_gb300.sim import Sim

    return Sim


def _f32(U):
    return U.astype(np.float32).astype(np.float64)


def _errors(g, opos, ovel, osrc, N):
    order = g["ids"].astype(np.int64)
    h = 1.0 / N
    pos_err = np.abs(min_image(g["pos"], opos[:, order])).max() / h
    vel_err = (np.abs(g["vel"] - ovel[:, order]) / (np.abs(ovel[:, order]) + 1.0)).max()
    src_l2 = np.linalg.norm(g["src"] - osrc) / np.linalg.norm(osrc)
    src_max = np.abs(g["src"] - osrc).max() / np.abs(osrc).max()
    return dict(pos_h=pos_err, vel=vel_err, src_l2=src_l2, src_max=src_max)


def _path(ovel_max, steps, dt):
    return steps * dt * max(ovel_max, 1.0)


def _run(Sim, prec, N, U, pos, vel, d, steps, dt, reorder_every=10, chunk_edge=8):
    sim = Sim(N, precision=prec, chunk_edge=chunk_edge)
    sim.set_params(reorder_every=reorder_every)
    sim.set_fluid(U.astype(np.float32))
    sim.add_particles(pos, d, vel)
    sim.step(steps, dt)
    g = dict(src=sim.sources(host=True), inv=sim.invariants())
    g["pos"], g["vel"], g["d"], g["ids"] = sim.particles()
    g["cells"] = sim.cells()
    sim.close()
    return g


@pytest.mark.parametrize("prec", ["mixed_f32", "mixed_bf16"])
@pytest.mark.parametrize("N,n,steps", [(64, 200_003, 20), (32, 5_001, 40)])
def test_mixed_within_bounds_fourier(Sim, prec, N, n, steps):
    dt = 5e-4
    U = _f32(inputs.random_fourier(N, seed=11))
    pos, vel, d, _ = inputs.particles(2024, 0, n)
    g = _run(Sim, prec, N, U, pos, vel, d, steps, dt)
    opos, ovel, osrc, _ = oracle.run(oracle.make_grid(N), U, pos, vel, d, steps, dt)
    err = _errors(g, opos, ovel, osrc, N)
    err["pos_path"] = err["pos_h"] / N / _path(np.abs(ovel).max(), steps, dt)
    print(prec, N, n, {k: float(v) for k, v in err.items()})
    b = BOUNDS[prec] if prec == "mixed_f32" else BF16_BOUNDS[(N, n, steps)]
    for k, lim in b.items():
        assert err[k] <= lim, (prec, k, err[k], lim)
    # cells agree bit-exactly away from faces (band = the position bound, in cell widths)
    order = g["ids"].astype(np.int64)
    band = b["pos_h"] if "pos_h" in b else b["pos_path"] * _path(np.abs(ovel).max(), steps, dt) * N
    far = face_distance(opos[:, order], (N, N, N)) > band
    assert np.array_equal(g["cells"][far], linear_cells(opos[:, order], (N, N, N))[far])
    assert g["inv"][0] == n


@pytest.mark.parametrize("prec", ["mixed_f32", "mixed_bf16"])
def test_mixed_momentum_balance(Sim, prec):
    N, n, steps, dt = 32, 100_000, 30, 5e-4
    U = _f32(inputs.taylor_green(N))
    pos, vel, d, _ = inputs.particles(4, 0, n, vmax=0.3)
    sim = Sim(N, precision=prec)
    sim.set_fluid(U.astype(np.float32))
    sim.add_particles(pos, d, vel)
    inv0 = sim.invariants()
    sim.step(steps, dt)
    inv1 = sim.invariants()
    sim.close()
    gv = np.array([0.0, 0.0, -9.81])
    bal = inv1[1:4] - inv0[1:4] - inv1[7] * gv * steps * dt + inv1[4:7]
    scale = np.abs(inv1[4:7]).max() + np.abs(inv1[7] * gv * steps * dt).max()
    assert np.abs(bal).max() <= 1e-5 * scale


def test_mixed_uniform_flow_closed_form(Sim):
    N, n, steps, dt = 32, 20_000, 50, 5e-4
    u = np.array([0.3, -0.2, 0.1])
    U = inputs.uniform_field(N, u)
    pos, vel, d, _ = inputs.particles(99, 0, n, vmax=1.0)
    g = _run(Sim, "mixed_f32", N, U, pos, vel, d, steps, dt)
    order = g["ids"].astype(np.int64)
    gv = np.array([0.0, 0.0, -9.81])
    # the particle's stored diameter is FP32: the closed form uses the same value
    dd = d[order].astype(np.float32).astype(np.float64)
    a = 18 * 1.8e-5 / (1000.0 * dd ** 2)
    T = steps * dt
    vinf = u[:, None] + gv[:, None] / a
    v0 = vel[:, order].astype(np.float32).astype(np.float64)
    vT = vinf + (v0 - vinf) * np.exp(-a * T)
    xT = pos[:, order] + vinf * T + (v0 - vinf) * (-np.expm1(-a * T)) / a
    assert np.abs(min_image(g["pos"], xT)).max() * N <= 1e-5
    assert (np.abs(g["vel"] - vT) / (np.abs(vT) + 1.0)).max() <= 1e-5


def test_mixed_deterministic(Sim):
    N, n, steps, dt = 32, 60_000, 25, 5e-4
    U = _f32(inputs.random_fourier(N, seed=3))
    pos, vel, d, _ = inputs.particles(8, 0, n)
    a = _run(Sim, "mixed_f32", N, U, pos, vel, d, steps, dt)
    b = _run(Sim, "mixed_f32", N, U, pos, vel, d, steps, dt)
    assert np.array_equal(a["src"], b["src"])
    assert np.array_equal(a["pos"], b["pos"]) and np.array_equal(a["ids"], b["ids"])


@pytest.mark.parametrize("prec", ["mixed_f32", "mixed_bf16"])
def test_mixed_non_power_of_two_box_grid(Sim, prec):
    """A 40 x 48 x 56 grid (multiples of the chunk edge, not powers of two) on a 1.25 x 1.5 x 1.75
    box: the sorted path's periodic offsets and relocation take the general (compare-and-wrap)
    branch, and the cells are not cubes."""
    grid, box = (40, 48, 56), (1.25, 1.5, 1.75)
    n, steps, dt = 150_001, 20, 5e-4
    U = _f32(inputs.taylor_green(grid, L=box) + 0.2)
    pos, vel, d, _ = inputs.particles(77, 0, n, L=box, vmax=0.5)
    sim = Sim(grid, box=box, precision=prec)
    sim.set_params(reorder_every=10)
    sim.set_fluid(U.astype(np.float32))
    sim.add_particles(pos, d, vel)
    sim.step(steps, dt)
    src = sim.sources(host=True)
    gpos, gvel, _, ids = sim.particles()
    cells = sim.cells()
    sim.close()
    order = ids.astype(np.int64)
    G = oracle.make_grid(grid, L=box)
    opos, ovel, osrc, _ = oracle.run(G, U, pos, vel, d, steps, dt)
    h = np.array(box) / np.array(grid)
    dpos = np.abs(min_image(gpos, opos[:, order], L=box)) / h[:, None]
    vmax = np.abs(ovel).max()
    if prec == "mixed_f32":
        assert dpos.max() <= 1e-5
        assert (np.abs(gvel - ovel[:, order]) / (np.abs(ovel[:, order]) + 1.0)).max() <= 1e-5
        assert np.linalg.norm(src - osrc) <= 1e-5 * np.linalg.norm(osrc)
        band = 1e-5
    else:
        path = steps * dt * max(vmax, 1.0)
        bound = steps * 2.0 ** -8
        assert (dpos * h[:, None]).max() <= bound * path
        assert np.abs(gvel - ovel[:, order]).max() <= bound * (vmax + 1.0)
        assert np.linalg.norm(src - osrc) <= 1e-2 * np.linalg.norm(osrc)
        band = (bound * path / h).max()
    far = face_distance(opos[:, order], grid, L=box) > band
    assert np.array_equal(cells[far], linear_cells(opos[:, order], grid, L=box)[far])


@pytest.mark.parametrize("N", [32, 40])
def test_mixed_moves_longer_than_the_box(Sim, N):
    """Particles launched at up to 2.5 box lengths per step: every coordinate carries whole box
    lengths (the masked wrap on a power-of-two grid, the general relocation otherwise); the error
    bound scales with the path in cells (FP32 relative rounding of the displacement)."""
    n, steps, dt = 4_099, 3, 1e-3
    U = _f32(inputs.taylor_green(N))
    pos, vel, d, _ = inputs.particles(5, 0, n, vmax=2500.0)
    g = _run(Sim, "mixed_f32", N, U, pos, vel, d, steps, dt)
    opos, ovel, osrc, _ = oracle.run(oracle.make_grid(N), U, pos, vel, d, steps, dt)
    order = g["ids"].astype(np.int64)
    path_cells = steps * dt * np.abs(vel).max() * N
    assert np.abs(min_image(g["pos"], opos[:, order])).max() * N <= 1e-6 * (1.0 + path_cells)
    assert (np.abs(g["vel"] - ovel[:, order]) / (np.abs(ovel[:, order]) + 1.0)).max() <= 1e-5
    assert np.linalg.norm(g["src"] - osrc) <= 1e-5 * np.linalg.norm(osrc)
    assert g["inv"][0] == n


def test_reads_between_the_pre_sort_step_and_the_sort(Sim):
    # the step just before a due sort leaves the state as records for the sort's gather; reading
    # particles, invariants or chunk boxes, adding particles, or stepping without the sort in
    # between turns them back into arrays first, and the sort from records gives the same result
    N, n, dt = 32, 30_001, 5e-4
    U = _f32(inputs.random_fourier(N, seed=13))
    pos, vel, d, _ = inputs.particles(515, 0, n, vmax=0.5)
    G = oracle.make_grid(N)
    sim = Sim(N, precision="mixed_f32")
    sim.set_params(reorder_every=5)
    sim.set_fluid(U.astype(np.float32))
    sim.add_particles(pos, d, vel)
    sim.step(5, dt)  # sorts before step 0; step 4 leaves records (a sort is due before step 5)
    opos, ovel, osrc, _ = oracle.run(G, U, pos, vel, d, 5, dt)
    inv = sim.invariants()
    p5, v5, d5, ids5 = sim.particles()
    o5 = ids5.astype(np.int64)
    assert np.abs(min_image(p5, opos[:, o5])).max() * N <= 1e-5
    assert (np.abs(v5 - ovel[:, o5]) / (np.abs(ovel[:, o5]) + 1.0)).max() <= 1e-5
    m = np.array([oracle.mass(G, x) for x in d5])
    assert abs(inv[7] - m.sum()) <= 1e-6 * m.sum()
    # more particles while records may be pending, then 5 steps (the sort gathers from records)
    pos2, vel2, d2, _ = inputs.particles(516, n, 999, vmax=0.5)
    sim.step(4, dt)
    sim.add_particles(pos2, d2, vel2)
    sim.step(6, dt)
    g = dict(src=sim.sources(host=True))
    g["pos"], g["vel"], g["d"], g["ids"] = sim.particles()
    sim.close()
    # oracle: the first n particles 15 steps, the added ones 6
    P1, V1, S1, _ = oracle.run(G, U, pos, vel, d, 9, dt)
    allp = np.concatenate([P1, pos2], axis=1)
    allv = np.concatenate([V1, vel2], axis=1)
    alld = np.concatenate([d, d2])
    P2, V2, S2, _ = oracle.run(G, U, allp, allv, alld, 6, dt, src=S1)
    order = g["ids"].astype(np.int64)
    assert np.abs(min_image(g["pos"], P2[:, order])).max() * N <= 1e-5
    assert (np.abs(g["vel"] - V2[:, order]) / (np.abs(V2[:, order]) + 1.0)).max() <= 1e-5
    assert np.linalg.norm(g["src"] - S2) <= 1e-5 * np.linalg.norm(S2)


@pytest.mark.parametrize("prec", ["mixed_f32", "mixed_bf16"])
def test_sort_from_records_equals_sort_from_arrays(Sim, prec):
    # the step before a due sort leaves 32-byte records that the sort gathers from; reading the
    # invariants in between turns them back into arrays first, so the sort gathers from the arrays
    # instead: both paths must give bit-identical states and sources
    N, n, dt = 32, 40_003, 5e-4
    U = _f32(inputs.random_fourier(N, seed=17)).astype(np.float32)
    pos, vel, d, _ = inputs.particles(77, 0, n, vmax=0.5)
    out = []
    for read_between in (False, True):
        sim = Sim(N, precision=prec)
        sim.set_params(reorder_every=5)
        sim.set_fluid(U)
        sim.add_particles(pos, d, vel)
        for _ in range(3):
            sim.step(5, dt)
            if read_between:
                sim.invariants()
        sim.step(2, dt)
        g = dict(src=sim.sources(host=True), cells=sim.cells())
        g["pos"], g["vel"], g["d"], g["ids"] = sim.particles()
        sim.close()
        out.append(g)
    for k in ("src", "cells", "pos", "vel", "d", "ids"):
        assert np.array_equal(out[0][k], out[1][k]), k
