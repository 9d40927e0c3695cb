"""Physics variants on the GPU (nearest-grid-point gather, semi-implicit Euler, Schiller-Naumann
drag, cloud-in-cell deposit; every combination) against the FP64 oracle through the C ABI.

Particles whose oracle trajectory passes within a small band of a cell face at a step start can
legitimately take the other cell (the nearest-grid-point gather and the containing-cell deposit
jump there); they are left out of the per-particle comparison, and the cells within one cell of
any of their deposits out of the source comparison.  Every other particle and cell is compared
element by element."""
import itertools

import numpy as np
import pytest

import oracle
from paper_2603_26691_gb300 import inputs
from tests.helpers import face_distance, min_image

pytestmark = pytest.mark.gpu

COMBOS = list(itertools.product(["trilinear", "ngp"], ["exponential", "semi_implicit"],
                                ["stokes", "schiller_naumann"], ["cell", "cic"]))
DEFAULT = ("trilinear", "exponential", "stokes", "cell")


@pytest.fixture(scope="module")
def Sim():
    import torch

    assert torch.cuda.is_available()
    from paper_2603_26691_gb300.sim import Sim

    return Sim


def _phys(c):
    return dict(gather=c[0], integrator=c[1], drag=c[2], deposit=c[3])


def _oracle(N, U, pos, vel, d, steps, dt, combo, band):
    """Oracle one step at a time; returns pos, vel, src and the cells to leave out."""
    G = oracle.make_grid(N, **_phys(combo), rho_f=1.2)
    p, v = pos.copy(), vel.copy()
    src = np.zeros((3, N ** 3))
    near = np.zeros(p.shape[1], dtype=bool)
    first = np.full(p.shape[1], steps)  # the first step that starts within the band of a face
    trace = []
    for s in range(steps):
        now = face_distance(p, (N, N, N)) < band
        first[now & ~near] = s
        near |= now
        p, v, src, tr = oracle.run(G, U, p, v, d, 1, dt, src=src, trace=True)
        trace.append(tr[0])
    trace = np.array(trace)
    after = np.arange(steps)[:, None] >= first[None, :]  # deposits from that step on
    bad = np.zeros((N, N, N), dtype=bool)
    for c in np.unique(trace[after]):
        i, j, k = c % N, (c // N) % N, c // (N * N)
        for a, b, e in itertools.product((-1, 0, 1), repeat=3):
            bad[(k + e) % N, (j + b) % N, (i + a) % N] = True
    return p, v, src, near, bad.reshape(-1)


def _gpu(Sim, prec, N, U, pos, vel, d, steps, dt, combo, reorder_every):
    sim = Sim(N, precision=prec, chunk_edge=8)
    sim.set_params(reorder_every=reorder_every)
    sim.set_physics(**_phys(combo), rho_f=1.2)
    sim.set_fluid(U if prec == "fp64" else U.astype(np.float32))
    sim.add_particles(pos, d, vel)
    sim.step(steps, dt)
    g = dict(src=sim.sources(host=True), inv=sim.invariants())
    g["pos"], g["vel"], g["d"], g["ids"] = sim.particles()
    sim.close()
    return g


def _check(g, o, N, pos_tol, vel_tol, src_l2, src_max):
    opos, ovel, osrc, near, bad = o
    order = g["ids"].astype(np.int64)
    keep = ~near[order]
    assert keep.mean() > 0.9
    dx = np.abs(min_image(g["pos"], opos[:, order]))[:, keep].max() * N
    dv = (np.abs(g["vel"] - ovel[:, order]) / (np.abs(ovel[:, order]) + 1.0))[:, keep].max()
    cells = ~bad
    assert cells.mean() > 0.5
    es = (g["src"] - osrc)[:, cells]
    ref = osrc[:, cells]
    e_l2 = np.linalg.norm(es) / np.linalg.norm(ref)
    e_max = np.abs(es).max() / np.abs(ref).max()
    if src_l2 is None:  # the caller checks the sources itself
        e_l2, e_max, src_l2, src_max = 0.0, 0.0, 1.0, 1.0
    assert dx <= pos_tol and dv <= vel_tol and e_l2 <= src_l2 and e_max <= src_max, (dx, dv, e_l2, e_max)
    return cells


CASE = dict(N=12, n=4097, steps=9, dt=1e-3)


def _inputs(seed, c=CASE):
    U = (inputs.taylor_green(c["N"]) + inputs.random_fourier(c["N"], rms=0.3, seed=seed)).astype(np.float32)
    U = U.astype(np.float64)  # the FP32-rounded field for both sides
    pos, vel, d, _ = inputs.particles(seed, 0, c["n"], vmax=0.5)
    return U, pos, vel, d


# grids the sorted-particle (TMA) step kernel takes: edges multiples of the 8-cell unit, at least 14
# cells; power-of-two and other edges run different instances
TMA_COMBOS = [c for c in COMBOS if c != DEFAULT]


@pytest.mark.parametrize("N", [32, 24])
@pytest.mark.parametrize("combo", TMA_COMBOS, ids=["-".join(c) for c in TMA_COMBOS])
def test_sorted_step_kernel_variant_within_bounds(Sim, combo, N):
    c = dict(N=N, n=20_011, steps=9, dt=1e-3)
    U, pos, vel, d = _inputs(35, c)
    o = _oracle(N, U, pos, vel, d, c["steps"], c["dt"], combo, band=2e-5)
    g = _gpu(Sim, "mixed_f32", N, U, pos, vel, d, c["steps"], c["dt"], combo, reorder_every=4)
    _check(g, o, N, 1e-5, 1e-5, 1e-5, 1e-4)


@pytest.mark.parametrize("combo", COMBOS, ids=["-".join(c) for c in COMBOS])
def test_fp64_variant_matches_oracle(Sim, combo):
    c = CASE
    U, pos, vel, d = _inputs(31)
    o = _oracle(c["N"], U, pos, vel, d, c["steps"], c["dt"], combo, band=1e-9)
    g = _gpu(Sim, "fp64", c["N"], U, pos, vel, d, c["steps"], c["dt"], combo, reorder_every=4)
    _check(g, o, c["N"], 1e-10 * c["N"], 1e-10, 1e-10, 1e-10)
    if combo != DEFAULT:
        # the variant changes the result far beyond the tolerance, so the match above means something
        od = _oracle(c["N"], U, pos, vel, d, c["steps"], c["dt"], DEFAULT, band=1e-9)
        assert np.abs(od[2] - o[2]).max() > 1e-4 * np.abs(o[2]).max()


@pytest.mark.parametrize("combo", COMBOS, ids=["-".join(c) for c in COMBOS])
def test_mixed_f32_variant_within_bounds(Sim, combo):
    c = CASE
    U, pos, vel, d = _inputs(32)
    o = _oracle(c["N"], U, pos, vel, d, c["steps"], c["dt"], combo, band=1e-4)
    for reorder in (0, 4):  # generation order and sorted order
        g = _gpu(Sim, "mixed_f32", c["N"], U, pos, vel, d, c["steps"], c["dt"], combo, reorder_every=reorder)
        _check(g, o, c["N"], 1e-5, 1e-5, 1e-5, 1e-4)


@pytest.mark.parametrize("combo", [("ngp", "semi_implicit", "schiller_naumann", "cell"),
                                   ("trilinear", "exponential", "stokes", "cic")],
                         ids=["paper", "cic"])
def test_mixed_bf16_variant_one_step_within_bounds(Sim, combo):
    # BF16 velocity storage drifts positions by up to ~1e-4 cells over several steps, so many
    # particles could take the other side of a face; the step is compared from a common state: the
    # GPU runs 7 steps, the oracle takes the GPU's state (stored BF16 velocities, exact in FP64) and
    # both run one more step.  Bounds for one step: velocity 2^-8 (|v| + 1) (its storage rounding),
    # position 1e-5 cells; the impulse m (v' - v - g dt) is taken from the stored v', so each
    # particle's impulse is off by at most m |v'| 2^-8 per component, deposited like the impulse
    c = CASE
    N = c["N"]
    U, pos, vel, d = _inputs(33)
    sim = Sim(N, precision="mixed_bf16")
    sim.set_params(reorder_every=4)
    sim.set_physics(**_phys(combo), rho_f=1.2)
    sim.set_fluid(U.astype(np.float32))
    sim.add_particles(pos, d, vel)
    sim.step(7, c["dt"])
    sim.sources(reset=True, host=True)
    p0, v0, d0, ids0 = sim.particles()
    sim.step(1, c["dt"])
    g = dict(src=sim.sources(host=True))
    g["pos"], g["vel"], g["d"], g["ids"] = sim.particles()
    sim.close()
    assert np.array_equal(ids0, g["ids"])  # no sort between the two reads (sorts before steps 0, 4, 8)
    o = _oracle(N, U, p0, v0, d0, 1, c["dt"], combo, band=1e-4)
    # the oracle ran on the GPU's storage order: ids map GPU rows onto themselves
    g["ids"] = np.arange(p0.shape[1])
    cells = _check(g, o, N, 1e-5, 2.0 ** -8, None, None)
    G = oracle.make_grid(N, **_phys(combo))
    bound = np.zeros((3, N ** 3))
    for p in range(p0.shape[1]):
        bound = oracle.deposit(G, p0[:, p], oracle.mass(G, d0[p]) * np.abs(o[1][:, p]), bound)
    err = np.abs(g["src"] - o[2])[:, cells]
    slack = 1e-6 * np.abs(o[2]).max()  # FP32 arithmetic of the step
    assert np.all(err <= 2.0 ** -8 * bound[:, cells] * 1.001 + slack), (err / (bound[:, cells] + 1e-300)).max()


@pytest.mark.parametrize("combo", [("ngp", "semi_implicit", "schiller_naumann", "cell"),
                                   ("trilinear", "semi_implicit", "schiller_naumann", "cic")],
                         ids=["paper", "cic"])
def test_variant_momentum_budget_exact(Sim, combo):
    # particles' momentum change - gravity impulse + sources = 0 to FP64 rounding, on the GPU's
    # own output (both precisions)
    c = CASE
    U, pos, vel, d = _inputs(34)
    G = oracle.make_grid(c["N"])
    for prec in ("fp64", "mixed_f32"):
        g = _gpu(Sim, prec, c["N"], U, pos, vel, d, 20, c["dt"], combo, reorder_every=4)
        m = np.array([oracle.mass(G, x) for x in g["d"]])
        order = g["ids"].astype(np.int64)
        P0 = (m * vel[:, order]).sum(1)
        gv = np.array([0.0, 0.0, -9.81])
        bal = g["inv"][1:4] - P0 - m.sum() * gv * 20 * c["dt"] + g["inv"][4:7]
        scale = (m * (np.abs(g["vel"]) + np.abs(vel[:, order]))).sum() + m.sum() * 9.81 * 20 * c["dt"]
        assert np.abs(bal).max() <= (1e-12 if prec == "fp64" else 1e-6) * scale


def test_set_physics_rejects_bad_arguments_and_the_adjoint_needs_its_physics(Sim):
    from paper_2603_26691_gb300 import _lib

    sim = Sim(8, precision="fp64")
    lib, h = sim.lib, sim.h
    assert lib.st_set_physics(h, 2, 0, 0, 0, 1.2) == _lib.ST_ERR_INVALID_ARG
    assert lib.st_set_physics(h, 0, 0, 0, -1, 1.2) == _lib.ST_ERR_INVALID_ARG
    assert lib.st_set_physics(h, 0, 0, 1, 0, 0.0) == _lib.ST_ERR_INVALID_ARG
    assert lib.st_set_physics(h, 0, 0, 1, 0, float("nan")) == _lib.ST_ERR_NONFINITE
    pos, vel, d, _ = inputs.particles(1, 0, 64)
    sim.set_fluid(inputs.taylor_green(8))
    sim.add_particles(pos, d, vel)
    sim.set_physics(drag="schiller_naumann")
    assert lib.st_adjoint_forward(h, 4, 1e-3, 2) == _lib.ST_ERR_STATE
    sim.set_physics(deposit="cic")  # the cloud-in-cell deposit is differentiated
    assert lib.st_adjoint_forward(h, 4, 1e-3, 2) == _lib.ST_OK
    sim.set_physics()
    assert lib.st_adjoint_forward(h, 4, 1e-3, 2) == _lib.ST_OK
    sim.close()


@pytest.mark.parametrize("combo", [("trilinear", "exponential", "stokes", "cic"),
                                   ("ngp", "semi_implicit", "schiller_naumann", "cic")], ids=["cic", "paper-cic"])
def test_sorted_kernel_cic_far_from_the_sort_time_unit(Sim, combo):
    # one sort, then 60 steps in a fast flow: many start cells leave their unit's deposit tile,
    # so the cloud-in-cell corners go through the global accumulator as well as the tile
    N, n, steps, dt = 32, 20_011, 60, 1e-3
    c = dict(N=N, n=n)
    U, pos, vel, d = _inputs(36, c)
    U = U * 4.0  # particles follow the flow: several cells in 60 ms
    o = _oracle(N, U, pos, vel, d, steps, dt, combo, band=2e-5)
    g = _gpu(Sim, "mixed_f32", N, U, pos, vel, d, steps, dt, combo, reorder_every=1000)
    _check(g, o, N, 1e-5, 1e-5, 1e-5, 1e-4)
