"""The FP32 adjoint of mixed FP32-velocity handles against the oracle's FP64 adjoint of the same run
(the FP32-rounded field and the handle's own FP32 initial state), and its own consistency: the
recomputed segments reproduce the forward run bit for bit, so every checkpoint interval gives the
same gradients."""
import numpy as np
import pytest

import oracle
from paper_2603_26691_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Sim():
    import torch

    assert torch.cuda.is_available()
    from paper_2603_26691_gb300.sim import Sim

    return Sim


def _case(N=16, n=5000, alpha=0.9):
    U = (inputs.taylor_green(N) + 0.1 * inputs.random_fourier(N, seed=13)).astype(np.float32).astype(np.float64)
    pos, vel, d, _ = inputs.particles(78, 0, n, vmax=0.2)
    return N, U, pos, vel, d * 1.5, alpha


def _smooth_lam(N):
    # a smooth dL/dJtot: a deposit cell decided on the other side of a face by FP32 rounding changes
    # a particle's lam by a fraction h |grad lam| / |lam| only
    c = (np.arange(N) + 0.5) / N
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    return np.stack([np.sin(2 * np.pi * (x + 0.3 * q)) * np.cos(2 * np.pi * y) * (1.5 + np.sin(2 * np.pi * z))
                     for q in range(3)]).reshape(3, -1)


def _gpu(Sim, N, U, pos, vel, d, alpha, nsteps, dt, ck, lam, cells=False):
    sim = Sim(N, precision="mixed_f32")
    sim.set_params(drag_scale=alpha, reorder_every=0)
    sim.set_fluid(U.astype(np.float32))
    sim.add_particles(pos, d, vel)
    p0, v0, d0, _ = sim.particles()  # the FP32 initial state, exactly
    sim.adjoint_forward(nsteps, dt, ck)
    J = sim.sources(host=True)
    gd, ga, gU = sim.adjoint_backward(lam)
    trace = None
    if cells:
        # the run again, one step at a time (the same general kernel, storage order kept), keeping the
        # start cell of every step
        sim.clear_particles()
        sim.add_particles(p0, d0, v0)
        trace = []
        for _ in range(nsteps):
            trace.append(sim.cells())
            sim.step(1, dt)
        trace = np.stack(trace)
    sim.close()
    return (p0, v0, d0), J, gd, ga, gU, trace


def test_fp32_adjoint_against_the_oracle(Sim):
    N, U, pos, vel, d, alpha = _case()
    nsteps, dt, ck = 30, 1e-3, 7
    lam = _smooth_lam(N)
    (p0, v0, d0), J, gd, ga, gU, trace = _gpu(Sim, N, U, pos, vel, d, alpha, nsteps, dt, ck, lam, cells=True)
    G = oracle.make_grid(N, alpha=alpha)
    _, _, oJ, otrace = oracle.run(G, U, p0, v0, d0, nsteps, dt, trace=True)
    ogd, oga, ogU = oracle.adjoint(G, U, p0, v0, d0, nsteps, dt, lam)
    ocells = np.asarray(otrace).reshape(nsteps, -1)
    same = (trace == ocells).all(axis=0)  # particles whose deposit cells agree at every step
    err = dict(J_l2=np.linalg.norm(J - oJ) / np.linalg.norm(oJ),
               gd_max=np.abs(gd - ogd)[same].max() / np.abs(ogd).max(),
               ga=abs(ga - oga) / abs(oga),
               gU_l2=np.linalg.norm(gU - ogU) / np.linalg.norm(ogU),
               gU_max=np.abs(gU - ogU).max() / np.abs(ogU).max(),
               flipped=int((~same).sum()))
    print(err)
    # FP32 arithmetic (unit roundoff 6e-8) through 30 steps forward and back: measured on GB300 with
    # this case 1.9e-7 (J), 6.4e-7 (dL/dd, particles without a flipped deposit cell), 3.5e-7 (dL/dalpha),
    # 1.8e-7 (dL/dU, relative L2); the bounds are about six times those
    assert err["flipped"] <= 0.01 * d.shape[0]
    assert err["J_l2"] <= 1e-6
    assert err["gd_max"] <= 4e-6 and err["ga"] <= 2e-6 and err["gU_l2"] <= 1e-6


def test_fp32_adjoint_is_independent_of_the_checkpoint_interval(Sim):
    N, U, pos, vel, d, alpha = _case(n=3001)
    nsteps, dt = 23, 1e-3
    lam = np.random.default_rng(6).standard_normal((3, N ** 3))
    ref = None
    for ck in (1, 7, 40):
        _, J, gd, ga, gU, _ = _gpu(Sim, N, U, pos, vel, d, alpha, nsteps, dt, ck, lam)
        if ref is None:
            ref = (J, gd, ga, gU)
        else:
            assert np.array_equal(J, ref[0]) and np.array_equal(gd, ref[1])
            assert ga == ref[2] and np.array_equal(gU, ref[3])


def test_fp32_adjoint_refuses_bf16_velocities(Sim):
    from paper_2603_26691_gb300._lib import StError

    N, U, pos, vel, d, alpha = _case(n=100)
    sim = Sim(N, precision="mixed_bf16")
    sim.set_fluid(U.astype(np.float32))
    sim.add_particles(pos, d, vel)
    with pytest.raises(StError):
        sim.adjoint_forward(3, 1e-3, 2)
    sim.close()


def test_fp32_adjoint_on_a_non_cubic_grid(Sim):
    """24 x 16 x 12 cells (non-power-of-two axes, cells of different widths): J, dL/dalpha, dL/dU and
    dL/dd against the oracle's FP64 adjoint of the same run, in relative L2 (a smooth dL/dJtot)."""
    grid, n, alpha = (24, 16, 12), 4000, 0.9
    U = (inputs.taylor_green(grid) * 0.8 + 0.1).astype(np.float32).astype(np.float64)
    pos, vel, d, _ = inputs.particles(79, 0, n, vmax=0.2)
    d = d * 1.5
    cz, cy, cx = [(np.arange(m) + 0.5) / m for m in grid[::-1]]
    z, y, x = np.meshgrid(cz, cy, cx, indexing="ij")
    lam = np.stack([np.cos(2 * np.pi * (x + 0.2 * q)) * (1.2 + np.sin(2 * np.pi * y)) * np.cos(2 * np.pi * z)
                    for q in range(3)]).reshape(3, -1)
    nsteps, dt, ck = 25, 1e-3, 6
    sim = Sim(grid, precision="mixed_f32")
    sim.set_params(drag_scale=alpha, reorder_every=0)
    sim.set_fluid(U.astype(np.float32))
    sim.add_particles(pos, d, vel)
    p0, v0, d0, _ = sim.particles()
    sim.adjoint_forward(nsteps, dt, ck)
    J = sim.sources(host=True)
    gd, ga, gU = sim.adjoint_backward(lam)
    sim.close()
    G = oracle.make_grid(grid, alpha=alpha)
    _, _, oJ, _ = oracle.run(G, U, p0, v0, d0, nsteps, dt)
    ogd, oga, ogU = oracle.adjoint(G, U, p0, v0, d0, nsteps, dt, lam)
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)  # noqa: E731
    err = dict(J=rel(J, oJ), gd=rel(gd, ogd), ga=abs(ga - oga) / abs(oga), gU=rel(gU, ogU))
    print(err)
    # FP32 rounding through 25 steps forward and back (the cubic case above measures ~2e-7 to 6e-7)
    assert err["J"] <= 2e-6 and err["gd"] <= 1e-5 and err["ga"] <= 1e-5 and err["gU"] <= 1e-5


def test_fp32_adjoint_sorted_dense_stencils_grouped(Sim):
    """Sorted by cell at about 40 particles per cell, most warps hold several particles with the same
    trilinear stencil, and their dL/dU products are summed in FP32 before one exact commit per stencil:
    J, dL/dalpha, dL/dU and dL/dd against the oracle's FP64 adjoint, and bit-identical gradients from a
    second run (the grouping depends only on the stencils)."""
    N, n, alpha = 8, 20_000, 0.9
    U = (inputs.taylor_green(N) + 0.1 * inputs.random_fourier(N, seed=21)).astype(np.float32).astype(np.float64)
    pos, vel, d, _ = inputs.particles(80, 0, n, vmax=0.2)
    d = d * 1.5
    lam = _smooth_lam(N)
    nsteps, dt, ck = 20, 1e-3, 5
    runs = []
    for _ in range(2):
        sim = Sim(N, precision="mixed_f32")
        sim.set_params(drag_scale=alpha, reorder_every=0)
        sim.set_fluid(U.astype(np.float32))
        sim.add_particles(pos, d, vel)
        sim.reorder()
        p0, v0, d0, _ = sim.particles()
        sim.adjoint_forward(nsteps, dt, ck)
        J = sim.sources(host=True)
        gd, ga, gU = sim.adjoint_backward(lam)
        sim.close()
        runs.append((p0, v0, d0, J, gd, ga, gU))
    for a, b in zip(runs[0][3:], runs[1][3:]):
        assert np.array_equal(np.asarray(a), np.asarray(b))
    p0, v0, d0, J, gd, ga, gU = runs[0]
    G = oracle.make_grid(N, alpha=alpha)
    _, _, oJ, _ = oracle.run(G, U, p0, v0, d0, nsteps, dt)
    ogd, oga, ogU = oracle.adjoint(G, U, p0, v0, d0, nsteps, dt, lam)
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)  # noqa: E731
    err = dict(J=rel(J, oJ), gd=rel(gd, ogd), ga=abs(ga - oga) / abs(oga), gU=rel(gU, ogU))
    print(err)
    # FP32 rounding through 20 steps forward and back, and FP32 sums over up to 32 products per stencil
    assert err["J"] <= 2e-6 and err["gd"] <= 1e-5 and err["ga"] <= 1e-5 and err["gU"] <= 1e-5
