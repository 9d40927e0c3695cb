"""The CUDA adjoint (FP64) against the oracle's adjoint and the oracle's central finite differences."""
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


def _case(N=12, n=257, alpha=0.9):
    U = inputs.taylor_green(N) + 0.1 * inputs.random_fourier(N, seed=13)
    pos, vel, d, _ = inputs.particles(77, 0, n, vmax=0.2)
    return N, U, pos, vel, d * 1.5, alpha


def _gpu_grads(Sim, N, U, pos, vel, d, alpha, nsteps, dt, ck, lam, deposit="cell"):
    sim = Sim(N, precision="fp64")
    sim.set_params(drag_scale=alpha, reorder_every=0)
    sim.set_physics(deposit=deposit)
    sim.set_fluid(U)
    sim.add_particles(pos, d, vel)
    sim.adjoint_forward(nsteps, dt, ck)
    J = sim.sources(host=True)
    gd, ga, gU = sim.adjoint_backward(lam)
    sim.close()
    return J, gd, ga, gU


@pytest.mark.parametrize("ck", [1, 7, 40])
def test_adjoint_matches_oracle_adjoint(Sim, ck):
    N, U, pos, vel, d, alpha = _case()
    nsteps, dt = 23, 1e-3
    lam = np.random.default_rng(5).standard_normal((3, N ** 3))
    J, gd, ga, gU = _gpu_grads(Sim, N, U, pos, vel, d, alpha, nsteps, dt, ck, lam)
    G = oracle.make_grid(N, alpha=alpha)
    _, _, oJ, _ = oracle.run(G, U, pos, vel, d, nsteps, dt)
    ogd, oga, ogU = oracle.adjoint(G, U, pos, vel, d, nsteps, dt, lam)
    assert np.abs(J - oJ).max() <= 1e-10 * np.abs(oJ).max()
    assert np.abs(gd - ogd).max() <= 1e-9 * np.abs(ogd).max()
    assert abs(ga - oga) <= 1e-9 * abs(oga)
    assert np.abs(gU - ogU).max() <= 1e-9 * np.abs(ogU).max()


def test_adjoint_matches_central_finite_differences(Sim):
    """Gradient of L = 1/2 |Jtot - Jtarget|^2 (target from diameters x 1.05) against FD (eps 1e-4)."""
    N, U, pos, vel, d, alpha = _case(N=10, n=40)
    nsteps, dt = 20, 1e-3
    G = oracle.make_grid(N, alpha=alpha)
    _, _, J0, trace = oracle.run(G, U, pos, vel, d, nsteps, dt, trace=True)
    _, _, Jt, _ = oracle.run(G, U, pos, vel, d * 1.05, nsteps, dt)
    lam = J0 - Jt
    _, gd, ga, gU = _gpu_grads(Sim, N, U, pos, vel, d, alpha, nsteps, dt, 6, lam)

    def loss(Gx, Ux, dx):
        _, _, J, _ = oracle.run(Gx, Ux, pos, vel, dx, nsteps, dt, frozen=trace)
        return 0.5 * float(((J - Jt) ** 2).sum())

    eps = 1e-4
    for p in range(0, d.shape[0], 4):
        dp, dm = d.copy(), d.copy()
        dp[p] *= 1 + eps
        dm[p] *= 1 - eps
        fd = (loss(G, U, dp) - loss(G, U, dm)) / (2 * eps * d[p])
        assert abs(fd - gd[p]) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(gd).max())
    fd = (loss(oracle.make_grid(N, alpha=alpha + eps), U, d) - loss(oracle.make_grid(N, alpha=alpha - eps), U, d)) / (2 * eps)
    assert abs(fd - ga) <= 1e-5 * abs(fd)
    for f in np.argsort(-np.abs(gU).ravel())[:8]:
        Up, Um = U.copy().reshape(-1), U.copy().reshape(-1)
        Up[f] += eps
        Um[f] -= eps
        fd = (loss(G, Up.reshape(U.shape), d) - loss(G, Um.reshape(U.shape), d)) / (2 * eps)
        assert abs(fd - gU.ravel()[f]) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(gU).max())


@pytest.mark.parametrize("ck", [1, 7])
def test_adjoint_cic_matches_oracle_adjoint(Sim, ck):
    """The cloud-in-cell deposit's adjoint (deposit weights differentiated) against the oracle's."""
    N, U, pos, vel, d, alpha = _case()
    nsteps, dt = 23, 1e-3
    lam = np.random.default_rng(15).standard_normal((3, N ** 3))
    J, gd, ga, gU = _gpu_grads(Sim, N, U, pos, vel, d, alpha, nsteps, dt, ck, lam, deposit="cic")
    G = oracle.make_grid(N, alpha=alpha, deposit="cic")
    _, _, oJ, _ = oracle.run(G, U, pos, vel, d, nsteps, dt)
    ogd, oga, ogU = oracle.adjoint(G, U, pos, vel, d, nsteps, dt, lam)
    assert np.abs(J - oJ).max() <= 1e-10 * np.abs(oJ).max()
    assert np.abs(gd - ogd).max() <= 1e-9 * np.abs(ogd).max()
    assert abs(ga - oga) <= 1e-9 * abs(oga)
    assert np.abs(gU - ogU).max() <= 1e-9 * np.abs(ogU).max()
    # not the cell deposit's gradient under another name
    cgd = oracle.adjoint(oracle.make_grid(N, alpha=alpha), U, pos, vel, d, nsteps, dt, lam)[0]
    assert np.abs(gd - cgd).max() > 1e-3 * np.abs(cgd).max()


def test_adjoint_cic_matches_central_finite_differences_unfrozen(Sim):
    """With the cloud-in-cell deposit nothing is held fixed: the GPU gradient of
    L = 1/2 |Jtot - Jtarget|^2 against central differences of the oracle's full run (eps 1e-4)."""
    N, U, pos, vel, d, alpha = _case(N=10, n=40)
    nsteps, dt = 20, 1e-3
    G = oracle.make_grid(N, alpha=alpha, deposit="cic")
    _, _, J0, _ = oracle.run(G, U, pos, vel, d, nsteps, dt)
    _, _, Jt, _ = oracle.run(G, U, pos, vel, d * 1.05, nsteps, dt)
    lam = J0 - Jt
    _, gd, ga, gU = _gpu_grads(Sim, N, U, pos, vel, d, alpha, nsteps, dt, 6, lam, deposit="cic")

    def loss(Gx, Ux, dx):
        _, _, J, _ = oracle.run(Gx, Ux, pos, vel, dx, nsteps, dt)
        return 0.5 * float(((J - Jt) ** 2).sum())

    eps = 1e-4
    for p in range(0, d.shape[0], 4):
        dp, dm = d.copy(), d.copy()
        dp[p] *= 1 + eps
        dm[p] *= 1 - eps
        fd = (loss(G, U, dp) - loss(G, U, dm)) / (2 * eps * d[p])
        assert abs(fd - gd[p]) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(gd).max())
    fd = (loss(oracle.make_grid(N, alpha=alpha + eps, deposit="cic"), U, d)
          - loss(oracle.make_grid(N, alpha=alpha - eps, deposit="cic"), U, d)) / (2 * eps)
    assert abs(fd - ga) <= 1e-5 * abs(fd)
    for f in np.argsort(-np.abs(gU).ravel())[:8]:
        Up, Um = U.copy().reshape(-1), U.copy().reshape(-1)
        Up[f] += eps
        Um[f] -= eps
        fd = (loss(G, Up.reshape(U.shape), d) - loss(G, Um.reshape(U.shape), d)) / (2 * eps)
        assert abs(fd - gU.ravel()[f]) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(gU).max())


def test_adjoint_refuses_physics_it_does_not_differentiate(Sim):
    from paper_2603_26691_gb300._lib import StError

    N, U, pos, vel, d, alpha = _case(N=8, n=33)
    sim = Sim(N, precision="fp64")
    sim.set_params(reorder_every=0)
    sim.set_fluid(U)
    sim.add_particles(pos, d, vel)
    for ph in (dict(drag="schiller_naumann"), dict(gather="ngp"), dict(integrator="semi_implicit")):
        sim.set_physics(**ph)
        with pytest.raises(StError):
            sim.adjoint_forward(3, 1e-3, 1)
    sim.close()


@pytest.mark.parametrize("deposit", ["cell", "cic"])
def test_autograd_function_quadratic_loss(Sim, deposit):
    import torch

    from paper_2603_26691_gb300.autograd import lagrangian_sources

    N, U, pos, vel, d, alpha = _case(N=12, n=500)
    nsteps, dt = 25, 1e-3
    sim = Sim(N, precision="fp64")
    sim.set_physics(deposit=deposit)
    dev = torch.device("cuda")
    dt_ = torch.tensor(d, device=dev, requires_grad=True)
    at = torch.tensor(alpha, dtype=torch.float64, requires_grad=True)
    Ut = torch.tensor(U, device=dev, requires_grad=True)
    with torch.no_grad():
        Jt = lagrangian_sources(dt_ * 1.05, at, Ut, sim, pos, vel, nsteps, dt, 10).clone()
    J = lagrangian_sources(dt_, at, Ut, sim, pos, vel, nsteps, dt, 10)
    L = 0.5 * ((J - Jt) ** 2).sum()
    L.backward()
    sim.close()
    G = oracle.make_grid(N, alpha=alpha, deposit=deposit)
    _, _, oJ, _ = oracle.run(G, U, pos, vel, d, nsteps, dt)
    _, _, oJt, _ = oracle.run(G, U, pos, vel, d * 1.05, nsteps, dt)
    ogd, oga, ogU = oracle.adjoint(G, U, pos, vel, d, nsteps, dt, oJ - oJt)
    gd = dt_.grad.cpu().numpy()
    assert np.abs(gd - ogd).max() <= 1e-8 * np.abs(ogd).max()
    assert abs(at.grad.item() - oga) <= 1e-8 * abs(oga)
    gU = Ut.grad.cpu().numpy().reshape(-1, 3)
    assert np.abs(gU - ogU).max() <= 1e-8 * np.abs(ogU).max()


def test_autograd_backward_after_another_forward_raises(Sim):
    """One handle records one run: a backward through an earlier forward, after a second forward
    replaced the recorded run, must raise instead of returning the second run's gradients."""
    import torch

    from paper_2603_26691_gb300.autograd import lagrangian_sources

    N, U, pos, vel, d, alpha = _case(N=12, n=200)
    sim = Sim(N, precision="fp64")
    dev = torch.device("cuda")
    d1 = torch.tensor(d, device=dev, requires_grad=True)
    d2 = torch.tensor(d * 1.1, device=dev, requires_grad=True)
    at = torch.tensor(alpha, dtype=torch.float64, requires_grad=True)
    Ut = torch.tensor(U, device=dev)
    J1 = lagrangian_sources(d1, at, Ut, sim, pos, vel, 5, 1e-3, 5)
    J2 = lagrangian_sources(d2, at, Ut, sim, pos, vel, 5, 1e-3, 5)
    with pytest.raises(RuntimeError, match="changed after this forward"):
        (J1.sum() + J2.sum()).backward()
    # the latest forward alone still differentiates
    J3 = lagrangian_sources(d1, at, Ut, sim, pos, vel, 5, 1e-3, 5)
    (J3 ** 2).sum().backward()
    assert torch.isfinite(d1.grad).all()
    sim.close()


def test_adjoint_tg_fourier_64_1e7_sampled(Sim):
    """Adjoint workload: 64^3 Taylor-Green + 10% Fourier (FP32-rounded), 1e7 particles, 200 steps of 1e-3,
    checkpoints every 20.  Per-particle dL/dd of a linear loss depends only on that particle's path, so
    the oracle checks a seeded sample of particles at full size."""
    import torch

    w = inputs.WORKLOADS["tgf64_adjoint_1e7"]
    U = w.make_field()
    N, n = w.grid, w.n
    lam = np.random.default_rng(17).standard_normal((3, N ** 3)) * 1e-3
    sim = Sim(N, precision="fp64")
    sim.set_params(reorder_every=0)
    sim.set_fluid(U)
    sim.reserve(n)
    q = inputs.lognormal_qtable()
    for first in range(0, n, 5_000_000):
        cnt = min(5_000_000, n - first)
        p, v, dd, ids = sim.gen_particles(w.seed, first, cnt, q)
        sim.add_particles(p, dd, v, ids)
    sim.adjoint_forward(w.steps, w.dt, w.extra["checkpoint"])
    gd, ga, gU = sim.adjoint_backward(torch.as_tensor(lam, device="cuda"))
    gd = gd.cpu().numpy()
    sim.close()
    sample = np.random.default_rng(3).choice(n, 64, replace=False)
    pos, vel, d, _ = inputs.particles_at(w.seed, sample)
    ogd, _, _ = oracle.adjoint(oracle.make_grid(N), U, pos, vel, d, w.steps, w.dt, lam)
    assert np.abs(gd[sample] - ogd).max() <= 1e-8 * np.abs(ogd).max()
    assert np.isfinite(ga) and np.all(np.isfinite(gU.cpu().numpy()))
