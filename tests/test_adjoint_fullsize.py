"""The FP64 adjoint at the adjoint workload's full size: a 64^3 Taylor-Green field with a 10 % random
Fourier perturbation (FP32-rounded), 1e7 particles with lognormal diameters, 200 steps of 1e-3 with
checkpoints every 20, and the loss L = 1/2 |Jtot - Jtarget|^2 with the target field from the same run with
diameters x 1.05.  The gradients with respect to the diameters, the drag scale and the fluid field are
checked at that size in two ways.

* With the cloud-in-cell deposit J is a continuous function of every input, so the full run's loss can
  be differentiated by central differences (eps 1e-4) of the GPU's own FP64 forward run: the drag scale
  alone, and one direction each in the 1e7 diameters and in the 786,432 fluid values, taken along the
  adjoint's own gradient plus a random part (a directional derivative checks every component at once;
  along the gradient the terms do not cancel, so the derivative stands well above the finite
  differences' noise from particles that cross the trilinear weights' kinks).  The bound is 1e-5
  relative.
* With the default deposit into the containing cell (piecewise constant in the positions, so central
  differences of the full run jump where a particle changes cell) the adjoint of a fixed lam = dL/dJtot is
  a sum of per-particle terms, each depending on that particle's path alone: the full run's dL/dalpha and
  dL/dU equal those of a seeded 64-particle sample plus those of the rest, run apart with the same lam,
  and the sample's three gradients equal the oracle's FP64 adjoint of the sample."""
import numpy as np
import pytest

import oracle
from paper_2603_26691_gb300 import inputs

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

W = inputs.WORKLOADS["tgf64_adjoint_1e7"]


@pytest.fixture(scope="module")
def setup():
    import torch

    assert torch.cuda.is_available()
    from paper_2603_26691_gb300.sim import Sim

    U = W.make_field()
    sim = Sim(W.grid, precision="fp64")
    q = inputs.lognormal_qtable()
    parts = [sim.gen_particles(W.seed, first, min(5_000_000, W.n - first), q)
             for first in range(0, W.n, 5_000_000)]
    pos = torch.cat([p[0] for p in parts], dim=1)
    vel = torch.cat([p[1] for p in parts], dim=1)
    d = torch.cat([p[2] for p in parts])
    del parts
    yield Sim, sim, U, pos, vel, d
    sim.close()


def _load(sim, U, pos, vel, d, alpha=1.0, deposit="cell"):
    sim.set_params(drag_scale=alpha, reorder_every=0)
    sim.set_physics(deposit=deposit)
    sim.set_fluid(U)
    sim.clear_particles()
    sim.sources(reset=True)
    sim.reserve(int(d.shape[0]))
    sim.add_particles(pos, d, vel)


def _sources(sim, U, pos, vel, d, alpha=1.0, deposit="cell"):
    """Jtot of the forward run (the plain FP64 step, no reordering), on the device."""
    _load(sim, U, pos, vel, d, alpha, deposit)
    sim.step(W.steps, W.dt)
    return sim.sources(reset=True)


def _grads(sim, U, pos, vel, d, lam, deposit="cell"):
    _load(sim, U, pos, vel, d, 1.0, deposit)
    sim.adjoint_forward(W.steps, W.dt, W.extra["checkpoint"])
    J = sim.sources(reset=True)
    gd, ga, gU = sim.adjoint_backward(lam)
    return J, gd, ga, gU


def test_adjoint_fullsize_cic_central_differences(setup):
    import torch

    _, sim, U, pos, vel, d = setup
    Jt = _sources(sim, U, pos, vel, d * 1.05, deposit="cic")
    J0 = _sources(sim, U, pos, vel, d, deposit="cic")
    lam = J0 - Jt
    J, gd, ga, gU = _grads(sim, U, pos, vel, d, lam, deposit="cic")
    # the recorded forward run is the plain run
    assert float((J - J0).abs().max()) <= 1e-14 * float(J0.abs().max())

    def loss(Ux=U, dx=d, alpha=1.0):
        Jx = _sources(sim, Ux, pos, vel, dx, alpha, deposit="cic")
        return 0.5 * float(((Jx - Jt) ** 2).sum())

    eps = 1e-4
    fd = (loss(alpha=1.0 + eps) - loss(alpha=1.0 - eps)) / (2 * eps)
    assert abs(fd - ga) <= 1e-5 * abs(fd), (fd, ga)

    # relative diameter changes r: the gradient's direction (scaled to at most 1) plus a random part
    gen = torch.Generator(device=d.device).manual_seed(23)
    gdd = gd * d
    r = gdd / gdd.abs().max() + 0.2 * torch.randn(d.shape, dtype=torch.float64, device=d.device, generator=gen)
    fd = (loss(dx=d * (1 + eps * r)) - loss(dx=d * (1 - eps * r))) / (2 * eps)
    adj = float((gdd * r).sum())
    assert abs(fd - adj) <= 1e-5 * abs(fd), (fd, adj)

    gUn = gU.cpu().numpy().reshape(U.shape)
    R = gUn / np.abs(gUn).max() + 0.2 * np.random.default_rng(29).standard_normal(U.shape)
    fd = (loss(Ux=U + eps * R) - loss(Ux=U - eps * R)) / (2 * eps)
    adj = float((gUn * R).sum())
    assert abs(fd - adj) <= 1e-5 * abs(fd), (fd, adj)


def test_adjoint_fullsize_cell_deposit_sum_of_particles_and_oracle_sample(setup):
    import torch

    _, sim, U, pos, vel, d = setup
    Jt = _sources(sim, U, pos, vel, d * 1.05)
    J0 = _sources(sim, U, pos, vel, d)
    lam = J0 - Jt
    _, gd, ga, gU = _grads(sim, U, pos, vel, d, lam)

    n = int(d.shape[0])
    sample = np.sort(np.random.default_rng(31).choice(n, 64, replace=False))
    keep = torch.ones(n, dtype=torch.bool, device=d.device)
    keep[torch.as_tensor(sample, device=d.device)] = False
    si = torch.as_tensor(sample, device=d.device)
    _, gdS, gaS, gUS = _grads(sim, U, pos[:, si], vel[:, si], d[si], lam)
    _, gdR, gaR, gUR = _grads(sim, U, pos[:, keep], vel[:, keep], d[keep], lam)

    # per-particle gradients do not depend on the other particles
    gmax = float(gd.abs().max())
    assert float((gd[si] - gdS).abs().max()) <= 1e-14 * gmax
    assert float((gd[keep] - gdR).abs().max()) <= 1e-14 * gmax
    # the full run's dL/dalpha (FP64 block sums) and dL/dU (exact fixed-point sums, one rounding) are the
    # sums of the two parts' within rounding
    assert abs(ga - (gaS + gaR)) <= 1e-12 * abs(ga)
    gUn, gUSn, gURn = gU.cpu().numpy(), gUS.cpu().numpy(), gUR.cpu().numpy()
    assert np.abs(gUn - (gUSn + gURn)).max() <= 1e-13 * np.abs(gUn).max()
    # the sample's own contribution is not negligible beside rounding (the sum check sees it)
    assert np.abs(gUSn).max() > 1e-9 * np.abs(gUn).max()

    # the sample against the oracle's FP64 adjoint with the same lam
    G = oracle.make_grid(W.grid)
    P = pos[:, si].cpu().numpy()
    V = vel[:, si].cpu().numpy()
    D = d[si].cpu().numpy()
    ogd, oga, ogU = oracle.adjoint(G, U, P, V, D, W.steps, W.dt, lam.cpu().numpy())
    assert np.abs(gdS.cpu().numpy() - ogd).max() <= 1e-9 * np.abs(ogd).max()
    assert abs(gaS - oga) <= 1e-9 * abs(oga)
    assert np.abs(gUSn - ogU).max() <= 1e-9 * np.abs(ogU).max()
