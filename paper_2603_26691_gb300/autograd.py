"""Differentiable time-summed source field: a torch.autograd.Function over the CUDA adjoint.

J = LagrangianSources.apply(d, alpha, U, sim, pos0, vel0, nsteps, dt, checkpoint_every)
runs nsteps steps of the particles (initial positions pos0, velocities vel0, diameters d) with
drag scale alpha through the frozen fluid U - in FP64 on an FP64 Sim, in FP32 on a mixed
FP32-velocity Sim - and returns the per-cell impulse summed over the run, J [3, ncell].  Its backward calls the library's adjoint
(st_adjoint_backward): dL/dd per particle, dL/dalpha and dL/dU, with the deposit cell held
fixed under the cell deposit (its derivative is zero almost everywhere) and the deposit weights
differentiated under the cloud-in-cell deposit.  All arithmetic runs in the CUDA library.

The handle keeps one recorded run: the backward of a forward raises if anything changed the
simulation after that forward (another forward, a step, new parameters, particles or fluid),
because the handle would then differentiate a different run.
"""
from __future__ import annotations

import torch


class LagrangianSources(torch.autograd.Function):
    @staticmethod
    def forward(ctx, d, alpha, U, sim, pos0, vel0, nsteps, dt, checkpoint_every):
        p = dict(sim.params)
        p["drag_scale"] = float(alpha)
        sim.set_params(**p)
        sim.set_fluid(U.detach())
        sim.clear_particles()
        dd = d.detach()
        if isinstance(dd, torch.Tensor) and dd.is_cuda:
            pos0 = torch.as_tensor(pos0, dtype=torch.float64, device=dd.device)
            vel0 = None if vel0 is None else torch.as_tensor(vel0, dtype=torch.float64, device=dd.device)
        sim.add_particles(pos0, dd, vel0)
        sim.sources(reset=True)
        sim.adjoint_forward(int(nsteps), float(dt), int(checkpoint_every))
        J = sim.sources()
        ctx.sim = sim
        ctx.generation = sim.generation
        ctx.meta = (d.dtype, d.device, alpha, U.shape, U.dtype, U.device)
        return J

    @staticmethod
    def backward(ctx, gJ):
        d_dtype, d_dev, alpha, U_shape, U_dtype, U_dev = ctx.meta
        if ctx.sim.generation != ctx.generation:
            raise RuntimeError("the simulation changed after this forward (another forward, a step, or new "
                               "parameters, particles or fluid): its recorded run is no longer this one; "
                               "call backward before changing the simulation, or use one Sim per graph")
        gd, ga, gU = ctx.sim.adjoint_backward(gJ.detach().to(torch.float64).contiguous())
        gd = gd.to(device=d_dev, dtype=d_dtype)
        ga_t = torch.as_tensor(ga, dtype=alpha.dtype if isinstance(alpha, torch.Tensor) else torch.float64,
                               device=alpha.device if isinstance(alpha, torch.Tensor) else d_dev)
        gU = gU.reshape(U_shape).to(device=U_dev, dtype=U_dtype)
        return gd, ga_t, gU, None, None, None, None, None, None


def lagrangian_sources(d, alpha, U, sim, pos0, vel0, nsteps, dt, checkpoint_every=20):
    return LagrangianSources.apply(d, alpha, U, sim, pos0, vel0, nsteps, dt, checkpoint_every)
