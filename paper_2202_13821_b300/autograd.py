"""torch.autograd wrappers of the DG-HGKS step and kinetic energy.

``rollout(Q0, mu, solver, dt, nsteps)`` advances ``nsteps`` S2O4 steps
(Sec. 3, Eq. two-stage) with the FP64 solver, keeping a device checkpoint of
Q^n before every step; its backward pass runs ``dghgks_adjoint_step`` from
the last checkpoint to the first (each recomputes its Q*), accumulating the
viscosity cotangent on the device.  ``kinetic_energy(Q, solver, rho0)`` is
E_k of Sec. 5.3 with its gradient from ``dghgks_kinetic_energy_vjp``.  All
arithmetic runs in libdghgks.so; torch only holds buffers and the tape.

    J = kinetic_energy(rollout(Q0, mu, solver, dt, N), solver)
    J.backward()   # -> Q0.grad, mu.grad
"""
from __future__ import annotations

import torch

from . import api


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, Q0, mu, solver, dt, nsteps):
        solver.set_mu(float(mu))
        Q = Q0.detach().contiguous().clone()
        ckpts = []
        for _ in range(int(nsteps)):
            ckpts.append(Q.clone())
            solver.step(Q, dt)
        solver.status()
        ctx.solver, ctx.dt, ctx.ckpts = solver, float(dt), ckpts
        ctx.mu_shape = mu.shape
        return Q

    @staticmethod
    def backward(ctx, gQ):
        lam = gQ.detach().contiguous().clone()
        dmu = torch.zeros(1, dtype=torch.float64, device=lam.device)
        for Qn in reversed(ctx.ckpts):
            api.dghgks_adjoint_step(ctx.solver.ctx, Qn, lam, ctx.dt, lam, dmu)
        ctx.ckpts = None
        return lam, dmu.reshape(ctx.mu_shape), None, None, None


class _KineticEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, Q, solver, rho0):
        ctx.save_for_backward(Q)
        ctx.solver, ctx.rho0 = solver, float(rho0)
        return torch.tensor(solver.kinetic_energy(Q, rho0), dtype=torch.float64, device=Q.device)

    @staticmethod
    def backward(ctx, g):
        (Q,) = ctx.saved_tensors
        out = torch.empty_like(Q)
        api.dghgks_kinetic_energy_vjp(ctx.solver.ctx, Q.contiguous(), ctx.rho0, out)
        return g * out, None, None


def rollout(Q0, mu, solver, dt, nsteps):
    """nsteps S2O4 steps with checkpointed adjoint; mu is a 0-dim float64 tensor."""
    return _Rollout.apply(Q0, mu, solver, dt, nsteps)


def kinetic_energy(Q, solver, rho0=1.0):
    return _KineticEnergy.apply(Q, solver, rho0)
