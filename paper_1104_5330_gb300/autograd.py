"""Differentiable time stepping over the C ABI's ts_step / ts_adjoint_step.

``transport_steps(grid, F0, kappa, eta, kappa_s, dt, nsteps)`` returns F after
nsteps RK4 steps; its backward pass calls the library's discrete adjoint
(exact transpose of the discrete step; the paper defines no adjoint) and
returns dObj/dF0, dObj/dkappa and dObj/deta. Step states are kept by sqrt(N)
checkpointing: the forward stores every ceil(sqrt(n))-th state; the backward
recomputes one segment at a time from its checkpoint (ts_step) and walks it
back (ts_adjoint_step), so memory is O(sqrt(n)) fields and the forward is
recomputed once.

``outgoing_flux(grid, F)`` is the radial flux through R2 per group (Eq. Flux,
App. A) with the library's quadrature weights (ts_flux_weights).

All tensors live on the grid's device; kappa, eta, kappa_s are float64
[G][Nr][Ntheta][Nphi]; F has the grid's element type. The grid's scattering
kernel (set with set_scattering_anisotropy / set_scattering_quadrupole) applies
to the forward steps and to their adjoint alike; the grid must use the TS_RK4
scheme on the Chebyshev radial grid (the adjoint's scope).
"""
from __future__ import annotations

import math

import torch

from . import ts as _ts


class TransportSteps(torch.autograd.Function):
    @staticmethod
    def forward(ctx, F0, kappa, eta, grid, kappa_s, inflow_R1, inflow_R2, dt, nsteps, segment):
        grid.set_coeffs(kappa, eta, kappa_s, inflow_R1, inflow_R2)
        seg = segment or max(1, math.ceil(math.sqrt(nsteps)))
        F = F0.detach().clone().contiguous()
        checkpoints = [F.clone()]
        for n in range(nsteps):
            _ts.ts_step(grid.handle, F, dt, 1)
            if (n + 1) % seg == 0 and n + 1 < nsteps:
                checkpoints.append(F.clone())
        ctx.grid = grid
        ctx.dt, ctx.nsteps, ctx.seg = dt, nsteps, seg
        ctx.coeffs = (kappa.detach(), eta.detach(), kappa_s, inflow_R1, inflow_R2)
        ctx.checkpoints = checkpoints
        return F

    @staticmethod
    def backward(ctx, gF):
        grid, dt, nsteps, seg = ctx.grid, ctx.dt, ctx.nsteps, ctx.seg
        kappa, eta, kappa_s, g1, g2 = ctx.coeffs
        grid.set_coeffs(kappa, eta, kappa_s, g1, g2)       # the adjoint uses the forward's fields
        lam = gF.detach().to(grid.dtype).clone().contiguous()
        gk = torch.zeros(grid.coef_shape, dtype=torch.float64, device=lam.device)
        ge = torch.zeros_like(gk)
        nseg = len(ctx.checkpoints)
        for s in range(nseg - 1, -1, -1):
            start = s * seg
            stop = min(nsteps, start + seg)
            states = [ctx.checkpoints[s]]
            F = ctx.checkpoints[s].clone()
            for _ in range(start, stop - 1):
                _ts.ts_step(grid.handle, F, dt, 1)
                states.append(F.clone())
            for n in range(stop - 1, start - 1, -1):
                _ts.ts_adjoint_step(grid.handle, states[n - start], lam, gk, ge, dt)
            del states
        ctx.checkpoints = None
        return lam, gk, ge, None, None, None, None, None, None, None


def transport_steps(grid, F0, kappa, eta, kappa_s=None, dt=None, nsteps=1, inflow_R1=None,
                    inflow_R2=None, segment=None):
    """F after `nsteps` steps, differentiable in F0, kappa and eta."""
    if kappa_s is None:
        kappa_s = torch.zeros(grid.coef_shape, dtype=torch.float64, device=F0.device)
    return TransportSteps.apply(F0, kappa, eta, grid, kappa_s, inflow_R1, inflow_R2, dt,
                                int(nsteps), segment)


def outgoing_flux(grid, F):
    """J_R2 per group: R2^2 int sin(th) dth dph int sin(Th) cos(Th) dTh dPh F(R2) (Eq. Flux)."""
    w = grid.flux_weights().to(F.dtype)
    return torch.einsum("gjlkm,jlkm->g", F[:, -1], w)
