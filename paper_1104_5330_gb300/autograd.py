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
App. A), evaluated by the library (ts_outgoing_flux) with the adjoint seed of
ts_outgoing_flux_adjoint as its backward.

All tensors live on the grid's device; kappa, eta, kappa_s are float64
[G][Nr][Ntheta][Nphi]; F has the grid's element type. The grid's scattering
kernel (set with set_scattering_anisotropy / set_scattering_quadrupole) applies
to the forward steps and to their adjoint alike; the grid must use the TS_RK4 or
TS_AB2 scheme on the Chebyshev radial grid, filter off (the adjoint's scope).
"""
from __future__ import annotations

import math

import torch

from . import ts as _ts


class TransportSteps(torch.autograd.Function):
    """RK4 grids checkpoint F at segment starts. AB2 grids (the paper's scheme)
    checkpoint the pair (F_s, K_{s-1}) -- K of the state before, from ts_rhs -- so
    that a segment's recomputation resumes the two-level marching through
    ts_set_history; their backward walks ts_adjoint_step_ab2 with the two adjoint
    levels (dObj/dF_{n+1}, dObj/dF_{n+2})."""

    @staticmethod
    def forward(ctx, F0, kappa, eta, grid, kappa_s, inflow_R1, inflow_R2, dt, nsteps, segment):
        grid.set_coeffs(kappa, eta, kappa_s, inflow_R1, inflow_R2)
        ab2 = grid.desc.scheme == _ts.TS_AB2
        seg = segment or max(1, math.ceil(math.sqrt(nsteps)))
        F = F0.detach().clone().contiguous()
        checkpoints = [(F.clone(), None)]
        if ab2:
            grid.reset_history()
        for n in range(nsteps):
            Kh = None
            if ab2 and (n + 1) % seg == 0 and n + 1 < nsteps:
                Kh = torch.empty_like(F)
                _ts.ts_rhs(grid.handle, F, Kh)          # K_n: the history of step n + 1
            _ts.ts_step(grid.handle, F, dt, 1)
            if (n + 1) % seg == 0 and n + 1 < nsteps:
                checkpoints.append((F.clone(), Kh))
        ctx.grid = grid
        ctx.ab2 = ab2
        ctx.dt, ctx.nsteps, ctx.seg = dt, nsteps, seg
        ctx.coeffs = (kappa.detach(), eta.detach(), kappa_s, inflow_R1, inflow_R2)
        ctx.checkpoints = checkpoints
        return F

    @staticmethod
    def backward(ctx, gF):
        grid, dt, nsteps, seg, ab2 = ctx.grid, ctx.dt, ctx.nsteps, ctx.seg, ctx.ab2
        kappa, eta, kappa_s, g1, g2 = ctx.coeffs
        grid.set_coeffs(kappa, eta, kappa_s, g1, g2)       # the adjoint uses the forward's fields
        lam = gF.detach().to(grid.dtype).clone().contiguous()
        lam_prev = torch.zeros_like(lam)
        gk = torch.zeros(grid.coef_shape, dtype=torch.float64, device=lam.device)
        ge = torch.zeros_like(gk)
        nseg = len(ctx.checkpoints)
        for s in range(nseg - 1, -1, -1):
            start = s * seg
            stop = min(nsteps, start + seg)
            F0s, Kh = ctx.checkpoints[s]
            states = [F0s]
            F = F0s.clone()
            if ab2:
                if Kh is None:
                    grid.reset_history()
                else:
                    _ts.ts_set_history(grid.handle, F, Kh)
            for _ in range(start, stop - 1):
                _ts.ts_step(grid.handle, F, dt, 1)
                states.append(F.clone())
            for n in range(stop - 1, start - 1, -1):
                if ab2:
                    _ts.ts_adjoint_step_ab2(grid.handle, states[n - start], lam, lam_prev, gk, ge,
                                            dt, n == 0)
                else:
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


class OutgoingFlux(torch.autograd.Function):
    """J_R2 per group through the library (ts_outgoing_flux); its backward is
    the library's adjoint seed (ts_outgoing_flux_adjoint)."""

    @staticmethod
    def forward(ctx, F, grid):
        ctx.grid = grid
        J = torch.empty(grid.shape[0], dtype=torch.float64, device=F.device)
        _ts.ts_outgoing_flux(grid.handle, F.detach().contiguous(), J)
        return J

    @staticmethod
    def backward(ctx, gJ):
        grid = ctx.grid
        lam = torch.empty(grid.shape, dtype=grid.dtype, device=gJ.device)
        _ts.ts_outgoing_flux_adjoint(grid.handle, gJ.detach().to(torch.float64).contiguous(), lam)
        return lam, None


def outgoing_flux(grid, F):
    """J_R2 per group, R2^2 int sin(th) dth dph int sin(Th) cos(Th) dTh dPh F(R2)
    (Eq. Flux), float64 [G], differentiable in F."""
    return OutgoingFlux.apply(F, grid)
