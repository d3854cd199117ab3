"""Differentiable Chebyshev time propagation w.r.t. the on-site (gate) potential.

ChebPropagate.apply(V, psi0, lat, dt, nsteps, a, b, every, trunc) returns
psi_S = U(dt)^nsteps psi0 for the lattice `lat` with its potential set to V.
Both passes are single library calls: the forward pass is
pvsc_cheb_propagate_checkpointed (the state kept every `every` steps), the
backward pass pvsc_cheb_propagate_adjoint (the segments walked in reverse,
each recomputed from its checkpoint, the hand-written adjoint step run from
its last step to its first, dL/dV accumulated in fp64).  a and b (the
Chebyshev scaling of Eq. U_1) are held fixed.  This module only marshals
tensors.

Gradients follow torch's convention for complex tensors: for a real loss L,
grad_output G satisfies dL = Re <G | d psi_S>.
"""
from __future__ import annotations

import torch

from . import cheb_propagate_adjoint, cheb_propagate_checkpointed


class ChebPropagate(torch.autograd.Function):
    @staticmethod
    def forward(ctx, V, psi0, lat, dt, nsteps, a, b, every=20, trunc=1e-14):
        lat.set_potential(V.detach())
        psi = psi0.detach().to(torch.complex128).clone().contiguous()
        psi, ckpts = cheb_propagate_checkpointed(lat, psi, dt, nsteps, every, a, b, trunc)
        ctx.lat, ctx.dt, ctx.nsteps, ctx.a, ctx.b, ctx.every, ctx.trunc = lat, dt, nsteps, a, b, every, trunc
        ctx.ckpts = ckpts
        ctx.V = V.detach()
        return psi

    @staticmethod
    def backward(ctx, grad_psi):
        lat = ctx.lat
        lat.set_potential(ctx.V)
        G = grad_psi.detach().to(torch.complex128).clone().contiguous()
        dLdV = torch.zeros(lat.n_sites, dtype=torch.float64, device=G.device)
        cheb_propagate_adjoint(lat, ctx.ckpts, G, ctx.dt, ctx.nsteps, ctx.every, ctx.a, ctx.b, dLdV, ctx.trunc)
        return dLdV.to(ctx.V.dtype), G, None, None, None, None, None, None, None


def propagate_with_grad(V, psi0, lat, dt, nsteps, a, b, every=20, trunc=1e-14):
    return ChebPropagate.apply(V, psi0, lat, dt, nsteps, a, b, every, trunc)
