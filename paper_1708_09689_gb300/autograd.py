"""Differentiable Chebyshev time propagation w.r.t. the on-site (gate) potential.

ChebPropagate.apply(V, psi0, lat, dt, nsteps, a, b, every, trunc) returns
psi_S = U(dt)^nsteps psi0 for the lattice `lat` with its potential set to V.
The backward pass is the library's hand-written adjoint: the forward pass
keeps the state every `every` steps; the backward pass walks the segments in
reverse, recomputes the states of a segment from its checkpoint with the
forward kernels, and runs pvsc_cheb_adjoint_step from the last step of the
segment to the first, accumulating dL/dV in fp64 and carrying dL/dpsi back.
a and b (the Chebyshev scaling of Eq. U_1) are held fixed.

Gradients follow torch's convention for complex tensors: for a real loss L,
grad_output G satisfies dL = Re <G | d psi_S>.
"""
from __future__ import annotations

import torch

from . import (C128, OP_ADJOINT, OP_SERIES, cheb_adjoint_step, cheb_propagate,
               propagation_coeffs, work_buffer)


class ChebPropagate(torch.autograd.Function):
    @staticmethod
    def forward(ctx, V, psi0, lat, dt, nsteps, a, b, every=20, trunc=1e-14):
        lat.set_potential(V.detach())
        K = len(propagation_coeffs(a * dt, trunc))
        R = 1 if psi0.dim() == 1 else psi0.shape[1]
        work = work_buffer(lat.work_bytes(OP_SERIES, R, C128, K))
        psi = psi0.detach().clone().contiguous()
        ckpts = []
        s = 0
        while s < nsteps:
            ckpts.append(psi.clone())
            n = min(every, nsteps - s)
            cheb_propagate(lat, psi, dt, n, a, b, trunc, C128, work)
            s += n
        ctx.lat, ctx.dt, ctx.nsteps, ctx.a, ctx.b, ctx.every, ctx.trunc = lat, dt, nsteps, a, b, every, trunc
        ctx.ckpts = ckpts
        ctx.V = V.detach()
        return psi

    @staticmethod
    def backward(ctx, grad_psi):
        lat, dt, a, b, every, trunc = ctx.lat, ctx.dt, ctx.a, ctx.b, ctx.every, ctx.trunc
        lat.set_potential(ctx.V)
        K = len(propagation_coeffs(a * dt, trunc))
        R = 1 if grad_psi.dim() == 1 else grad_psi.shape[1]
        fwork = work_buffer(lat.work_bytes(OP_SERIES, R, C128, K))
        awork = work_buffer(lat.work_bytes(OP_ADJOINT, R, C128, K))
        G = grad_psi.detach().to(torch.complex128).clone().contiguous()
        dLdV = torch.zeros(lat.n_sites, dtype=torch.float64, device=G.device)
        nseg = len(ctx.ckpts)
        tmp = torch.empty_like(G)  # one fixed buffer, so the captured step graph is reused
        for seg in range(nseg - 1, -1, -1):
            s0 = seg * every
            n = min(every, ctx.nsteps - s0)
            states = [ctx.ckpts[seg]]
            for _ in range(n - 1):
                tmp.copy_(states[-1])
                cheb_propagate(lat, tmp, dt, 1, a, b, trunc, C128, fwork)
                states.append(tmp.clone())
            for j in range(n - 1, -1, -1):
                cheb_adjoint_step(lat, states[j], G, dt, a, b, dLdV, trunc, awork)
        return dLdV.to(ctx.V.dtype), G, None, None, None, None, None, None, None


def propagate_with_grad(V, psi0, lat, dt, nsteps, a, b, every=20, trunc=1e-14):
    return ChebPropagate.apply(V, psi0, lat, dt, nsteps, a, b, every, trunc)
