"""torch.autograd.Function for the SHO projection.

Forward:  c = P(psi; X)  (sho_project).
Backward, for an upstream gradient g = dL/dc:
  dL/dpsi = h^3 E(g)          -- sho_add_scaled(alpha = h^3, overwrite): the expansion is the adjoint of
                                 the projection in the plain grid inner product up to the quadrature
                                 weight h^3 (Sec. 3.2 steps 1 and 3); the library applies the weight in
                                 its z-pass and clears the output itself
  dL/dX   = sho_forces(psi, g) -- projection at numax+1 and the ladder relation of the Hermite
                                 functions (derivative of the recursion of Sec. 3.7)
Every step runs in libsho's kernels; this module only wires them into autograd.
"""
from __future__ import annotations

import torch

from . import api


class ShoProject(torch.autograd.Function):
    @staticmethod
    def forward(ctx, psi, pos, sigma, numax, cube, h, periodic, prec):
        pos_h = pos.detach().to("cpu", torch.float64).contiguous()
        sig_h = sigma.detach().to("cpu", torch.float64).contiguous() if torch.is_tensor(sigma) else \
            torch.as_tensor(sigma, dtype=torch.float64)
        c = api.project(psi.detach(), pos_h.numpy(), sig_h.numpy(), numax, cube, h, periodic, prec=prec)
        ctx.save_for_backward(psi)
        ctx.pos_h, ctx.sig_h = pos_h, sig_h
        ctx.args = (numax, cube, h, periodic, prec)
        ctx.pos_meta = (pos.dtype, pos.device)
        return c

    @staticmethod
    def backward(ctx, g):
        (psi,) = ctx.saved_tensors
        numax, cube, h, periodic, prec = ctx.args
        g = g.contiguous()
        grad_psi = grad_pos = None
        if ctx.needs_input_grad[0]:
            grad_psi = torch.empty_like(psi)
            api.add(grad_psi, g, ctx.pos_h.numpy(), ctx.sig_h.numpy(), numax, cube, h, periodic, prec=prec,
                    alpha=h ** 3, overwrite=True)
        if ctx.needs_input_grad[1]:
            f = api.forces(psi.detach(), g, ctx.pos_h.numpy(), ctx.sig_h.numpy(), numax, cube, h, periodic,
                           prec=prec)
            grad_pos = f.to(dtype=ctx.pos_meta[0], device=ctx.pos_meta[1])
        return grad_psi, grad_pos, None, None, None, None, None, None


def sho_project(psi, pos, sigma, numax: int, cube: int, h: float, periodic: bool = True, prec: str = "fp64"):
    """Differentiable projection: gradients flow to psi (via the expansion) and to the atom positions
    (via the forces kernel)."""
    if not torch.is_tensor(pos):
        pos = torch.as_tensor(pos, dtype=torch.float64)
    return ShoProject.apply(psi, pos, sigma, numax, cube, h, periodic, prec)
