"""torch.autograd access to the fermion action S = phi^+ (D^+ D)^-1 phi.

The forward pass runs the two solves of the link force in the CUDA library
and returns S; the backward pass multiplies the library's dS/dU (the
hand-written hopping outer-product and clover-leaf kernels) by the incoming
gradient.  For a real S, dS/dU = dS/dRe U + i dS/dIm U is torch's gradient
convention for complex leaves.
"""
from __future__ import annotations

import torch

from .api import CloverOperator, Gauge, Lattice, solve_params


class FermionAction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U, phi, lattice: Lattice, kappa: float, csw: float, params):
        prec = params.smoother_prec if params.precond else 64
        if params.method == 2:
            prec = min(prec, 32)
        gauge = Gauge(lattice, U.detach(), storage_prec=prec)
        op = CloverOperator(gauge, kappa, csw)
        g, S, info = op.force(phi.detach(), params)
        ctx.save_for_backward(g)
        ctx.info = info
        return torch.tensor(S, dtype=torch.float64, device=U.device)

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return grad_out.to(g.device) * g, None, None, None, None, None


def fermion_action(U: torch.Tensor, phi: torch.Tensor, lattice: Lattice, kappa: float, csw: float,
                   params=None, **kw) -> torch.Tensor:
    """S = phi^+ (D^+ D)^-1 phi as a differentiable function of the links U."""
    p = params if params is not None else solve_params(**kw)
    return FermionAction.apply(U, phi, lattice, kappa, csw, p)
