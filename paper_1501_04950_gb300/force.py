"""torch.autograd.Function for the fermion action S = phi^+ (D_bb^+ D_bb)^-1 phi.

The forward pass asks libdwf for S = Re phi^+ X with X = (D_bb^+ D_bb)^-1 phi
(dwf_action: CG and an FP64 device reduction).  The backward pass asks libdwf
for the link gradient (dwf_force), recomputing X instead of keeping any solver
history; the gradient of a complex tensor follows torch's convention
dS/dRe U + i dS/dIm U, which is what dwf_force returns.
"""
from __future__ import annotations

import torch

from . import dwf


class FermionAction(torch.autograd.Function):
    """S(U) for a fixed pseudofermion phi (canonical black half-field, complex128, cuda)."""

    @staticmethod
    def forward(ctx, U, phi, op):
        op.load_gauge(U.detach())
        S, stats = op.action(phi)
        ctx.op = op
        ctx.save_for_backward(U, phi)
        ctx.stats = stats
        return torch.tensor(S, dtype=torch.float64, device=phi.device)

    @staticmethod
    def backward(ctx, grad_out):
        U, phi = ctx.saved_tensors
        op = ctx.op
        op.load_gauge(U.detach())
        G = torch.empty_like(U)
        op.force(G, phi, None, projected=False)
        return grad_out * G, None, None


def fermion_action(U, phi, op):
    return FermionAction.apply(U, phi, op)
