"""E(L) as a torch.autograd.Function over the CUDA library.

The LNV band energy E = 2 Tr[KH] with K = 3LSL - 2LSLSL (Eq. 3) is a cubic
function of the auxiliary density matrix L, whose minimisation the paper
describes (Sec. 2).  forward() evaluates E and N_e without the gradient
products; backward() asks the library for dE/dL, which recomputes the LS / LH
/ SLS / SLH / LSLS intermediates in the system's workspace instead of keeping
anything from the forward pass: the only saved tensor is L itself, and LSL or
LSLSL are never formed.  The gradient is the elementwise derivative with
respect to each stored block entry of L (block-CSR layout of L's pattern).
"""
from __future__ import annotations

import torch

from .lnv import System


class LNVEnergy(torch.autograd.Function):
    """E(L) (and N_e, not differentiated) for a fixed system, S and H."""

    @staticmethod
    def forward(ctx, L: torch.Tensor, system: System, S: torch.Tensor, H: torch.Tensor):
        out, _ = system.energy_grad(S, H, L.detach(), grad=False)
        ctx.system, ctx.S, ctx.H = system, S, H
        ctx.save_for_backward(L)
        E = out[0, 0].clone()
        Ne = out[0, 1].clone()
        ctx.mark_non_differentiable(Ne)
        return E, Ne

    @staticmethod
    def backward(ctx, gE: torch.Tensor, gNe: torch.Tensor):
        (L,) = ctx.saved_tensors
        gL = None
        if ctx.needs_input_grad[0]:
            _, G = ctx.system.energy_grad(ctx.S, ctx.H, L.detach(), grad=True)
            gL = (G.to(torch.float64) * gE.to(torch.float64)).to(L.dtype)
        return gL, None, None, None


def lnv_energy(L: torch.Tensor, system: System, S: torch.Tensor, H: torch.Tensor):
    """(E, N_e) with E differentiable with respect to L."""
    return LNVEnergy.apply(L, system, S, H)
