"""torch.autograd.Function over the fused fit + MHD right-hand side.

forward = phb_mhd_rhs (the requested precision); backward = phb_rhs_adjoint
(FP64, recomputing each factorisation), with the neighbour lists of the
plan's last build held fixed and lambda treated as a constant.
"""
from __future__ import annotations

import dataclasses

import torch

from .api import Params, Plan, mhd_rhs, rhs_adjoint


class PhbRHS(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pos: torch.Tensor, U: torch.Tensor, lam: torch.Tensor, plan: Plan,
                params: Params):
        dudt, _ = mhd_rhs(plan, params, pos.contiguous(), lam.contiguous(), U.contiguous())
        ctx.save_for_backward(pos, U, lam)
        ctx.plan = plan
        ctx.params = params
        return dudt

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        pos, U, lam = ctx.saved_tensors
        p64 = dataclasses.replace(ctx.params, precision="fp64")
        Ubar, xbar = rhs_adjoint(ctx.plan, p64, pos.contiguous(), lam.contiguous(), U.contiguous(),
                                 grad_out.contiguous())
        return xbar, Ubar, None, None, None


def rhs_autograd(pos, U, lam, plan: Plan, params: Params) -> torch.Tensor:
    """dU/dt [8, n] with gradients flowing to pos [3, n] and U [8, n]."""
    return PhbRHS.apply(pos, U, lam, plan, params)
