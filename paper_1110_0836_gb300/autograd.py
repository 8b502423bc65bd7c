"""torch.autograd.Function over the fused fit + MHD right-hand side.

forward = phb_mhd_rhs (the requested precision); backward = phb_rhs_adjoint
(FP64), with the neighbour lists of the plan's last build held fixed and
lambda treated as a constant.  By default the backward pass recomputes each
particle's factorisation; with store_factors=True the forward pass also
records the FP64 factors and coefficients (343 doubles per particle) and the
backward pass starts from that record (phb_rhs_adjoint_stored).
"""
from __future__ import annotations

import dataclasses

import torch

from .api import Params, Plan, adjoint_record, mhd_rhs, rhs_adjoint, rhs_adjoint_stored


class PhbRHS(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pos: torch.Tensor, U: torch.Tensor, lam: torch.Tensor, plan: Plan,
                params: Params, store_factors: bool = False):
        pos, U, lam = pos.contiguous(), U.contiguous(), lam.contiguous()
        dudt, _ = mhd_rhs(plan, params, pos, lam, U)
        ctx.plan = plan
        ctx.params = params
        ctx.record = None
        if store_factors:
            ctx.record = adjoint_record(plan, dataclasses.replace(params, precision="fp64"),
                                        pos, lam, U)
        ctx.save_for_backward(pos, U, lam)
        return dudt

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        pos, U, lam = ctx.saved_tensors
        p64 = dataclasses.replace(ctx.params, precision="fp64")
        if ctx.record is not None:
            Ubar, xbar = rhs_adjoint_stored(ctx.plan, p64, pos, lam, U, grad_out.contiguous(),
                                            ctx.record)
            ctx.record = None
        else:
            Ubar, xbar = rhs_adjoint(ctx.plan, p64, pos, lam, U, grad_out.contiguous())
        return xbar, Ubar, None, None, None, None


def rhs_autograd(pos, U, lam, plan: Plan, params: Params, store_factors: bool = False) -> torch.Tensor:
    """dU/dt [8, n] with gradients flowing to pos [3, n] and U [8, n]."""
    return PhbRHS.apply(pos, U, lam, plan, params, store_factors)
