"""alm2map as a differentiable PyTorch op.

The backward pass is the library's hand-written transpose
(``map2alm_adjoint``: ring analysis then Legendre accumulation), so for a real
loss the coefficient gradient follows PyTorch's convention for complex leaves,
dL/dRe(a) + i dL/dIm(a), with Im of the m = 0 entries zero (they do not enter
the real map).  With a BF16 tensor-core forward whose plan-time Lambda operand
is built, the transpose runs in the same form on the tensor cores; otherwise
in FP64.
"""
from __future__ import annotations

import torch

from . import sht


class SHTAlm2Map(torch.autograd.Function):
    @staticmethod
    def forward(ctx, alm: torch.Tensor, plan: "sht.Plan", prec: str = "fp64"):
        ctx.plan = plan
        ctx.prec = prec
        return plan.alm2map(alm, prec)

    @staticmethod
    def backward(ctx, grad_map: torch.Tensor):
        g = grad_map.contiguous()
        if ctx.prec in ("bf16x6_tc", "bf16x3_tc") and ctx.prec in ctx.plan.lambda_cached:
            return ctx.plan.map2alm_adjoint(g.float(), ctx.prec), None, None
        if g.dtype != torch.float64:
            g = g.double()  # the transpose runs in FP64
        return ctx.plan.map2alm_adjoint(g, "fp64"), None, None


def alm2map(alm: torch.Tensor, plan: "sht.Plan", prec: str = "fp64") -> torch.Tensor:
    """Differentiable alm2map of cuda complex128 coefficients ([B, nalm] or [nalm])."""
    return SHTAlm2Map.apply(alm, plan, prec)
