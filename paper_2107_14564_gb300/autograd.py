"""torch.autograd.Function over the estimator: B(delta) per kept bin, with the hand-written
adjoint (bsp_grad) as its backward. Both directions run in the library's CUDA kernels."""
from __future__ import annotations

import torch

from .binding import Plan, bsp_grad, bsp_spectrum


class BispectrumFunction(torch.autograd.Function):
    """B_t(delta) for every kept bin of `plan` (FP32 or mixed plan); delta: [Ng]^3 float32 CUDA."""

    @staticmethod
    def forward(ctx, delta: torch.Tensor, plan: Plan):
        delta = delta.contiguous()
        spec = torch.empty(plan.spec_shape(), dtype=torch.complex64, device=delta.device)
        bsp_spectrum(plan.handle, delta, spec)
        b, _ = plan.estimate(spec, with_grid=False)
        ctx.plan = plan
        ctx.save_for_backward(spec)
        return b

    @staticmethod
    def backward(ctx, grad_b: torch.Tensor):
        (spec,) = ctx.saved_tensors
        plan = ctx.plan
        out = torch.empty((plan.ng,) * 3, dtype=torch.float32, device=spec.device)
        bsp_grad(plan.handle, spec, grad_b.to(torch.float64).contiguous(), out)
        return out, None


def bispectrum(delta: torch.Tensor, plan: Plan) -> torch.Tensor:
    """Differentiable per-bin bispectrum of a real field."""
    return BispectrumFunction.apply(delta, plan)
