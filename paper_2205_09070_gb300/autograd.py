"""torch.autograd wrapper: ln L(h) as a differentiable function of the
hyperparameters, with the gradient from the library's adjoint kernels
(computed in the same call as the forward value and stashed for backward)."""

from __future__ import annotations

import torch

from .gpsparse import GP, Opts


class LogMarginalLikelihood(torch.autograd.Function):
    @staticmethod
    def forward(ctx, h: torch.Tensor, x, y, gp: GP, opts: Opts):
        hv = h.detach().to("cpu", torch.float64).numpy()
        lml, grad, _ = gp.lml_grad(x, y, hv, opts)
        ctx.save_for_backward(torch.as_tensor(grad, dtype=h.dtype, device=h.device))
        return torch.tensor(lml, dtype=h.dtype, device=h.device)

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return grad_out * g, None, None, None, None


def log_marginal_likelihood(h: torch.Tensor, x, y, gp: GP, opts: Opts) -> torch.Tensor:
    return LogMarginalLikelihood.apply(h, x, y, gp, opts)
