"""torch.autograd wrapper of the ILT loss (litho_ilt_grad).

The library computes the loss and its adjoint gradient in one call (the
adjoint reuses the forward pass's stage-1 fields), so the Function's forward
runs both and keeps dL/dtheta; backward only scales it by the incoming
gradient of the per-clip losses.
"""
from __future__ import annotations

import torch

from . import litho as L


class IltLoss(torch.autograd.Function):
    """loss[b] = sum_f sum_x (sigmoid(resist_steep (g (x) I_f(sigmoid(mask_steep theta)) - threshold)) - target)^2."""

    @staticmethod
    def forward(ctx, theta, target, kernels, dose=1.0, mask_steep=4.0, resist_steep=25.0, threshold=0.3,
                sigma_nm=10.0, workspace=None):
        th = theta.detach().contiguous()
        grad, loss = L.litho_ilt_grad(kernels, th, target.contiguous(), dose=dose, mask_steep=mask_steep,
                                      resist_steep=resist_steep, threshold=threshold, sigma_nm=sigma_nm,
                                      workspace=workspace)
        ctx.save_for_backward(grad)
        return torch.as_tensor(loss, dtype=torch.float64, device=theta.device)

    @staticmethod
    def backward(ctx, grad_loss):
        (grad,) = ctx.saved_tensors
        g = grad * grad_loss.to(grad.dtype).view(-1, 1, 1)
        return g, None, None, None, None, None, None, None, None


def ilt_loss(theta, target, kernels, **kw):
    return IltLoss.apply(theta, target, kernels, kw.get("dose", 1.0), kw.get("mask_steep", 4.0),
                         kw.get("resist_steep", 25.0), kw.get("threshold", 0.3), kw.get("sigma_nm", 10.0),
                         kw.get("workspace"))
