"""torch.autograd wrappers: the forward projection W and the back projection W^T.

The gradient of x -> W x is the library's W^T kernel (csm_back); the gradient of
p -> W^T p is the forward kernel W, so second derivatives also run on the same kernels.
Because both kernels evaluate the same entries, the pair is an exact adjoint up to
floating-point summation order (the paper's adjoint-mismatch check, Section "Numerical
Experiments").
"""
from __future__ import annotations

import torch

from .projector import Projector


class ProjectFn(torch.autograd.Function):
    """p = W x  (x: [B, *vol_shape] or vol_shape)."""

    @staticmethod
    def forward(ctx, x: torch.Tensor, projector: Projector) -> torch.Tensor:
        ctx.projector = projector
        return projector.forward(x.contiguous())

    @staticmethod
    def backward(ctx, grad_p: torch.Tensor):
        return BackProjectFn.apply(grad_p.contiguous(), ctx.projector), None


class BackProjectFn(torch.autograd.Function):
    """x = W^T p  (p: [B, *sino_shape] or sino_shape)."""

    @staticmethod
    def forward(ctx, p: torch.Tensor, projector: Projector) -> torch.Tensor:
        ctx.projector = projector
        return projector.back(p.contiguous())

    @staticmethod
    def backward(ctx, grad_x: torch.Tensor):
        return ProjectFn.apply(grad_x.contiguous(), ctx.projector), None


def project(x: torch.Tensor, projector: Projector) -> torch.Tensor:
    return ProjectFn.apply(x, projector)


def backproject(p: torch.Tensor, projector: Projector) -> torch.Tensor:
    return BackProjectFn.apply(p, projector)
