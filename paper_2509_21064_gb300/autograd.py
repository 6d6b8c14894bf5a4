"""``torch.autograd.Function`` over PDBO's Lagrangian (section 3.1), backed by libsbo.

Forward returns ``L_r = 1/2 x_r^T A x_r + c'^T x_r + sum_i y_ri (x_ri^2 - x_ri)`` for every row
r of X, Y.  Backward calls the fused adjoint kernel again: it recomputes ``A x`` (nothing is
stored between forward and backward but X and Y) and writes ``gout_r * dL/dx`` and
``gout_r * dL/dy`` directly, the same epilogue arithmetic the GDA loop applies.
"""
from __future__ import annotations

import torch

from . import sbo as _sbo


def _stream():
    return torch.cuda.current_stream().cuda_stream


class GdaLagrangian(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X: torch.Tensor, Y: torch.Tensor, problem: "_sbo.Problem"):
        if not (X.is_cuda and Y.is_cuda) or X.dtype != torch.float32 or Y.dtype != torch.float32:
            raise TypeError("X and Y must be float32 CUDA tensors")
        X = X.contiguous()
        Y = Y.contiguous()
        B, n = X.shape
        if Y.shape != X.shape or n != problem.n:
            raise ValueError("X and Y must be [B, n] with the problem's n")
        L = torch.empty(B, device=X.device, dtype=torch.float32)
        _sbo.sbo_lagrangian(problem.h, B, X.data_ptr(), Y.data_ptr(), None, L.data_ptr(), None, None, _stream())
        ctx.save_for_backward(X, Y)
        ctx.problem = problem
        return L

    @staticmethod
    def backward(ctx, gL: torch.Tensor):
        X, Y = ctx.saved_tensors
        B = X.shape[0]
        gL = gL.contiguous().to(torch.float32)
        need_x, need_y = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        GX = torch.empty_like(X) if need_x else None
        GY = torch.empty_like(Y) if need_y else None
        if need_x or need_y:
            _sbo.sbo_lagrangian(ctx.problem.h, B, X.data_ptr(), Y.data_ptr(), gL.data_ptr(), None,
                                GX.data_ptr() if need_x else None, GY.data_ptr() if need_y else None, _stream())
        return GX, GY, None


def lagrangian(X: torch.Tensor, Y: torch.Tensor, problem: "_sbo.Problem") -> torch.Tensor:
    """Per-restart Lagrangian values with autograd support (see :class:`GdaLagrangian`)."""
    return GdaLagrangian.apply(X, Y, problem)
