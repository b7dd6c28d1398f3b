"""Differentiable codebook refinement: the soft-assignment PQ reconstruction loss.

For rows X [N][D] and codebooks C [M][Ks][Ds] with temperature tau,

    p_{n,m,k} = softmax_k(-||x_{n,m} - c_{m,k}||^2 / tau)
    L         = (1/N) sum_n sum_m || sum_k p_{n,m,k} c_{m,k} - x_{n,m} ||^2

is a smooth relaxation of the hard PQ assignment of Sec. 2.1 (tau -> 0 gives
the hard reconstruction error).  Forward and backward are CUDA kernels behind
the C ABI (``softpq_forward`` / ``softpq_backward``); the backward recomputes
the soft assignments instead of keeping them from the forward pass, so the
only saved tensors are the inputs.
"""
from __future__ import annotations

import torch

from . import pqgb


class SoftPQLoss(torch.autograd.Function):
    """L(X, C; tau) with gradients with respect to X and C."""

    @staticmethod
    def forward(ctx, X: torch.Tensor, codebooks: torch.Tensor, tau: float):
        ctx.save_for_backward(X, codebooks)
        ctx.tau = float(tau)
        return pqgb.softpq_forward(X, codebooks, tau)

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        X, codebooks = ctx.saved_tensors
        need_dx = ctx.needs_input_grad[0]
        g = grad_out if grad_out.dtype == torch.float32 and grad_out.is_contiguous() else None
        if g is None:
            raise TypeError("SoftPQLoss expects a float32 upstream gradient")
        dC, dX = pqgb.softpq_backward(X, codebooks, ctx.tau, grad_loss=g, need_dx=need_dx)
        return dX, (dC if ctx.needs_input_grad[1] else None), None


def softpq_loss(X: torch.Tensor, codebooks: torch.Tensor, tau: float) -> torch.Tensor:
    """Soft-assignment reconstruction loss (device float32 scalar), differentiable in X and codebooks."""
    return SoftPQLoss.apply(X, codebooks, tau)


def refine(X: torch.Tensor, codebooks: torch.Tensor, tau: float, steps: int, lr: float) -> torch.Tensor:
    """Plain gradient descent on the codebooks for ``steps`` steps; returns the refined codebooks."""
    C = codebooks.detach().clone().requires_grad_(True)
    for _ in range(steps):
        loss = softpq_loss(X, C, tau)
        (g,) = torch.autograd.grad(loss, C)
        with torch.no_grad():
            C -= lr * g
    return C.detach()
