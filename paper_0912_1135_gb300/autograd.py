"""The null-space projection as a differentiable operation (a projection layer).

``NullProject.apply(A, B, projector)`` returns Z = rows of Zb for the rows b of B, where
the projector is a preconditioned :class:`Projector` bound to A. Its backward pass is the
adjoint of Eq. 1 (rtproj_grad_A in include/rtproj.h): for an upstream gradient G (rows
g_j),
    dL/dB = Z G                                  (Z is symmetric),
    dL/dA = -(H^* (Z G) + W^* Z B),               H = lstsq(B), W = lstsq(G) (Remark 4.1),
computed by one apply of the projector to G (null space and least squares together) and
one tensor-core rank-2k product. Everything runs in librtproj's kernels.
"""
from __future__ import annotations

import torch

from . import Projector

__all__ = ["NullProject", "null_project"]


class NullProject(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A: torch.Tensor, B: torch.Tensor, projector: Projector):
        if projector.A.data_ptr() != A.data_ptr():
            raise ValueError("the projector must be bound to A")
        Z, _, H = projector.project(B.detach(), null=True, lstsq=True)
        ctx.projector = projector
        ctx.save_for_backward(Z, H)
        return Z

    @staticmethod
    def backward(ctx, G: torch.Tensor):
        P: Projector = ctx.projector
        Z, H = ctx.saved_tensors
        G = G.contiguous()
        need_a, need_b = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        Y, _, W = P.project(G, null=True, lstsq=need_a)           # Z g_j and w_j = lstsq(g_j)
        dA = P.grad_A(H, Y, W, Z) if need_a else None
        return dA, (Y if need_b else None), None


def null_project(A: torch.Tensor, B: torch.Tensor, seed: int = 1, l: int | None = None, **kw) -> torch.Tensor:
    """Z B^* rows for a fresh preconditioner of A (sketch seed, size l), differentiable in
    A and B. kw: Projector options (mode, omega, slices ...)."""
    k = B.shape[0] if B.dim() == 2 else 1
    P = Projector(A.detach(), l_max=l, k_max=k, **kw)
    P.precondition(seed, l)
    return NullProject.apply(A, B, P)
