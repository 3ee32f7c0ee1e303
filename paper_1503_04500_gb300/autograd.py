"""Differentiation through the frozen-pattern RSAI solves (torch.autograd.Function).

The pattern of M is chosen by discrete steps (dominant rows, drops) and is not
differentiated.  On a frozen pattern J_k every column is the LS solution
m_k = argmin ||A(:,J_k) x - e_k|| (Eq. 2.3), a smooth function of the values of
A; the forward is ``rsai_refit`` and the backward is the hand-written adjoint
``rsai_backward`` (both CUDA kernels behind the C ABI).
"""
from __future__ import annotations

import torch

from . import rsai


class FrozenRSAI(torch.autograd.Function):
    """(values of A) -> (values of M in CSR order, ||r_k||^2) on a built pattern."""

    @staticmethod
    def forward(ctx, A_val: torch.Tensor, handle: "rsai.Handle"):
        A_val = A_val.contiguous()
        M_val, rho2 = handle.refit(A_val)
        ctx.handle = handle
        ctx.save_for_backward(A_val)
        return M_val, rho2

    @staticmethod
    def backward(ctx, grad_M, grad_rho2):
        (A_val,) = ctx.saved_tensors
        h = ctx.handle
        if grad_M is None:
            nnz = h.stats()["nnz_M"]
            grad_M = torch.zeros(max(nnz, 1), dtype=torch.float64, device=A_val.device)
        grad_M = grad_M.contiguous()
        if grad_rho2 is not None:
            grad_rho2 = grad_rho2.contiguous()
        return h.backward(A_val, grad_M, grad_rho2), None


def frozen_rsai(A_val: torch.Tensor, handle: "rsai.Handle"):
    """M values (CSR order of ``handle``'s M) and rho_k^2 as differentiable functions of A_val."""
    return FrozenRSAI.apply(A_val, handle)
