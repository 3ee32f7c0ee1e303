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


# ---------------------------------------------------------------------------
# Differentiating a Krylov solve preconditioned by M (right-preconditioned
# BiCGStab, Eq. 1.2): products with A and M are CSR products on the GPU
# (rsai_spmv); their adjoints are products with A^T and M^T (rsai_spmv on the
# CSC arrays read as the CSR of the transpose) and, for the stored values,
# rsai_spmv_grad_values.  The vector operations between products are torch's.


class Pattern:
    """The structure of a square CSR matrix and of its transpose, on the device:
    row_ptr/col_idx (CSR), col_ptr/row_idx (CSC = CSR of the transpose) and
    csc_to_csr, the CSR position of every CSC entry."""

    def __init__(self, row_ptr, col_idx, col_ptr, row_idx, csc_to_csr):
        self.row_ptr, self.col_idx = row_ptr.contiguous(), col_idx.contiguous()
        self.col_ptr, self.row_idx = col_ptr.contiguous(), row_idx.contiguous()
        self.csc_to_csr = csc_to_csr.contiguous()
        self.n = int(row_ptr.numel()) - 1

    @classmethod
    def of_matrix(cls, A, device="cuda") -> "Pattern":
        """From a SparseMatrix (host arrays, csc_to_csr included)."""
        import numpy as np

        t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a, dtype=dt)).to(device)  # noqa: E731
        return cls(t(A.row_ptr, np.int64), t(A.col_idx, np.int32), t(A.col_ptr, np.int64), t(A.row_idx, np.int32),
                   t(A.csc_to_csr, np.int64))

    @classmethod
    def of_M(cls, handle: "rsai.Handle") -> "Pattern":
        """M's pattern as built (rsai_get_M and rsai_get_M_csc)."""
        rp, ci, _ = handle.M()
        cp, ri, pos = handle.M_csc()
        return cls(rp, ci, cp, ri, pos)


class SpMV(torch.autograd.Function):
    """y = A x, differentiable in the stored values of A (CSR order) and in x."""

    @staticmethod
    def forward(ctx, val: torch.Tensor, x: torch.Tensor, pat: Pattern):
        val, x = val.contiguous(), x.contiguous()
        ctx.save_for_backward(val, x)
        ctx.pat = pat
        return rsai.spmv(pat.row_ptr, pat.col_idx, val, x)

    @staticmethod
    def backward(ctx, gy):
        val, x = ctx.saved_tensors
        pat = ctx.pat
        gy = gy.contiguous()
        gval = gx = None
        if ctx.needs_input_grad[0]:
            gval = rsai.spmv_grad_values(pat.row_ptr, pat.col_idx, gy, x)
        if ctx.needs_input_grad[1]:
            gx = rsai.spmv(pat.col_ptr, pat.row_idx, val[pat.csc_to_csr].contiguous(), gy)
        return gval, gx, None


def bicgstab_fixed(apply_op, b: torch.Tensor, iters: int) -> torch.Tensor:
    """``iters`` full iterations of BiCGStab on op(y) = b from y = 0, with no
    stopping test, so that the iterate is a smooth function of the operator
    (the same recurrences as ``rsai_bicgstab``: rhat = r0 = b)."""
    y = torch.zeros_like(b)
    r = b
    rhat = b.detach().clone()
    p = torch.zeros_like(b)
    v = torch.zeros_like(b)
    rho_old = alpha = omega = None
    for it in range(iters):
        rho = torch.dot(rhat, r)
        if it == 0:
            p = r
        else:
            beta = (rho / rho_old) * (alpha / omega)
            p = r + beta * (p - omega * v)
        v = apply_op(p)
        alpha = rho / torch.dot(rhat, v)
        s = r - alpha * v
        t = apply_op(s)
        omega = torch.dot(t, s) / torch.dot(t, t)
        y = y + alpha * p + omega * s
        r = s - omega * t
        rho_old = rho
    return y


def preconditioned_solve_loss(A_val: torch.Tensor, handle: "rsai.Handle", patA: Pattern, patM: Pattern,
                              b: torch.Tensor, iters: int = 20):
    """loss = ||b - A M y_iters||^2, y_iters from ``iters`` iterations of
    BiCGStab on A M y = b, with M = M(A) on the handle's frozen pattern.
    Differentiable in A_val (through A directly and through M)."""
    M_val, _ = frozen_rsai(A_val, handle)

    def AM(z):
        return SpMV.apply(A_val, SpMV.apply(M_val, z, patM), patA)

    y = bicgstab_fixed(AM, b, iters)
    res = b - AM(y)
    return torch.dot(res, res)
