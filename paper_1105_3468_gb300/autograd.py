"""Differentiable solves: torch.autograd.Function wrappers over the C ABI.

The backward pass runs the adjoint solve A^T lambda = dL/dx through the
transposed hierarchy (amg_adjoint: coarse correction first, then the
transposed ILU(0) smoother), then
  dL/db = lambda,  dL/dA_ij = -lambda_i x_j on the sparsity pattern
(amg_csr_value_grad), or, for the finite-volume problem, the chain through
the harmonic-mean transmissibilities to per-cell log-conductivities
(amg_fv_grad_logk_iso).  All arithmetic runs in the library's kernels: the
binding only passes device buffers.

Handle lifetime: the hierarchy built in forward lives as long as the autograd
graph that holds it (it is released with the graph, or at once when no input
needs a gradient), so a second backward with retain_graph=True reuses it.
"""
from __future__ import annotations

import torch

from . import (amg_adjoint, amg_csr_value_grad, amg_fv_grad_logk_iso, amg_setup, amg_solve)
from .device import CsrDevice, assemble_fv_logk


def _keep_handle(ctx, h):
    if any(ctx.needs_input_grad):
        ctx.h = h
    else:
        h.close()
        ctx.h = None


def _handle(ctx):
    h = getattr(ctx, "h", None)
    if h is None or not h.ptr.value:
        raise RuntimeError("the hierarchy of this solve was released: no input required a gradient")
    return h


class AmgSolve(torch.autograd.Function):
    """x = A^{-1} b for CSR values `val` on a fixed pattern (row_ptr, col)."""

    @staticmethod
    def forward(ctx, val, b, row_ptr, col, tol=1e-10, opts=None):
        A = CsrDevice(int(b.numel()), row_ptr, col, val.detach().contiguous())
        h = amg_setup(A, opts, build_adjoint=1)
        x = torch.zeros_like(b)
        st = amg_solve(h, b.detach().contiguous(), x, tol)
        ctx.A, ctx.tol, ctx.stats = A, tol, st
        _keep_handle(ctx, h)
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        lam = torch.zeros_like(x)
        amg_adjoint(_handle(ctx), gx.contiguous(), lam, ctx.tol)
        gval = torch.empty_like(ctx.A.val)
        amg_csr_value_grad(ctx.A, lam, x, gval)
        return gval, lam, None, None, None, None


class FvLogKappaSolve(torch.autograd.Function):
    """x(log kappa) for an isotropic grid problem: kappa = exp(log kappa) and
    the assembly of eq. (2) on the GPU (amg_fv_assemble_logk), the solve, and
    the derivative through the adjoint solve and the transmissibilities
    (amg_fv_grad_logk_iso)."""

    @staticmethod
    def forward(ctx, logk, prob, tol=1e-10, opts=None):
        A, b, kappa = assemble_fv_logk(prob, logk)
        h = amg_setup(A, opts, build_adjoint=1)
        x = torch.zeros_like(b)
        st = amg_solve(h, b, x, tol)
        ctx.prob, ctx.kappa, ctx.tol, ctx.stats = prob, kappa, tol, st
        _keep_handle(ctx, h)
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        lam = torch.zeros_like(x)
        amg_adjoint(_handle(ctx), gx.contiguous(), lam, ctx.tol)
        p = ctx.prob
        g = torch.empty_like(x)
        amg_fv_grad_logk_iso(p.dim, p.nx, p.ny, p.nz, ctx.kappa, lam, x, g)
        return g, None, None, None
