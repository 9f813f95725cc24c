"""Differentiable solves: torch.autograd.Function wrappers over the C ABI.

The backward pass runs the adjoint solve A^T lambda = dL/dx through the
transposed hierarchy (amg_adjoint: coarse correction first, then the
transposed ILU(0) smoother), then
  dL/db = lambda,  dL/dA_ij = -lambda_i x_j on the sparsity pattern
(amg_csr_value_grad), or, for the finite-volume problem, the chain through
the harmonic-mean transmissibilities to per-cell log-conductivities
(amg_fv_grad_logk).  All arithmetic runs in the library's kernels.
"""
from __future__ import annotations

import torch

from . import (amg_adjoint, amg_csr_value_grad, amg_fv_grad_logk, amg_setup, amg_solve)
from .device import CsrDevice, assemble_fv


class AmgSolve(torch.autograd.Function):
    """x = A^{-1} b for CSR values `val` on a fixed pattern (row_ptr, col)."""

    @staticmethod
    def forward(ctx, val, b, row_ptr, col, tol=1e-10, opts=None):
        A = CsrDevice(int(b.numel()), row_ptr, col, val.detach().contiguous())
        h = amg_setup(A, opts, build_adjoint=1)
        x = torch.zeros_like(b)
        st = amg_solve(h, b.detach().contiguous(), x, tol)
        ctx.h, ctx.A, ctx.tol, ctx.stats = h, A, tol, st
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        lam = torch.zeros_like(x)
        amg_adjoint(ctx.h, gx.contiguous(), lam, ctx.tol)
        gval = torch.empty_like(ctx.A.val)
        amg_csr_value_grad(ctx.A, lam, x, gval)
        ctx.h.close()
        return gval, lam, None, None, None, None


class FvLogKappaSolve(torch.autograd.Function):
    """x(log kappa) for an isotropic block-kappa grid problem: assemble eq. (2)
    on the GPU from exp(log kappa), solve, and differentiate through the
    adjoint solve and the transmissibilities."""

    @staticmethod
    def forward(ctx, logk, prob, tol=1e-10, opts=None):
        import dataclasses
        k = torch.exp(logk.detach()).contiguous()
        kn = k.cpu().numpy()
        p = dataclasses.replace(prob, kx=kn, ky=kn, kz=kn)
        A, b = assemble_fv(p, device=logk.device)
        h = amg_setup(A, opts, build_adjoint=1)
        x = torch.zeros_like(b)
        st = amg_solve(h, b, x, tol)
        ctx.h, ctx.prob, ctx.k, ctx.tol, ctx.stats = h, prob, k, tol, st
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        lam = torch.zeros_like(x)
        amg_adjoint(ctx.h, gx.contiguous(), lam, ctx.tol)
        p, k = ctx.prob, ctx.k
        gs = [torch.zeros_like(x) for _ in range(3)]
        kz = k if p.dim == 3 else None
        amg_fv_grad_logk(p.dim, p.nx, p.ny, p.nz, k, k, kz, lam, x, gs[0], gs[1],
                         gs[2] if p.dim == 3 else None)
        g = gs[0] + gs[1] + (gs[2] if p.dim == 3 else 0)
        ctx.h.close()
        return g, None, None, None
