"""Device-memory conveniences over the C ABI (torch tensors as buffers).

Nothing here computes: tensors are allocated with torch and handed to the
library's entry points.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np


@dataclasses.dataclass
class CsrDevice:
    """CSR arrays on the GPU: int64 row pointers, int32 columns, FP64 values."""

    n: int
    row_ptr: "object"
    col: "object"
    val: "object"

    @property
    def nnz(self) -> int:
        return int(self.col.numel())

    @staticmethod
    def from_host(A, device="cuda") -> "CsrDevice":
        import torch
        return CsrDevice(int(A.n),
                         torch.as_tensor(np.ascontiguousarray(A.row_ptr, dtype=np.int64)).to(device),
                         torch.as_tensor(np.ascontiguousarray(A.col, dtype=np.int32)).to(device),
                         torch.as_tensor(np.ascontiguousarray(A.val, dtype=np.float64)).to(device))


def assemble_fv(prob, device="cuda"):
    """Assemble eq. (2) on the GPU (amg_fv_assemble) from a GridProblem."""
    import torch
    from . import amg_fv_assemble

    def dev(a):
        return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).to(device)

    N = prob.nx * prob.ny * prob.nz
    cap = (2 * prob.dim + 1) * N
    rp = torch.empty(N + 1, dtype=torch.int64, device=device)
    ci = torch.empty(cap, dtype=torch.int32, device=device)
    v = torch.empty(cap, dtype=torch.float64, device=device)
    b = torch.empty(N, dtype=torch.float64, device=device)
    kz = dev(prob.kz) if prob.dim == 3 else None
    fz = dev(prob.fz) if prob.dim == 3 else None
    kx, ky, fx, fy, f = dev(prob.kx), dev(prob.ky), dev(prob.fx), dev(prob.fy), dev(prob.f)
    nnz = amg_fv_assemble(prob.dim, prob.nx, prob.ny, prob.nz, kx, ky, kz, fx, fy, fz, f, rp, ci, v, b)
    return CsrDevice(N, rp, ci[:nnz].clone(), v[:nnz].clone()), b


def assemble_fv_logk(prob, logk):
    """Assemble eq. (2) on the GPU for an isotropic conductivity given as the
    device tensor `logk` (amg_fv_assemble_logk: exp and assembly in the
    library); the grid, fluxes and source come from `prob`.  Returns
    (A, b, kappa) with kappa = exp(logk) on the device."""
    import torch
    from . import amg_fv_assemble_logk
    device = logk.device

    def dev(a):
        return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).to(device)

    N = prob.nx * prob.ny * prob.nz
    cap = (2 * prob.dim + 1) * N
    rp = torch.empty(N + 1, dtype=torch.int64, device=device)
    ci = torch.empty(cap, dtype=torch.int32, device=device)
    v = torch.empty(cap, dtype=torch.float64, device=device)
    b = torch.empty(N, dtype=torch.float64, device=device)
    kappa = torch.empty(N, dtype=torch.float64, device=device)
    fz = dev(prob.fz) if prob.dim == 3 else None
    lk = logk.detach().to(torch.float64).contiguous()
    nnz = amg_fv_assemble_logk(prob.dim, prob.nx, prob.ny, prob.nz, lk, kappa, dev(prob.fx), dev(prob.fy), fz,
                               dev(prob.f), rp, ci, v, b)
    return CsrDevice(N, rp, ci[:nnz].clone(), v[:nnz].clone()), b, kappa


def solve(A, b, x0=None, tol: float = 1e-8, opts=None, **overrides):
    """Set up and solve A x = b once; returns (x, stats, history)."""
    import torch
    from . import amg_get_history, amg_setup, amg_solve
    x = torch.zeros_like(b) if x0 is None else x0.clone()
    h = amg_setup(A, opts, **overrides)
    try:
        st = amg_solve(h, b, x, tol)
        hist = amg_get_history(h)
    finally:
        h.close()
    return x, st, hist
