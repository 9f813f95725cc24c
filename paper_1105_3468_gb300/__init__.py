"""GB300 matching-aggregation AMG as the preconditioner of FGMRES.

Python binding of libamg_gb (C ABI in include/amg.h); every entry point keeps
the C name and only marshals arguments (tensors or arrays -> pointers).  The
arithmetic runs in the library's CUDA kernels; if the library is missing the
calls raise instead of falling back to anything else.

Arrays may be torch tensors (CUDA or CPU) or numpy arrays; CUDA tensors are
used in place, host arrays are copied by the library.
"""
from __future__ import annotations

import ctypes as C
from typing import Optional

import numpy as np

from . import _lib
from ._lib import (AMG_NOALLOC_MAX_ROWS, AMG_LOOP_DEVICE, AMG_LOOP_HOST, AMG_MATCH_PLAIN, AMG_MATCH_SCALED, AMG_COARSE_ILUT, AMG_COARSE_RECURSIVE, AMG_ORTHO_CGS2, AMG_ORTHO_MGS, AMG_BF16, AMG_BF16_ALL, AMG_COLOR_FIRST_FIT, AMG_COLOR_HASH_JP, AMG_ERR_BREAKDOWN,  # noqa: F401
                   AMG_ERR_CUDA, AMG_ERR_INVALID_ARG, AMG_ERR_LIMIT, AMG_ERR_NOT_CONVERGED,
                   AMG_ERR_NOT_SUPPORTED, AMG_ERR_NUMERIC, AMG_ERR_OOM, AMG_FP32, AMG_FP64, AMG_OK,
                   AMG_ORDER_COLOR, AMG_ORDER_NATURAL, AmgCsr, AmgOptions, AmgStats)

__all__ = [
    "AmgError", "Handle", "amg_default_options", "amg_setup", "amg_destroy", "amg_solve",
    "amg_adjoint", "amg_get_history", "amg_precond_apply", "amg_spmv", "amg_get_level_info",
    "amg_get_tile_grid", "amg_get_sweep_kind",
    "amg_num_levels", "amg_get_aggregates", "amg_get_matrix", "amg_get_pass_matrix",
    "amg_get_colors", "amg_get_ilu", "amg_fv_assemble", "amg_fv_grad_logk", "amg_fv_assemble_logk",
    "amg_fv_grad_logk_iso", "amg_version",
    "amg_status_string", "lib", "amg_set_kernel_timing", "amg_get_kernel_timing",
    "amg_launch_counter", "amg_csr_value_grad", "amg_spmv_noalloc", "amg_setup_batched",
    "amg_solve_batched", "amg_batch_size", "amg_batch_member", "amg_get_spmv_config",
    "amg_update_values", "amg_ilut_host",
]


def lib():
    return _lib.load()


class AmgError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = lib().amg_last_error().decode(errors="replace")
        text = lib().amg_status_string(status).decode()
        super().__init__(f"{where}: {text} ({status}): {msg}")
        self.status = status


def _check(st: int, where: str, allow=(AMG_OK,)):
    if st not in allow:
        raise AmgError(st, where)
    return st


def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _ptr(a, dtype=None):
    """Pointer of a contiguous tensor/array (None -> NULL)."""
    if a is None:
        return None
    if _is_torch(a):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if dtype is not None and str(a.dtype) != f"torch.{dtype}":
            raise TypeError(f"expected {dtype}, got {a.dtype}")
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        if dtype is not None and a.dtype != np.dtype(dtype):
            raise TypeError(f"expected {dtype}, got {a.dtype}")
        return a.ctypes.data
    raise TypeError(f"unsupported array type {type(a)}")


def _stream_of(*arrays):
    for a in arrays:
        if a is not None and _is_torch(a) and a.is_cuda:
            import torch
            return torch.cuda.current_stream(a.device).cuda_stream
    return None


def _csr(A) -> AmgCsr:
    s = AmgCsr()
    s.n = int(A.n)
    s.nnz = int(A.row_ptr[-1])
    s.row_ptr = _ptr(A.row_ptr, "int64")
    s.col = _ptr(A.col, "int32")
    s.val = _ptr(A.val, "float64")
    return s


def amg_version() -> str:
    return lib().amg_version().decode()


def amg_status_string(st: int) -> str:
    return lib().amg_status_string(st).decode()


def _set_option(o: AmgOptions, k: str, v):
    if not hasattr(o, k):
        raise KeyError(k)
    setattr(o, k, float(v) if k == "ilut_tau" else int(v))


def amg_default_options(**overrides) -> AmgOptions:
    o = AmgOptions()
    _check(lib().amg_default_options(C.byref(o)), "amg_default_options")
    for k, v in overrides.items():
        _set_option(o, k, v)
    return o


class Handle:
    """Owns an amg_handle_t; destroyed with amg_destroy."""

    def __init__(self, ptr: int, n: int, opts: AmgOptions, keep=()):
        self.ptr = C.c_void_p(ptr)
        self.n = n
        self.opts = opts
        self._keep = keep      # keeps the stream's owner alive

    def close(self):
        if self.ptr and self.ptr.value:
            lib().amg_destroy(self.ptr)
            self.ptr = C.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def amg_setup(A, opts: Optional[AmgOptions] = None, stream=None, **overrides) -> Handle:
    """amg_setup: build the hierarchy of A (object with n, row_ptr, col, val)."""
    o = opts if opts is not None else amg_default_options()
    for k, v in overrides.items():
        _set_option(o, k, v)
    cs = _csr(A)
    if stream is None:
        stream = _stream_of(A.row_ptr, A.val)
    out = C.c_void_p()
    _check(lib().amg_setup(C.byref(cs), C.byref(o), stream, C.byref(out)), "amg_setup")
    return Handle(out.value, cs.n, o)


def amg_destroy(h: Handle):
    h.close()


def amg_update_values(h: Handle, val):
    """amg_update_values: new values on the same pattern; aggregates kept."""
    _check(lib().amg_update_values(h.ptr, _ptr(val, "float64")), "amg_update_values")


def amg_ilut_host(row_ptr, col, val, tau: float):
    """amg_ilut_host: ILUT(tau) factors of a host CSR matrix (numpy arrays:
    int64 row pointers, int32 columns, float64 values).  Returns
    (row_ptr, col, val, status) of the factor CSR, row i holding its L~ part
    (unit diagonal implied) then its U~ part; status is AMG_OK or
    AMG_ERR_BREAKDOWN."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(col, dtype=np.int32)
    v = np.ascontiguousarray(val, dtype=np.float64)
    n = len(rp) - 1
    frp = np.zeros(n + 1, np.int64)
    cap = max(1, 2 * len(ci))
    for _ in range(2):
        fci = np.zeros(cap, np.int32)
        fv = np.zeros(cap, np.float64)
        nnz = C.c_int64(0)
        st = lib().amg_ilut_host(n, _ptr(rp), _ptr(ci), _ptr(v), float(tau), cap, _ptr(frp), _ptr(fci),
                                 _ptr(fv), C.byref(nnz))
        if st != AMG_ERR_LIMIT:
            break
        cap = int(nnz.value)
    _check(st, "amg_ilut_host", (AMG_OK, AMG_ERR_BREAKDOWN))
    return frp, fci[:nnz.value].copy(), fv[:nnz.value].copy(), st


def amg_solve(h: Handle, b, x, tol: float = 1e-8, allow_not_converged: bool = True) -> AmgStats:
    """amg_solve: x (in: initial guess, out: solution) for A x = b."""
    st = AmgStats()
    allow = (AMG_OK, AMG_ERR_NOT_CONVERGED) if allow_not_converged else (AMG_OK,)
    _check(lib().amg_solve(h.ptr, _ptr(b, "float64"), _ptr(x, "float64"), float(tol), C.byref(st)),
           "amg_solve", allow)
    return st


def amg_adjoint(h: Handle, g, lam, tol: float = 1e-8, allow_not_converged: bool = True) -> AmgStats:
    """amg_adjoint: lam (in: initial guess, out: solution) for A^T lam = g."""
    st = AmgStats()
    allow = (AMG_OK, AMG_ERR_NOT_CONVERGED) if allow_not_converged else (AMG_OK,)
    _check(lib().amg_adjoint(h.ptr, _ptr(g, "float64"), _ptr(lam, "float64"), float(tol), C.byref(st)),
           "amg_adjoint", allow)
    return st


def amg_setup_batched(systems, opts: Optional[AmgOptions] = None, stream=None, **overrides) -> Handle:
    """amg_setup_batched: one hierarchy per system (list of CSR objects)."""
    o = opts if opts is not None else amg_default_options()
    for k, v in overrides.items():
        _set_option(o, k, v)
    arr = (AmgCsr * len(systems))(*[_csr(A) for A in systems])
    if stream is None:
        stream = _stream_of(systems[0].row_ptr)
    out = C.c_void_p()
    _check(lib().amg_setup_batched(arr, len(systems), C.byref(o), stream, C.byref(out)), "amg_setup_batched")
    return Handle(out.value, sum(int(A.n) for A in systems), o, keep=(arr,))


def amg_batch_size(h: Handle):
    """(count, row offsets [count+1]) of a batched handle."""
    c = C.c_int32(0)
    _check(lib().amg_batch_size(h.ptr, C.byref(c), None), "amg_batch_size")
    offs = np.zeros(c.value + 1, np.int64)
    _check(lib().amg_batch_size(h.ptr, C.byref(c), offs.ctypes.data), "amg_batch_size")
    return c.value, offs


def amg_batch_member(h: Handle, k: int) -> Handle:
    """Non-owning view of system k's handle (valid while the batch lives)."""
    p = lib().amg_batch_member(h.ptr, k)
    if not p:
        raise IndexError(k)
    v = Handle(p, 0, h.opts)
    v.close = lambda: None
    return v


def amg_solve_batched(h: Handle, b_cat, x_cat, tol: float = 1e-8):
    """amg_solve_batched: returns the per-system stats list."""
    count, _ = amg_batch_size(h)
    stats = (AmgStats * count)()
    _check(lib().amg_solve_batched(h.ptr, _ptr(b_cat, "float64"), _ptr(x_cat, "float64"), float(tol), stats),
           "amg_solve_batched", (AMG_OK, AMG_ERR_NOT_CONVERGED))
    return list(stats)


def amg_get_history(h: Handle) -> np.ndarray:
    n = C.c_int32(0)
    _check(lib().amg_get_history(h.ptr, None, 0, C.byref(n)), "amg_get_history")
    out = np.zeros(max(1, n.value))
    _check(lib().amg_get_history(h.ptr, out.ctypes.data, n.value, C.byref(n)), "amg_get_history")
    return out[:n.value]


def amg_precond_apply(h: Handle, z, q, transpose: bool = False):
    _check(lib().amg_precond_apply(h.ptr, _ptr(z, "float64"), _ptr(q, "float64"), int(transpose)),
           "amg_precond_apply")


def amg_spmv(A, x, y, stream=None):
    cs = _csr(A)
    if stream is None:
        stream = _stream_of(x)
    _check(lib().amg_spmv(C.byref(cs), _ptr(x, "float64"), _ptr(y, "float64"), stream), "amg_spmv")


def amg_spmv_noalloc(A, x, y, stream=None):
    """amg_spmv without any device allocation: its scratch is a fixed device
    array shared by all calls (at most AMG_NOALLOC_MAX_ROWS rows; calls that
    overlap on the GPU race on it)."""
    cs = _csr(A)
    if stream is None:
        stream = _stream_of(x)
    _check(lib().amg_spmv_noalloc(C.byref(cs), _ptr(x, "float64"), _ptr(y, "float64"), stream),
           "amg_spmv_noalloc")


def amg_set_kernel_timing(h: Handle, kclass: int):
    _check(lib().amg_set_kernel_timing(h.ptr, kclass), "amg_set_kernel_timing")


def amg_get_kernel_timing(h: Handle):
    """(total ms, timed launches, algorithmic bytes) of the timed kernel class."""
    ms, n, by = C.c_double(0), C.c_int64(0), C.c_double(0)
    _check(lib().amg_get_kernel_timing(h.ptr, C.byref(ms), C.byref(n), C.byref(by)), "amg_get_kernel_timing")
    return ms.value, n.value, by.value


def amg_launch_counter() -> int:
    return int(lib().amg_launch_counter())


def amg_get_spmv_config(h: Handle):
    """amg_get_spmv_config: (threads per block, unroll) of the outer SpMV."""
    blk, unr = C.c_int32(), C.c_int32()
    _check(lib().amg_get_spmv_config(h.ptr, C.byref(blk), C.byref(unr)), "amg_get_spmv_config")
    return blk.value, unr.value


def amg_num_levels(h: Handle) -> int:
    n = C.c_int32(0)
    _check(lib().amg_num_levels(h.ptr, C.byref(n)), "amg_num_levels")
    return n.value


def amg_get_level_info(h: Handle, level: int) -> dict:
    info = np.zeros(8, np.int64)
    _check(lib().amg_get_level_info(h.ptr, level, info.ctypes.data), "amg_get_level_info")
    keys = ["n", "nnz", "fwd_levels", "dense", "n_pass1", "n_next", "ncol", "bwd_levels"]
    return {k: int(v) for k, v in zip(keys, info)}


def amg_get_tile_grid(h: Handle) -> dict:
    """The finest level's grid tiling (persistent = 5): tiled, grid, tile extents, tile count."""
    info = np.zeros(8, np.int64)
    _check(lib().amg_get_tile_grid(h.ptr, info.ctypes.data), "amg_get_tile_grid")
    return {"tiled": bool(info[0]), "grid": tuple(int(v) for v in info[1:4]),
            "tile": tuple(int(v) for v in info[4:7]), "ntiles": int(info[7])}


SWEEP_KINDS = ("levels", "block", "cluster_grid", "grid", "dsm_replicated", "dataflow", "tiles")


def amg_get_sweep_kind(h: Handle, level: int) -> tuple:
    """The smoother variant of the level's last application (forward, transposed); None if not applied."""
    k = np.zeros(2, np.int32)
    _check(lib().amg_get_sweep_kind(h.ptr, level, k.ctypes.data), "amg_get_sweep_kind")
    return tuple(SWEEP_KINDS[v] if v >= 0 else None for v in k)


def amg_get_aggregates(h: Handle, level: int, pass_: int = 0) -> np.ndarray:
    info = amg_get_level_info(h, level)
    if pass_ <= 1:
        n = info["n"]
    else:
        n = amg_get_pass_matrix_info(h, level, pass_ - 1)[0]
    out = np.zeros(n, np.int32)
    _check(lib().amg_get_aggregates(h.ptr, level, pass_, out.ctypes.data), "amg_get_aggregates")
    return out


def amg_get_matrix(h: Handle, level: int):
    info = amg_get_level_info(h, level)
    rp = np.zeros(info["n"] + 1, np.int64)
    ci = np.zeros(max(1, info["nnz"]), np.int32)
    v = np.zeros(max(1, info["nnz"]))
    _check(lib().amg_get_matrix(h.ptr, level, rp.ctypes.data, ci.ctypes.data, v.ctypes.data), "amg_get_matrix")
    return rp, ci[:info["nnz"]], v[:info["nnz"]]


def amg_get_pass_matrix_info(h: Handle, level: int, pass_: int):
    info = np.zeros(2, np.int64)
    _check(lib().amg_get_pass_matrix(h.ptr, level, pass_, info.ctypes.data, None, None, None),
           "amg_get_pass_matrix")
    return int(info[0]), int(info[1])


def amg_get_pass_matrix(h: Handle, level: int, pass_: int):
    n, nnz = amg_get_pass_matrix_info(h, level, pass_)
    rp = np.zeros(n + 1, np.int64)
    ci = np.zeros(max(1, nnz), np.int32)
    v = np.zeros(max(1, nnz))
    _check(lib().amg_get_pass_matrix(h.ptr, level, pass_, None, rp.ctypes.data, ci.ctypes.data,
                                     v.ctypes.data), "amg_get_pass_matrix")
    return rp, ci[:nnz], v[:nnz]


def amg_get_colors(h: Handle, level: int) -> np.ndarray:
    out = np.zeros(amg_get_level_info(h, level)["n"], np.int32)
    _check(lib().amg_get_colors(h.ptr, level, out.ctypes.data), "amg_get_colors")
    return out


def amg_get_ilu(h: Handle, level: int) -> np.ndarray:
    nnz = amg_get_level_info(h, level)["nnz"]
    out = np.zeros(max(1, nnz))
    _check(lib().amg_get_ilu(h.ptr, level, out.ctypes.data), "amg_get_ilu")
    return out[:nnz]


def amg_fv_assemble(dim, nx, ny, nz, kx, ky, kz, fx, fy, fz, f, row_ptr, col, val, b, stream=None) -> int:
    """amg_fv_assemble on device tensors; returns nnz."""
    nnz = C.c_int64(0)
    if stream is None:
        stream = _stream_of(kx)
    _check(lib().amg_fv_assemble(dim, nx, ny, nz, _ptr(kx), _ptr(ky), _ptr(kz), _ptr(fx), _ptr(fy),
                                 _ptr(fz), _ptr(f), _ptr(row_ptr, "int64"), _ptr(col, "int32"),
                                 _ptr(val, "float64"), _ptr(b, "float64"), C.byref(nnz), stream),
           "amg_fv_assemble")
    return nnz.value


def amg_csr_value_grad(A, lam, x, grad_val, stream=None):
    cs = _csr(A)
    if stream is None:
        stream = _stream_of(x)
    _check(lib().amg_csr_value_grad(C.byref(cs), _ptr(lam, "float64"), _ptr(x, "float64"),
                                    _ptr(grad_val, "float64"), stream), "amg_csr_value_grad")


def amg_fv_grad_logk(dim, nx, ny, nz, kx, ky, kz, lam, x, gx, gy, gz=None, stream=None):
    if stream is None:
        stream = _stream_of(kx)
    _check(lib().amg_fv_grad_logk(dim, nx, ny, nz, _ptr(kx), _ptr(ky), _ptr(kz), _ptr(lam), _ptr(x),
                                  _ptr(gx), _ptr(gy), _ptr(gz), stream), "amg_fv_grad_logk")


def amg_fv_assemble_logk(dim, nx, ny, nz, logk, kappa, fx, fy, fz, f, row_ptr, col, val, b, stream=None) -> int:
    """amg_fv_assemble_logk on device tensors (kappa = exp(logk) written to
    `kappa`); returns nnz."""
    nnz = C.c_int64(0)
    if stream is None:
        stream = _stream_of(logk)
    _check(lib().amg_fv_assemble_logk(dim, nx, ny, nz, _ptr(logk, "float64"), _ptr(kappa, "float64"), _ptr(fx),
                                      _ptr(fy), _ptr(fz), _ptr(f), _ptr(row_ptr, "int64"), _ptr(col, "int32"),
                                      _ptr(val, "float64"), _ptr(b, "float64"), C.byref(nnz), stream),
           "amg_fv_assemble_logk")
    return nnz.value


def amg_fv_grad_logk_iso(dim, nx, ny, nz, kappa, lam, x, g, stream=None):
    if stream is None:
        stream = _stream_of(kappa)
    _check(lib().amg_fv_grad_logk_iso(dim, nx, ny, nz, _ptr(kappa, "float64"), _ptr(lam, "float64"),
                                      _ptr(x, "float64"), _ptr(g, "float64"), stream), "amg_fv_grad_logk_iso")


from .device import CsrDevice, assemble_fv, assemble_fv_logk, solve  # noqa: E402,F401
from .autograd import AmgSolve, FvLogKappaSolve  # noqa: E402,F401
