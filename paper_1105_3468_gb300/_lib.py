"""ctypes binding of libamg_gb (include/amg.h): structures and signatures.

This module only loads the in-tree shared library and declares its entry
points; it performs no arithmetic.  Loading fails loudly (RuntimeError) when
the library has not been built: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import build_lib

AMG_OK = 0
AMG_ERR_INVALID_ARG = 1
AMG_ERR_CUDA = 2
AMG_ERR_OOM = 3
AMG_ERR_NOT_SUPPORTED = 4
AMG_ERR_BREAKDOWN = 5
AMG_ERR_NUMERIC = 6
AMG_ERR_NOT_CONVERGED = 7
AMG_ERR_LIMIT = 8

AMG_FP64, AMG_FP32, AMG_BF16, AMG_BF16_ALL = 0, 1, 2, 3
AMG_NOALLOC_MAX_ROWS = 4194304
AMG_ORDER_COLOR, AMG_ORDER_NATURAL = 0, 1
AMG_COLOR_HASH_JP, AMG_COLOR_FIRST_FIT = 0, 1
AMG_ORTHO_MGS, AMG_ORTHO_CGS2 = 0, 1
AMG_COARSE_RECURSIVE, AMG_COARSE_ILUT = 0, 1
AMG_MATCH_PLAIN, AMG_MATCH_SCALED = 0, 1
AMG_LOOP_HOST, AMG_LOOP_DEVICE = 0, 1


class AmgCsr(C.Structure):
    _fields_ = [("n", C.c_int32), ("nnz", C.c_int64), ("row_ptr", C.c_void_p),
                ("col", C.c_void_p), ("val", C.c_void_p)]


class AmgOptions(C.Structure):
    _fields_ = [("passes", C.c_int32), ("coarse_inner", C.c_int32), ("deep_inner", C.c_int32),
                ("dense_max", C.c_int32), ("max_levels", C.c_int32), ("order_fine", C.c_int32),
                ("order_coarse", C.c_int32), ("coloring", C.c_int32), ("restart", C.c_int32),
                ("maxit", C.c_int32), ("vcycle_prec", C.c_int32), ("build_adjoint", C.c_int32),
                ("use_graphs", C.c_int32), ("persistent", C.c_int32), ("deep_block_max", C.c_int32),
                ("orthog", C.c_int32), ("spmv_block", C.c_int32), ("spmv_unroll", C.c_int32),
                ("dot2", C.c_int32), ("match_weight", C.c_int32),
                ("seed", C.c_uint64), ("coarse_solver", C.c_int32), ("solve_loop", C.c_int32),
                ("ilut_tau", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class AmgStats(C.Structure):
    _fields_ = [("status", C.c_int32), ("iters", C.c_int32), ("restarts", C.c_int32),
                ("nlevels", C.c_int32), ("rel_res_true", C.c_double), ("setup_ms", C.c_double),
                ("solve_ms", C.c_double), ("n_coarse", C.c_int32), ("n_colors", C.c_int32),
                ("nnz_coarse", C.c_int64), ("kernel_launches", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


# every symbol the header declares, with (restype, argtypes)
_P = C.c_void_p
SIGNATURES = {
    "amg_version": (C.c_char_p, []),
    "amg_status_string": (C.c_char_p, [C.c_int]),
    "amg_last_error": (C.c_char_p, []),
    "amg_default_options": (C.c_int, [C.POINTER(AmgOptions)]),
    "amg_setup": (C.c_int, [C.POINTER(AmgCsr), C.POINTER(AmgOptions), _P, C.POINTER(_P)]),
    "amg_destroy": (None, [_P]),
    "amg_update_values": (C.c_int, [_P, _P]),
    "amg_ilut_host": (C.c_int, [C.c_int32, _P, _P, _P, C.c_double, C.c_int64, _P, _P, _P,
                                C.POINTER(C.c_int64)]),
    "amg_solve": (C.c_int, [_P, _P, _P, C.c_double, C.POINTER(AmgStats)]),
    "amg_adjoint": (C.c_int, [_P, _P, _P, C.c_double, C.POINTER(AmgStats)]),
    "amg_get_history": (C.c_int, [_P, _P, C.c_int32, C.POINTER(C.c_int32)]),
    "amg_setup_batched": (C.c_int, [_P, C.c_int32, C.POINTER(AmgOptions), _P, C.POINTER(_P)]),
    "amg_solve_batched": (C.c_int, [_P, _P, _P, C.c_double, _P]),
    "amg_batch_size": (C.c_int, [_P, C.POINTER(C.c_int32), _P]),
    "amg_batch_member": (_P, [_P, C.c_int32]),
    "amg_precond_apply": (C.c_int, [_P, _P, _P, C.c_int32]),
    "amg_spmv": (C.c_int, [C.POINTER(AmgCsr), _P, _P, _P]),
    "amg_spmv_noalloc": (C.c_int, [C.POINTER(AmgCsr), _P, _P, _P]),
    "amg_get_level_info": (C.c_int, [_P, C.c_int32, _P]),
    "amg_get_tile_grid": (C.c_int, [_P, _P]),
    "amg_get_sweep_kind": (C.c_int, [_P, C.c_int32, _P]),
    "amg_num_levels": (C.c_int, [_P, C.POINTER(C.c_int32)]),
    "amg_get_spmv_config": (C.c_int, [_P, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "amg_get_aggregates": (C.c_int, [_P, C.c_int32, C.c_int32, _P]),
    "amg_get_matrix": (C.c_int, [_P, C.c_int32, _P, _P, _P]),
    "amg_get_pass_matrix": (C.c_int, [_P, C.c_int32, C.c_int32, _P, _P, _P, _P]),
    "amg_get_colors": (C.c_int, [_P, C.c_int32, _P]),
    "amg_get_ilu": (C.c_int, [_P, C.c_int32, _P]),
    "amg_set_kernel_timing": (C.c_int, [_P, C.c_int32]),
    "amg_get_kernel_timing": (C.c_int, [_P, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.POINTER(C.c_double)]),
    "amg_launch_counter": (C.c_int64, []),
    "amg_fv_assemble": (C.c_int, [C.c_int32] * 4 + [_P] * 7 + [_P, _P, _P, _P, C.POINTER(C.c_int64), _P]),
    "amg_csr_value_grad": (C.c_int, [C.POINTER(AmgCsr), _P, _P, _P, _P]),
    "amg_fv_grad_logk": (C.c_int, [C.c_int32] * 4 + [_P] * 8 + [_P]),
    "amg_fv_assemble_logk": (C.c_int, [C.c_int32] * 4 + [_P] * 6 + [_P, _P, _P, _P, C.POINTER(C.c_int64), _P]),
    "amg_fv_grad_logk_iso": (C.c_int, [C.c_int32] * 4 + [_P] * 4 + [_P]),
}

_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return build_lib.LIB


def load(build_if_missing: bool = False) -> C.CDLL:
    """Load libamg_gb.so; raise RuntimeError if it is absent."""
    global _lib
    with _lock:
        if _lib is None:
            path = build_lib.LIB
            if build_if_missing and not build_lib.up_to_date():
                build_lib.build()
            if not os.path.exists(path):
                raise RuntimeError(
                    f"libamg_gb.so is not built ({path}); run __graft_entry__.build() or "
                    "python paper_1105_3468_gb300/build_lib.py")
            L = C.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib
