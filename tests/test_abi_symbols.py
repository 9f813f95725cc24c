"""The C-ABI library builds, loads on a host without a GPU, and exports every
entry point include/amg.h declares; host-only calls behave as documented."""
import ctypes as C
import os
import re

import pytest

from conftest import ROOT


def _declared():
    src = open(os.path.join(ROOT, "include", "amg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(amg_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1105_3468_gb300 import build_lib
    build_lib.build()
    import paper_1105_3468_gb300 as pkg
    return pkg.lib()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_header():
    from paper_1105_3468_gb300 import _lib
    assert sorted(_lib.SIGNATURES) == _declared()


def test_host_only_calls(lib):
    import paper_1105_3468_gb300 as pkg
    o = pkg.amg_default_options()
    assert (o.passes, o.coarse_inner, o.restart, o.maxit, o.dense_max) == (2, 5, 30, 600, 4096)
    assert o.order_fine == pkg.AMG_ORDER_NATURAL and o.order_coarse == pkg.AMG_ORDER_COLOR
    assert o.coarse_solver == pkg.AMG_COARSE_RECURSIVE and o.ilut_tau == 1e-6
    assert o.match_weight == pkg.AMG_MATCH_SCALED and o.solve_loop == pkg.AMG_LOOP_DEVICE
    assert pkg.amg_status_string(pkg.AMG_ERR_NOT_CONVERGED) == "not converged"
    assert lib.amg_default_options(None) == pkg.AMG_ERR_INVALID_ARG
    out = C.c_void_p(123)
    assert lib.amg_setup(None, None, None, C.byref(out)) == pkg.AMG_ERR_INVALID_ARG
    assert out.value is None
    assert "null" in pkg.lib().amg_last_error().decode()
    assert "sm_103a" in pkg.amg_version()
    assert o.persistent == 5      # grid tiles on a stencil finest level, else as 3
    info = (C.c_int64 * 8)()
    kind = (C.c_int32 * 2)()
    assert lib.amg_get_tile_grid(None, info) == pkg.AMG_ERR_INVALID_ARG
    assert lib.amg_get_sweep_kind(None, 0, kind) == pkg.AMG_ERR_INVALID_ARG


def test_struct_sizes_match_header():
    from paper_1105_3468_gb300 import _lib
    assert C.sizeof(_lib.AmgOptions) == 20 * 4 + 8 + 2 * 4 + 8
    assert C.sizeof(_lib.AmgStats) == 4 * 4 + 3 * 8 + 2 * 4 + 2 * 8


def test_setup_rejects_bad_options_before_any_device_call(lib):
    """amg_setup validates its options first (no GPU needed to see that)."""
    import paper_1105_3468_gb300 as pkg
    from paper_1105_3468_gb300 import _lib
    A = _lib.AmgCsr()
    out = C.c_void_p()
    for field, value in (("coarse_solver", 2), ("ilut_tau", -1.0), ("ilut_tau", float("nan")),
                         ("ilut_tau", float("inf")), ("dense_max", 4097), ("persistent", 6), ("passes", 0),
                         ("match_weight", 2), ("match_weight", -1), ("solve_loop", 2),
                         ("vcycle_prec", 4)):
        o = pkg.amg_default_options()
        setattr(o, field, value)
        assert lib.amg_setup(C.byref(A), C.byref(o), None, C.byref(out)) == pkg.AMG_ERR_INVALID_ARG, field
        assert not out.value
