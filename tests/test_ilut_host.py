"""The library's host ILUT(tau) (`amg_ilut_host`, the inexact coarse
factorisation of Section 2) against the oracle's, on the CPU: the same
factor pattern and the same values bit for bit, for tau = 0 (complete LU),
the paper's 1e-6 and 1e-4, and a coarse 1e-2, on M-matrices, on a
convection-diffusion operator with upwinding and on a Galerkin coarse
operator of the matching hierarchy.  Also the documented errors: a bad CSR
or tau is rejected, a capacity below the factor's size reports the size,
a zero pivot reports a breakdown."""
import ctypes as C

import numpy as np
import pytest

from paper_1105_3468_gb300 import workloads as W


@pytest.fixture(scope="module")
def pkg():
    from paper_1105_3468_gb300 import build_lib
    build_lib.build()
    import paper_1105_3468_gb300 as p
    return p


def _mmatrix(n, density, seed):
    rng = np.random.default_rng(seed)
    D = -rng.random((n, n)) * (rng.random((n, n)) < density)
    np.fill_diagonal(D, 0.0)
    np.fill_diagonal(D, np.abs(D).sum(axis=1) + 0.1 + rng.random(n))
    return D


def _cases(O):
    yield "mmatrix-80", O.as_csr(_mmatrix(80, 0.06, 1))
    A, _ = O.fv_assemble(W.uniform_grid(24, 2, a=(40.0, -25.0, 0.0)))
    yield "convection-24^2", A
    A, _ = O.fv_assemble(W.c1_block_2d_64())
    yield "block-kappa-64^2", A
    A, _ = O.fv_assemble(W.c3_aniso_3d_128(n=12))
    yield "coarse-aniso-12^3", O.Hierarchy(A, dense_max=0, max_levels=2).matrix(1)


@pytest.mark.parametrize("tau", [0.0, 1e-6, 1e-4, 1e-2])
def test_host_ilut_equals_oracle(pkg, oracle_lib, tau):
    O = oracle_lib
    for name, A in _cases(O):
        rp, ci, v, st = pkg.amg_ilut_host(A.row_ptr, A.col, A.val, tau)
        ref = O.Ilut(A, tau)
        assert st == pkg.AMG_OK and ref.status == 0, name
        assert np.array_equal(rp, ref.F.row_ptr), name
        assert np.array_equal(ci, ref.F.col), name
        assert np.array_equal(v.view(np.int64), ref.F.val.view(np.int64)), name


def test_host_ilut_errors(pkg):
    lib = pkg.lib()
    rp = np.array([0, 2, 4], np.int64)
    ci = np.array([0, 1, 0, 1], np.int32)
    v = np.array([0.0, 1.0, 1.0, 1.0])
    frp = np.zeros(3, np.int64)
    fci = np.zeros(8, np.int32)
    fv = np.zeros(8)
    nnz = C.c_int64(0)

    def call(rp_, ci_, v_, tau, cap):
        return lib.amg_ilut_host(2, rp_.ctypes.data, ci_.ctypes.data, v_.ctypes.data, tau, cap, frp.ctypes.data,
                                 fci.ctypes.data, fv.ctypes.data, C.byref(nnz))

    assert call(rp, ci, v, 0.0, 8) == pkg.AMG_ERR_BREAKDOWN          # a_00 = 0
    v[0] = 2.0
    assert call(rp, ci, v, 0.0, 8) == pkg.AMG_OK and nnz.value == 4
    assert call(rp, ci, v, 0.0, 3) == pkg.AMG_ERR_LIMIT and nnz.value == 4
    assert call(rp, ci, v, -1.0, 8) == pkg.AMG_ERR_INVALID_ARG
    assert call(rp, ci, v, float("nan"), 8) == pkg.AMG_ERR_INVALID_ARG
    bad = np.array([1, 0, 0, 1], np.int32)                           # unsorted row 0
    assert call(rp, bad, v, 0.0, 8) == pkg.AMG_ERR_INVALID_ARG
    nodiag = np.array([0, 1, 0, 0], np.int32)
    assert call(np.array([0, 2, 3], np.int64), nodiag[:3], v[:3], 0.0, 8) == pkg.AMG_ERR_INVALID_ARG


def test_table_norm_value_from_library_factors(pkg, oracle_lib):
    """The paper's comparison of exact and inexact coarse operators
    (||LU - L~U~|| / ||LU||, Section 3) for the DC1 3D case at 30^3 and
    tau = 1e-4: the library's host factors give the value that
    oracle/table_norm.py wrote with the oracle's factors."""
    import json
    import os
    import sys
    O = oracle_lib
    here = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle")
    sys.path.insert(0, here)
    import table_norm
    ref = json.load(open(os.path.join(here, "table_norm.json")))["rows"]["30"]["tau_0.0001"]["rel_error"]
    Ac = table_norm.coarse_operator(30)
    rp, ci, v, st = pkg.amg_ilut_host(Ac.row_ptr, Ac.col, Ac.val, 1e-4)
    assert st == pkg.AMG_OK
    val = table_norm.factor_error(Ac, O.Csr(Ac.n, rp, ci, v))
    assert val == ref
