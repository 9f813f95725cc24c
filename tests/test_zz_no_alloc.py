"""amg_spmv_noalloc: the SpMV entry point for callers that cannot let the
library allocate device memory (a process whose own allocator has reserved
the free device memory, or a loop that must not be stalled by the device-wide
synchronisation of cudaFree).  Its scratch (the int32 row-pointer copy) lives in a
fixed device array shared by every call.  This file is collected last so a
failure here stops a -x run only after every other test has run; it also
passes alone in a fresh process (the first call looks the array up)."""
import numpy as np
import pytest

from paper_1105_3468_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1105_3468_gb300 as amg
    return amg, torch


def test_noalloc_matches_spmv_on_consecutive_calls(env):
    amg, torch = env
    rng = np.random.default_rng(11)
    cases = [W.rgg_matrix(50_001, 13, seed=21), W.rgg_matrix(7_777, 29, seed=22)]
    for A in cases:                                  # two calls in a row, different sizes
        Ad = amg.CsrDevice.from_host(A)
        x = torch.tensor(rng.standard_normal(A.n), device="cuda")
        y_ref = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        y = torch.full((A.n,), float("nan"), dtype=torch.float64, device="cuda")
        amg.amg_spmv(Ad, x, y_ref)
        amg.amg_spmv_noalloc(Ad, x, y)
        torch.cuda.synchronize()
        ref = y_ref.cpu().numpy()
        assert np.allclose(y.cpu().numpy(), ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())


def test_noalloc_rejects_oversized(env):
    amg, torch = env
    n = amg.AMG_NOALLOC_MAX_ROWS + 1

    class Fake:                                      # sizes only: rejected before any GPU work
        pass
    A = Fake()
    A.n = n
    A.row_ptr = np.zeros(2, np.int64)
    A.col = np.zeros(1, np.int32)
    A.val = np.zeros(1)
    x = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(amg.AmgError) as e:
        amg.amg_spmv_noalloc(A, x, x)
    assert e.value.status == amg.AMG_ERR_INVALID_ARG
    assert "AMG_NOALLOC_MAX_ROWS" in str(e.value)


def test_invalid_indices_rejected_without_out_of_range_reads(env):
    """A row pointer beyond nnz or a column outside [0, n) is reported as
    AMG_ERR_INVALID_ARG by amg_spmv and amg_spmv_noalloc.  The kernels clamp
    the row pointers to [0, nnz] and skip such columns, so no entry is used as
    an index outside the caller's buffers; the next valid call is exact."""
    amg, torch = env
    A = W.rgg_matrix(3_001, 9, seed=23)
    x = torch.tensor(np.random.default_rng(12).standard_normal(A.n), device="cuda")
    y_ref = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    good = amg.CsrDevice.from_host(A)
    amg.amg_spmv(good, x, y_ref)
    bad_rp = amg.CsrDevice.from_host(A)
    bad_rp.row_ptr[A.n // 2] = A.nnz + 100
    bad_col = amg.CsrDevice.from_host(A)
    bad_col.col[A.nnz // 3] = A.n + 5
    for call in (amg.amg_spmv, amg.amg_spmv_noalloc):
        for bad in (bad_rp, bad_col):
            y = torch.zeros(A.n, dtype=torch.float64, device="cuda")
            with pytest.raises(amg.AmgError) as e:
                call(bad, x, y)
            assert e.value.status == amg.AMG_ERR_INVALID_ARG
        y = torch.full((A.n,), float("nan"), dtype=torch.float64, device="cuda")
        call(good, x, y)
        torch.cuda.synchronize()
        ref = y_ref.cpu().numpy()
        assert np.allclose(y.cpu().numpy(), ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())
