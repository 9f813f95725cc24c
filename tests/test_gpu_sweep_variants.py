"""The default smoother variants (persistent = 5: grid tiles on the finest
level, cooperative grids with grid barriers, one-cluster and one-block
kernels on the coloured levels, as amg_get_sweep_kind reports them) against
one launch per schedule level (persistent = 0), at sizes where every
variant but the dataflow solve runs:

* the 3D anisotropic recipe at 64^3 (levels of 262 K, 72 K, 20 K, 6 K rows),
* the paper's DC1 3D case at 80^3.

The V-cycle (amg_precond_apply) is bit-identical in FP64, FP32, BF16 and
BF16-on-every-level, forward and transposed, over repeated applications, and
a whole solve gives the same iterations and the same bits.
"""
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


CASES = {
    "c3-64": (lambda: W.c3_aniso_3d_128(n=64), {}),
    "dc1-3d-80": (lambda: W.dc_problem(80, 3), {}),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_default_sweep_variants_bit_identical(env, name):
    amg, torch = env
    make, opts = CASES[name]
    A, b = amg.assemble_fv(make())
    g = torch.Generator(device="cuda").manual_seed(5)
    for prec in (amg.AMG_FP64, amg.AMG_FP32, amg.AMG_BF16, amg.AMG_BF16_ALL):
        h5 = amg.amg_setup(A, vcycle_prec=prec, build_adjoint=1, **opts)
        h0 = amg.amg_setup(A, vcycle_prec=prec, build_adjoint=1, persistent=0, **opts)
        for rep in range(2):
            z = torch.randn(A.n, dtype=torch.float64, device="cuda", generator=g)
            for tr in (False, True):
                q5 = torch.empty_like(z)
                q0 = torch.empty_like(z)
                amg.amg_precond_apply(h5, z, q5, tr)
                amg.amg_precond_apply(h0, z, q0, tr)
                assert torch.isfinite(q5).all()
                assert torch.equal(q5, q0), (prec, rep, tr, (q5 - q0).abs().max().item())
        nl = amg.amg_num_levels(h5)
        kinds = [amg.amg_get_sweep_kind(h5, l) for l in range(nl)]
        assert kinds[0] == ("tiles", "tiles"), kinds
        assert any(k[0] in ("grid", "dsm_replicated", "block", "cluster_grid") for k in kinds[1:]), kinds
        assert all(amg.amg_get_sweep_kind(h0, l)[0] in ("levels", None) for l in range(nl))
        x5 = torch.zeros_like(b)
        x0 = torch.zeros_like(b)
        s5 = amg.amg_solve(h5, b, x5, 1e-8)
        s0 = amg.amg_solve(h0, b, x0, 1e-8)
        assert s5.status == s0.status and s5.iters == s0.iters and torch.equal(x5, x0)
        print(f"{name} prec {prec}: {s5.iters} iterations, bit-identical; kinds {kinds}")
