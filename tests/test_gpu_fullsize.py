"""GPU parity at the benchmark's full sizes, in the configuration the
benchmark times.

* 3D anisotropic block-kappa problem, 128^3 cells (2,097,152 unknowns):
  the whole hierarchy bit-exact against the oracle (aggregates, Galerkin
  products, colourings, ILU(0) factors); one FP64 V-cycle application
  within 1e-12 relative; the FP64 FGMRES residual history within 1e-10 relative over
  the first 20 iterations; the benchmark's FP32 V-cycle solve reaches the
  true FP64 residual 1e-8 (recomputed on the host) within 10% of the FP64
  oracle's iteration count.
* 2D rotating-flow problem, 1024^2 cells (1,048,576 unknowns) with
  colour-major fine ILU(0): hierarchy bit-exact, history within 1e-10 over
  the first 20 iterations.

The oracle's full solve of the 128^3 problem takes about half an hour, so its
iteration count comes from oracle/workload_iters.json (written by
oracle/workload_iters.py, which runs only the oracle).
"""
import json
import os

import numpy as np
import pytest

from paper_1105_3468_gb300 import workloads as W

from hierarchy_check import check_hierarchy

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import oracle as O
    import paper_1105_3468_gb300 as amg
    return amg, O, torch


CASES = {
    # problem, options of the benchmark for it (GPU name -> oracle name)
    "c3": (lambda: W.c3_aniso_3d_128(), {}),
    "c2": (lambda: W.c2_rotating_2d_1024(), {"order_fine": 0, "match_weight": 0}),
}


@pytest.fixture(scope="module")
def full(env):
    amg, O, torch = env
    cache = {}

    def get(name):
        if name not in cache:
            make, opts = CASES[name]
            p = make()
            A, b = amg.assemble_fv(p)
            Ao, bo = O.fv_assemble(p)
            H = O.Hierarchy(Ao, **opts)
            cache[name] = (A, b, Ao, bo, H, opts)
        return cache[name]
    return get


@pytest.mark.parametrize("name", ["c3", "c2"])
def test_fullsize_hierarchy_bit_exact(env, full, name):
    amg, O, torch = env
    A, b, Ao, bo, H, opts = full(name)
    assert np.array_equal(A.val.cpu().numpy(), Ao.val) and np.array_equal(b.cpu().numpy(), bo)
    h = amg.amg_setup(A, **opts)
    check_hierarchy(amg, h, H)


def test_fullsize_c3_vcycle_fp64(env, full):
    """One FP64 V-cycle application within 1e-12 relative of the oracle's
    (the dense last level sums each row in another order on the GPU)."""
    amg, O, torch = env
    A, b, Ao, bo, H, opts = full("c3")
    h = amg.amg_setup(A, **opts)
    z = np.random.default_rng(33).standard_normal(A.n)
    q = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    amg.amg_precond_apply(h, torch.as_tensor(z).cuda(), q)
    qo = H.precond(z)
    qg = q.cpu().numpy()
    rel = np.abs(qg - qo).max() / np.abs(qo).max()
    print(f"128^3 FP64 V-cycle: {int((qg != qo).sum())} of {A.n} entries differ from the oracle, "
          f"max rel diff {rel:.2e}")
    assert rel <= 1e-12


@pytest.mark.parametrize("name", ["c3", "c2"])
def test_fullsize_fp64_history_first_20(env, full, name):
    amg, O, torch = env
    A, b, Ao, bo, H, opts = full(name)
    h = amg.amg_setup(A, maxit=20, **opts)
    x = torch.zeros_like(b)
    st = amg.amg_solve(h, b, x, 1e-8)
    assert st.iters == 20
    hist = amg.amg_get_history(h)
    _, info = H.fgmres(bo, tol=1e-8, maxit=20)
    assert len(hist) == len(info.hist) == 21
    rel = np.abs(hist - info.hist) / info.hist
    print(f"{name}: FP64 history max rel diff over 20 iterations {rel.max():.2e}")
    assert rel.max() <= 1e-10


def test_fullsize_c3_bench_configuration(env, full):
    """FP32 V-cycle inside FP64 FGMRES(30), tol 1e-8, maxit 3000."""
    amg, O, torch = env
    A, b, Ao, bo, H, opts = full("c3")
    h = amg.amg_setup(A, vcycle_prec=amg.AMG_FP32, maxit=3000, **opts)
    x = torch.zeros_like(b)
    st = amg.amg_solve(h, b, x, 1e-8)
    assert st.status == 0 and st.rel_res_true <= 1e-8
    r = bo - O.spmv(Ao, x.cpu().numpy())
    rel = np.linalg.norm(r) / np.linalg.norm(bo)
    assert rel <= 1.0000001e-8
    iters = json.load(open(os.path.join(ROOT, "oracle", "workload_iters.json")))["c3"]
    print(f"128^3 FP32 V-cycle: {st.iters} iterations (FP64 oracle {iters}), true rel. residual {rel:.3e}")
    assert abs(st.iters - iters) <= 0.1 * iters


def test_fullsize_c3_bf16_factors(env, full):
    """BF16 ILU(0) factors on the finest level (FP32 elsewhere) inside FP64
    FGMRES reach the true FP64 residual 1e-8 within 10% of the FP64 oracle's
    iteration count."""
    amg, O, torch = env
    A, b, Ao, bo, H, opts = full("c3")
    h = amg.amg_setup(A, vcycle_prec=amg.AMG_BF16, maxit=3000, **opts)
    x = torch.zeros_like(b)
    st = amg.amg_solve(h, b, x, 1e-8)
    assert st.status == 0
    rel = np.linalg.norm(bo - O.spmv(Ao, x.cpu().numpy())) / np.linalg.norm(bo)
    assert rel <= 1.0000001e-8
    iters = json.load(open(os.path.join(ROOT, "oracle", "workload_iters.json")))["c3"]
    print(f"128^3 BF16 factors: {st.iters} iterations (FP64 oracle {iters}), true rel. residual {rel:.3e}")
    assert abs(st.iters - iters) <= 0.1 * iters
