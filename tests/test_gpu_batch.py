"""Batched path: many systems of uneven size in one solve loop.

* every system's iterates and history equal those of a separate
  amg_setup/amg_solve on that system (same kernels, same order);
* FP64 histories agree with the CPU oracle over the first 20 iterations and
  solutions within 1e-8;
* converged systems drop out while the others continue (uneven iteration
  counts), and per-system statuses are reported.
Members follow the batch recipe at small sizes (and, in the last test, the full
64-member batch workload): block-kappa grids (8x8
blocks, a = (1, 0.5)) and random-geometric-graph matrices, b ~ N(0,1).
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
    import oracle as O
    import paper_1105_3468_gb300 as amg
    return amg, O, torch


def _members(O):
    specs = [W.BatchSpec("grid", 37, 0, 501), W.BatchSpec("rgg", 3001, 9, 502),
             W.BatchSpec("grid", 90, 0, 503), W.BatchSpec("grid", 23, 0, 504),
             W.BatchSpec("rgg", 12000, 21, 505), W.BatchSpec("grid", 64, 0, 506)]
    mats, rhs = [], []
    for s in specs:
        if s.kind == "grid":
            A, _ = O.fv_assemble(W.batch_grid_problem(s))
        else:
            A = O.as_csr(W.rgg_matrix(s.size, s.nnz_per_row, s.seed))
        mats.append(A)
        rhs.append(W.batch_rhs(s, A.n))
    return mats, rhs


@pytest.mark.parametrize("prec", [0, 1])
def test_batch_equals_individual_solves(env, prec):
    amg, O, torch = env
    mats, rhs = _members(O)
    dev = [amg.CsrDevice.from_host(A) for A in mats]
    hb = amg.amg_setup_batched(dev, vcycle_prec=prec)
    count, offs = amg.amg_batch_size(hb)
    assert count == len(mats) and offs[-1] == sum(A.n for A in mats)
    b = torch.tensor(np.concatenate(rhs), device="cuda")
    x = torch.zeros_like(b)
    stats = amg.amg_solve_batched(hb, b, x, 1e-8)
    iters = [s.iters for s in stats]
    assert all(s.status == 0 for s in stats) and all(s.rel_res_true <= 1e-8 for s in stats)
    assert len(set(iters)) > 1                      # uneven: systems leave the loop at different times
    for k, A in enumerate(dev):
        h = amg.amg_setup(A, vcycle_prec=prec)
        xk = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        st = amg.amg_solve(h, b[offs[k]:offs[k + 1]].contiguous(), xk, 1e-8)
        assert st.iters == iters[k]
        assert torch.equal(xk, x[offs[k]:offs[k + 1]])
        hist_b = amg.amg_get_history(amg.amg_batch_member(hb, k))
        assert np.array_equal(hist_b, amg.amg_get_history(h))


def test_batch_device_loop_matches_host_loop(env):
    """The batch's solve loops as one graph (every member a root chain of
    conditional nodes, masks in device memory) give the same bits as the
    host-driven batch loop."""
    amg, O, torch = env
    mats, rhs = _members(O)
    dev = [amg.CsrDevice.from_host(A) for A in mats]
    b = torch.tensor(np.concatenate(rhs), device="cuda")
    out = {}
    for loop in (amg.AMG_LOOP_HOST, amg.AMG_LOOP_DEVICE):
        hb = amg.amg_setup_batched(dev, vcycle_prec=amg.AMG_FP32, solve_loop=loop)
        x = torch.zeros_like(b)
        stats = amg.amg_solve_batched(hb, b, x, 1e-8)
        x2 = torch.zeros_like(b)
        amg.amg_solve_batched(hb, b, x2, 1e-8)              # the cached batch graph again
        assert torch.equal(x, x2)
        out[loop] = (x.cpu().numpy(), [(s.iters, s.restarts, s.status, s.rel_res_true) for s in stats],
                     [amg.amg_get_history(amg.amg_batch_member(hb, k)) for k in range(len(mats))])
    a, c = out[amg.AMG_LOOP_HOST], out[amg.AMG_LOOP_DEVICE]
    assert np.array_equal(a[0], c[0]) and a[1] == c[1]
    assert all(np.array_equal(p, q) for p, q in zip(a[2], c[2]))


def test_batch_fp64_against_oracle(env):
    amg, O, torch = env
    mats, rhs = _members(O)
    hb = amg.amg_setup_batched([amg.CsrDevice.from_host(A) for A in mats])
    _, offs = amg.amg_batch_size(hb)
    b = torch.tensor(np.concatenate(rhs), device="cuda")
    x = torch.zeros_like(b)
    amg.amg_solve_batched(hb, b, x, 1e-8)
    worst = []
    for k, A in enumerate(mats):
        xo, info = O.Hierarchy(A).fgmres(rhs[k], tol=1e-8)
        assert info.status == 0
        hist = amg.amg_get_history(amg.amg_batch_member(hb, k))
        m = min(21, len(hist), len(info.hist))
        rel = np.abs(hist[:m] - info.hist[:m]) / info.hist[:m]
        xk = x[offs[k]:offs[k + 1]].cpu().numpy()
        worst.append((k, A.n, float(rel.max()), int(rel.argmax()),
                      float(np.linalg.norm(xk - xo) / np.linalg.norm(xo))))
    print("member, n, max rel history diff, at iteration, rel x diff:", worst)
    for k, n, hdiff, _, xdiff in worst:
        assert hdiff <= 1e-10, (k, n, hdiff)
        assert xdiff <= 1e-8, (k, n, xdiff)


def test_batch_reports_per_system_failure(env):
    amg, O, torch = env
    mats, rhs = _members(O)
    hb = amg.amg_setup_batched([amg.CsrDevice.from_host(A) for A in mats], maxit=3)
    b = torch.tensor(np.concatenate(rhs), device="cuda")
    x = torch.zeros_like(b)
    stats = amg.amg_solve_batched(hb, b, x, 1e-12)
    assert all(s.status == amg.AMG_ERR_NOT_CONVERGED and s.iters == 3 for s in stats)
    with pytest.raises(amg.AmgError):
        amg.amg_solve(hb, b, x, 1e-8)               # a batch handle needs amg_solve_batched


def test_fullsize_batch_sampled_members(env):
    """The 64-member batch workload (48 block-kappa grids of side 64..512 and
    16 random-geometric-graph matrices of 10k..500k rows) in the configuration
    the benchmark times (last levels of up to 1024 rows solved exactly, every
    member's loop in one graph): all members converge with the FP64 and the
    FP32 V-cycle; for four sampled members (the smallest and a mid-size grid,
    the smallest and the largest graph matrix) the FP64 history agrees with
    the oracle's within 1e-10 over 20 iterations and the FP64 solution within
    1e-8; the FP32 V-cycle's solutions are printed and bounded (1e-6)."""
    amg, O, torch = env
    specs = W.c5_batch_specs()
    mats, hmats, rhs = [], [], []
    for sp in specs:
        if sp.kind == "grid":
            A, _ = O.fv_assemble(W.batch_grid_problem(sp))
        else:
            A = O.as_csr(W.rgg_matrix(sp.size, sp.nnz_per_row, sp.seed))
        hmats.append(A)
        mats.append(amg.CsrDevice.from_host(A))
        rhs.append(W.batch_rhs(sp, A.n))
    b = torch.tensor(np.concatenate(rhs), device="cuda")
    out = {}
    for prec in (amg.AMG_FP64, amg.AMG_FP32):
        hb = amg.amg_setup_batched(mats, vcycle_prec=prec, dense_max=1024)
        _, offs = amg.amg_batch_size(hb)
        x = torch.zeros_like(b)
        stats = amg.amg_solve_batched(hb, b, x, 1e-8)
        assert all(s.status == 0 and s.rel_res_true <= 1e-8 for s in stats)
        out[prec] = (hb, offs, x.cpu().numpy(), stats)
    grids = [k for k, s in enumerate(specs) if s.kind == "grid"]
    rggs = [k for k, s in enumerate(specs) if s.kind == "rgg"]
    by_n = lambda ks: sorted(ks, key=lambda k: hmats[k].n)
    sample = [by_n(grids)[0], by_n(grids)[len(grids) // 2], by_n(rggs)[0], by_n(rggs)[-1]]
    hb, offs, x64, _ = out[amg.AMG_FP64]
    _, _, x32, st32 = out[amg.AMG_FP32]
    for k in sample:
        A = hmats[k]
        H = O.Hierarchy(A, dense_max=1024)
        xo, info = H.fgmres(rhs[k], tol=1e-8)
        assert info.status == 0
        hist = amg.amg_get_history(amg.amg_batch_member(hb, k))
        m = min(21, len(hist), len(info.hist))
        hdiff = float((np.abs(hist[:m] - info.hist[:m]) / info.hist[:m]).max())
        e64 = float(np.linalg.norm(x64[offs[k]:offs[k + 1]] - xo) / np.linalg.norm(xo))
        e32 = float(np.linalg.norm(x32[offs[k]:offs[k + 1]] - xo) / np.linalg.norm(xo))
        print(f"batch member {k} ({specs[k].kind}, {A.n} rows): oracle {info.iters} iterations, FP32 "
              f"{st32[k].iters}; history diff {hdiff:.1e}, |x - x_oracle|/|x_oracle| FP64 {e64:.1e}, FP32 {e32:.1e}")
        assert hdiff <= 1e-10 and e64 <= 1e-8 and e32 <= 1e-6
