"""The finest level's ILU(0) solves in grid tiles (persistent = 5, the
default) against the dataflow solve (persistent = 3).

* Grids whose sizes are and are not multiples of the tile (16^3 in 3D, 64^2
  in 2D), one tile and many: the V-cycle (amg_precond_apply) is bit-identical
  in FP64, FP32 and BF16, forward and transposed, over repeated applications
  (the mailboxes are reset between launches), and a whole solve gives the
  same iterations and the same bits.
* The grid is detected from the pattern (amg_get_tile_grid).
* Matrices that are not natural-order grid stencils keep the dataflow solve:
  a random geometric graph, a grid matrix with one coupling removed (the
  factor check rejects it), colour-major order on the finest level.
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


def grid_problem(dim, nx, ny, nz, seed):
    """Log-normal conductivity per cell and axis, constant velocity (1, -0.5, 0.25), f = 1."""
    rng = np.random.default_rng(seed)
    n = nx * ny * nz
    k = [10.0 ** rng.uniform(-2, 2, n) for _ in range(3)]
    h = 1.0 / nx
    area = h ** (dim - 1)
    fx = np.full((nx + 1) * ny * nz, area * 1.0)
    fy = np.full(nx * (ny + 1) * nz, area * -0.5)
    fz = np.full(nx * ny * (nz + 1), area * 0.25) if dim == 3 else np.zeros(0)
    return W.GridProblem(dim, nx, ny, nz, k[0], k[1], k[2], fx, fy, fz, np.ones(n), name=f"grid{nx}x{ny}x{nz}")


GRIDS = [(3, 40, 24, 20), (3, 16, 16, 16), (3, 33, 17, 35), (2, 130, 70, 1), (2, 64, 64, 1), (2, 200, 9, 1)]


@pytest.mark.parametrize("grid", GRIDS, ids=lambda g: "x".join(map(str, g[1:])))
def test_tiled_vcycle_bit_identical(env, grid):
    amg, torch = env
    dim, nx, ny, nz = grid
    p = grid_problem(dim, nx, ny, nz, seed=nx * 7 + ny)
    A, b = amg.assemble_fv(p)
    n = nx * ny * nz
    g = torch.Generator(device="cuda").manual_seed(11)
    for prec in (amg.AMG_FP64, amg.AMG_FP32, amg.AMG_BF16):
        h5 = amg.amg_setup(A, vcycle_prec=prec, build_adjoint=1)
        h3 = amg.amg_setup(A, vcycle_prec=prec, build_adjoint=1, persistent=3)
        info = amg.amg_get_tile_grid(h5)
        assert info["tiled"] and info["grid"] == (nx, ny, nz), info
        assert info["tile"] == ((16, 16, 16) if dim == 3 else (64, 64, 1))
        assert not amg.amg_get_tile_grid(h3)["tiled"]
        for rep in range(3):
            z = torch.randn(n, dtype=torch.float64, device="cuda", generator=g)
            for tr in (False, True):
                q5 = torch.empty_like(z)
                q3 = torch.empty_like(z)
                amg.amg_precond_apply(h5, z, q5, tr)
                amg.amg_precond_apply(h3, z, q3, tr)
                assert torch.isfinite(q5).all()
                assert torch.equal(q5, q3), (prec, rep, tr, (q5 - q3).abs().max().item())
        x5 = torch.zeros_like(b)
        x3 = torch.zeros_like(b)
        s5 = amg.amg_solve(h5, b, x5, 1e-8)
        s3 = amg.amg_solve(h3, b, x3, 1e-8)
        assert s5.status == 0 and s3.status == 0
        assert s5.iters == s3.iters and torch.equal(x5, x3)
        print(f"{nx}x{ny}x{nz} prec {prec}: {info['ntiles']} tiles, {s5.iters} iterations, bit-identical")


def test_non_stencil_matrices_keep_dataflow(env):
    amg, torch = env
    # random geometric graph
    M = W.rgg_matrix(4000, 7, seed=3)
    from paper_1105_3468_gb300.device import CsrDevice
    A = CsrDevice(M.n, torch.as_tensor(M.row_ptr).cuda(), torch.as_tensor(M.col).cuda(),
                  torch.as_tensor(M.val).cuda())
    h = amg.amg_setup(A)
    assert not amg.amg_get_tile_grid(h)["tiled"]
    # a 2D grid matrix with one coupling removed: offsets still describe the
    # grid, the per-row check rejects it; both schedules still agree
    A2, b2 = amg.assemble_fv(grid_problem(2, 130, 70, 1, seed=5))
    rp = A2.row_ptr.cpu().numpy()
    ci = A2.col.cpu().numpy()
    v = A2.val.cpu().numpy()
    r = 70 * 130 // 2 + 17
    drop = [e for e in range(rp[r], rp[r + 1]) if ci[e] == r - 130][0]
    keep = np.ones(len(ci), bool)
    keep[drop] = False
    rp2 = rp.copy()
    rp2[r + 1:] -= 1
    A3 = CsrDevice(A2.n, torch.as_tensor(rp2).cuda(), torch.as_tensor(ci[keep]).cuda(),
                   torch.as_tensor(v[keep]).cuda())
    h5 = amg.amg_setup(A3)
    h3 = amg.amg_setup(A3, persistent=3)
    assert not amg.amg_get_tile_grid(h5)["tiled"]
    z = torch.randn(A2.n, dtype=torch.float64, device="cuda")
    q5 = torch.empty_like(z)
    q3 = torch.empty_like(z)
    amg.amg_precond_apply(h5, z, q5)
    amg.amg_precond_apply(h3, z, q3)
    assert torch.equal(q5, q3)
    # colour-major order on the finest level
    hc = amg.amg_setup(A2, order_fine=amg.AMG_ORDER_COLOR)
    assert not amg.amg_get_tile_grid(hc)["tiled"]
