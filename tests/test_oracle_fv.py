"""Pins of the oracle's finite-volume discretisation of eq. (2) (Section 1).

* a hand-derived 2x2 example (tests/golden/fv_2x2.txt) and its 3D analogue;
* convergence order on a manufactured solution: 2 for pure diffusion (also
  with a smooth variable conductivity), 1 for first-order upwind convection;
* for a = 0 the matrix is a symmetric, weakly diagonally dominant M-matrix
  (the M-matrix criterion of Section 2.1), with row sums equal to the
  Dirichlet transmissibilities;
* with a discretely divergence-free velocity every row sum is non-negative;
* the log-conductivity gradient matches central finite differences.
"""
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as sla

from conftest import GOLDEN
from paper_1105_3468_gb300 import workloads as W


def _golden_blocks(name):
    blocks, cur = [], []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line.startswith("#"):
            if cur:
                blocks.append(np.array(cur, dtype=float))
                cur = []
            continue
        if line:
            cur.append([float(t) for t in line.split()])
    if cur:
        blocks.append(np.array(cur, dtype=float))
    return blocks


def _sp(A):
    return sp.csr_matrix((A.val, A.col, A.row_ptr), shape=(A.n, A.n))


def test_golden_2x2(oracle_lib):
    O = oracle_lib
    A0, A1, bb = _golden_blocks("fv_2x2.txt")
    A, b = O.fv_assemble(W.uniform_grid(2, 2, a=(0.0, 0.0)))
    assert np.array_equal(A.dense(), A0)
    assert np.array_equal(b, bb.ravel())
    A, b = O.fv_assemble(W.uniform_grid(2, 2, a=(1.0, 0.0)))
    assert np.array_equal(A.dense(), A1)


def test_golden_2x2x2_diffusion(oracle_lib):
    """h = 1/2 in 3D: interior T = h*1 = 0.5, Dirichlet T = h*2 = 1;
    each cell has one interior neighbour per axis, one Dirichlet face (y)
    and two Neumann faces (x, z): diagonal 0.5*3 + 1 = 2.5."""
    O = oracle_lib
    A, b = O.fv_assemble(W.uniform_grid(2, 3))
    D = A.dense()
    assert np.all(np.diag(D) == 2.5)
    off = D - np.diag(np.diag(D))
    for i in range(8):
        nbrs = [i ^ 1, i ^ 2, i ^ 4]   # x, y, z neighbour in a 2x2x2 block
        assert sorted(np.nonzero(off[i])[0].tolist()) == sorted(nbrs)
        assert np.all(off[i, nbrs] == -0.5)
    assert np.all(b == 0.125)


def test_column_order_and_csr_valid(oracle_lib):
    O = oracle_lib
    for p in (W.c1_block_2d_64(), W.c3_aniso_3d_128(n=6), W.c2_rotating_2d_1024(n=20)):
        A, _ = O.fv_assemble(p)
        assert O.check_csr(A) == O.OK
        nnz_expect = (2 * p.dim + 1) * p.n - 2 * sum(p.n // s for s in [p.nx, p.ny, p.nz][:p.dim])
        assert A.nnz == nnz_expect


def _mms_2d(O, n, a, kfun):
    pi = np.pi
    xs = (np.arange(n) + 0.5) / n
    Y, X = np.meshgrid(xs, xs, indexing="ij")
    X, Y = X.ravel(), Y.ravel()
    u = np.cos(pi * X) * np.sin(pi * Y)     # u = 0 on y = 0,1; du/dx = 0 on x = 0,1
    ux = -pi * np.sin(pi * X) * np.sin(pi * Y)
    uy = pi * np.cos(pi * X) * np.cos(pi * Y)
    k, kx, ky = kfun(X, Y)
    f = a[0] * ux + a[1] * uy - (kx * ux + ky * uy + k * (-2 * pi ** 2 * u))
    p = W.uniform_grid(n, 2, a=a, f=f)
    p.kx, p.ky, p.kz = k.copy(), k.copy(), k.copy()
    A, b = O.fv_assemble(p)
    uh = sla.spsolve(_sp(A).tocsc(), b)
    return np.sqrt(np.mean((uh - u) ** 2))


def _mms_3d(O, n):
    pi = np.pi
    xs = (np.arange(n) + 0.5) / n
    Z, Y, X = np.meshgrid(xs, xs, xs, indexing="ij")
    X, Y, Z = X.ravel(), Y.ravel(), Z.ravel()
    u = np.cos(pi * X) * np.sin(pi * Y) * np.cos(pi * Z)
    f = 3 * pi ** 2 * u
    p = W.uniform_grid(n, 3, f=f)
    A, b = O.fv_assemble(p)
    uh = sla.spsolve(_sp(A).tocsc(), b)
    return np.sqrt(np.mean((uh - u) ** 2))


CONST = lambda x, y: (np.ones_like(x), 0 * x, 0 * x)
EXPK = lambda x, y: (np.exp(x + 0.5 * y), np.exp(x + 0.5 * y), 0.5 * np.exp(x + 0.5 * y))


@pytest.mark.parametrize("kfun", [CONST, EXPK])
def test_order_two_for_diffusion(oracle_lib, kfun):
    e = [_mms_2d(oracle_lib, n, (0.0, 0.0), kfun) for n in (32, 64, 128)]
    orders = np.log2(np.array(e[:-1]) / np.array(e[1:]))
    assert np.all(np.abs(orders - 2.0) < 0.1), orders


def test_order_two_3d(oracle_lib):
    e = [_mms_3d(oracle_lib, n) for n in (8, 16, 32)]
    orders = np.log2(np.array(e[:-1]) / np.array(e[1:]))
    assert np.all(np.abs(orders - 2.0) < 0.15), orders


@pytest.mark.parametrize("a", [(1.0, 0.5), (40.0, 20.0)])
def test_order_one_for_upwind(oracle_lib, a):
    e = [_mms_2d(oracle_lib, n, a, CONST) for n in (32, 64, 128, 256)]
    orders = np.log2(np.array(e[:-1]) / np.array(e[1:]))
    assert abs(orders[-1] - 1.0) < 0.1, orders
    assert np.all((orders > 0.8) & (orders < 1.2)), orders


def test_m_matrix_pure_diffusion(oracle_lib):
    O = oracle_lib
    p = W.block_kappa_grid(24, 2, 4, -4, 4, 11, velocity=("const", (0.0, 0.0)))
    A, _ = O.fv_assemble(p)
    D = A.dense()
    assert np.array_equal(D, D.T)
    assert np.all(np.diag(D) > 0)
    off = D - np.diag(np.diag(D))
    assert np.all(off <= 0)
    rs = D.sum(axis=1)
    # row sums: Dirichlet transmissibility 2*kappa_y on the y = 0 and y = 1 rows, else 0
    n = 24
    j = np.arange(n * n) // n
    expect = np.where((j == 0) | (j == n - 1), 2 * p.ky, 0.0)
    assert np.allclose(rs, expect, rtol=1e-12, atol=1e-12 * np.abs(np.diag(D)).max())
    assert np.linalg.eigvalsh(D).min() > 0


def test_convection_row_sums_nonnegative(oracle_lib):
    """Upwind with a discretely divergence-free field: off-diagonals <= 0 and
    every row sum >= 0 (weak diagonal dominance), so the M-matrix criterion
    of Section 2.1 applies."""
    O = oracle_lib
    for p in (W.c2_rotating_2d_1024(n=32), W.c1_block_2d_64(), W.c3_aniso_3d_128(n=8)):
        A, _ = O.fv_assemble(p)
        S = _sp(A)
        d = S.diagonal()
        off = S - sp.diags(d)
        assert off.data.max() <= 0
        rs = np.asarray(S.sum(axis=1)).ravel()
        assert rs.min() >= -1e-13 * d.max()


def test_grad_logk_finite_difference(oracle_lib):
    """dL/dlog(kappa) for L = ||x - x_t||^2 against central differences
    (dense solves, step 1e-6 in log kappa)."""
    O = oracle_lib
    p = W.block_kappa_grid(6, 2, 2, -1, 1, 5, velocity=("const", (1.0, 0.5)))
    rng = np.random.default_rng(0)
    xt = rng.standard_normal(p.n)

    def loss(logk):
        q = W.GridProblem(**{**p.__dict__})
        q.kx = np.exp(logk); q.ky = np.exp(logk); q.kz = np.exp(logk)
        A, b = O.fv_assemble(q)
        x = np.linalg.solve(A.dense(), b)
        return np.sum((x - xt) ** 2), A, x

    logk = np.log(p.kx)
    L0, A, x = loss(logk)
    lam = np.linalg.solve(A.dense().T, 2 * (x - xt))
    gx, gy = O.fv_grad_logk(p, lam, x)
    g = gx + gy                       # isotropic: one parameter drives both axes
    h = 1e-6
    fd = np.array([(loss(logk + h * e)[0] - loss(logk - h * e)[0]) / (2 * h)
                   for e in np.eye(p.n)])
    assert np.allclose(g, fd, rtol=1e-5, atol=1e-7 * np.abs(fd).max())
