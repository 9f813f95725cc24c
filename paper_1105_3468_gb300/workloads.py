"""Seeded synthetic inputs for the matching-aggregation two-grid AMG solver.

This module only draws and lays out input data: per-cell conductivities, the
discrete velocity field as face fluxes, source terms, right-hand sides and
random sparse test matrices.  It holds none of the solver's arithmetic and none
of the finite-volume discretisation (Section 1, eq. (2) of the paper): the CPU
oracle and the CUDA path each assemble their own matrix from these arrays.

Conventions
-----------
* Cells of an ``nx x ny (x nz)`` grid on ``[0,1]^d`` with ``h = 1/n`` are
  numbered ``idx = i + nx*(j + ny*k)`` (x fastest).
* ``fx[i + (nx+1)*(j + ny*k)]`` is the integrated velocity flux through the
  x-face at ``x = i*h`` in the +x direction (face area folded in), likewise
  ``fy`` (``i + nx*(j + (ny+1)*k)``) and ``fz`` (``i + nx*(j + ny*k)``).
* ``kx, ky, kz`` hold the diagonal of the conductivity tensor per cell; an
  isotropic field repeats the same array three times.
* Dirichlet u = 0 holds on the y = 0 and y = 1 faces, Neumann elsewhere
  (Section 1, the paragraph after eq. (2)).

All draws use ``numpy.random.default_rng(seed)`` (PCG64).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np


@dataclasses.dataclass
class GridProblem:
    """A cell-centred convection-diffusion problem on a uniform grid."""

    dim: int
    nx: int
    ny: int
    nz: int
    kx: np.ndarray
    ky: np.ndarray
    kz: np.ndarray
    fx: np.ndarray
    fy: np.ndarray
    fz: np.ndarray
    f: np.ndarray
    name: str = ""

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def h(self) -> float:
        return 1.0 / self.nx

    def cell_centres(self) -> Tuple[np.ndarray, ...]:
        """Cell-centre coordinates, each flattened with x fastest."""
        xs = (np.arange(self.nx) + 0.5) / self.nx
        ys = (np.arange(self.ny) + 0.5) / self.ny
        if self.dim == 2:
            Y, X = np.meshgrid(ys, xs, indexing="ij")
            return X.ravel(), Y.ravel()
        zs = (np.arange(self.nz) + 0.5) / self.nz
        Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
        return X.ravel(), Y.ravel(), Z.ravel()


@dataclasses.dataclass
class CsrMatrix:
    """A square FP64 CSR matrix: int64 row pointers, int32 sorted columns."""

    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])


# --------------------------------------------------------------------------
# velocity fields as face fluxes
# --------------------------------------------------------------------------

def constant_fluxes(dim: int, n: int, a: Sequence[float]):
    """Face fluxes of a constant velocity ``a``: flux = h^(d-1) * a_axis."""
    h = 1.0 / n
    area = h ** (dim - 1)
    nz = n if dim == 3 else 1
    fx = np.full((nx_faces := (n + 1) * n * nz), area * float(a[0]))
    fy = np.full(n * (n + 1) * nz, area * float(a[1]))
    if dim == 3:
        fz = np.full(n * n * (n + 1), area * float(a[2]))
    else:
        fz = np.zeros(0)
    assert fx.size == nx_faces
    return fx, fy, fz


def rotating_fluxes_2d(n: int, amplitude: float = 10.0):
    """Exact face integrals of a = amplitude*(sin px cos py, -cos px sin py).

    The field is the curl of the stream function
    psi = (amplitude/pi) sin(pi x) sin(pi y); the flux through a face is the
    difference of psi between its end points, so the discrete field is
    divergence free up to rounding.
    """
    xs = np.arange(n + 1) / n
    s = np.sin(np.pi * xs)
    psi = (amplitude / np.pi) * np.outer(s, s)        # psi[j, i] at (x_i, y_j)
    fx = psi[1:, :] - psi[:-1, :]                       # (ny, nx+1): x-face i, rows j
    fy = -(psi[:, 1:] - psi[:, :-1])                    # (ny+1, nx)
    return np.ascontiguousarray(fx).ravel(), np.ascontiguousarray(fy).ravel(), np.zeros(0)


# --------------------------------------------------------------------------
# block-kappa grid problems
# --------------------------------------------------------------------------

def block_kappa_grid(n: int, dim: int, blocks: int, log10_lo: float, log10_hi: float,
                     seed: int, anisotropic: bool = False,
                     velocity=("const", (1.0, 0.5)), name: str = "") -> GridProblem:
    """Piecewise-constant conductivity on a ``blocks^d`` block grid.

    Each block draws ``10**U(lo, hi)`` (one value, or one per axis x, y, z when
    anisotropic), blocks enumerated with x fastest.  Cell ``i`` along an axis
    lies in block ``(i*blocks)//n``.  f = 1.
    """
    rng = np.random.default_rng(seed)
    nb = blocks ** dim
    if anisotropic:
        u = rng.uniform(log10_lo, log10_hi, size=(nb, 3))
    else:
        u = rng.uniform(log10_lo, log10_hi, size=nb)
    kb = 10.0 ** u
    bi = (np.arange(n) * blocks) // n
    if dim == 2:
        BY, BX = np.meshgrid(bi, bi, indexing="ij")
        bid = (BX + blocks * BY).ravel()
        nz = 1
    else:
        BZ, BY, BX = np.meshgrid(bi, bi, bi, indexing="ij")
        bid = (BX + blocks * (BY + blocks * BZ)).ravel()
        nz = n
    if anisotropic:
        kx = np.ascontiguousarray(kb[bid, 0])
        ky = np.ascontiguousarray(kb[bid, 1])
        kz = np.ascontiguousarray(kb[bid, 2])
    else:
        kx = np.ascontiguousarray(kb[bid])
        ky = kx.copy()
        kz = kx.copy()
    kind, par = velocity
    if kind == "const":
        fx, fy, fz = constant_fluxes(dim, n, par)
    elif kind == "rotating":
        assert dim == 2
        fx, fy, fz = rotating_fluxes_2d(n, float(par))
    else:
        raise ValueError(kind)
    f = np.ones(n ** dim)
    return GridProblem(dim, n, n, nz, kx, ky, kz, fx, fy, fz, f, name=name)


def uniform_grid(n: int, dim: int, kappa: float = 1.0, a=(0.0, 0.0, 0.0),
                 f: Optional[np.ndarray] = None) -> GridProblem:
    """Constant conductivity and velocity; f defaults to 1."""
    N = n ** dim
    k = np.full(N, float(kappa))
    fx, fy, fz = constant_fluxes(dim, n, a)
    return GridProblem(dim, n, n, n if dim == 3 else 1, k, k.copy(), k.copy(), fx, fy, fz,
                       np.ones(N) if f is None else np.asarray(f, dtype=np.float64))


# --------------------------------------------------------------------------
# the paper's own discontinuous test cases (Section 4, test cases)
# --------------------------------------------------------------------------

def dc_kappa(n: int, dim: int) -> np.ndarray:
    """Conductivity of the DC1 cases at the cell centres x: kappa = 1000 ([10 x_2] + 1)
    where [10 x_i] is even for every axis i, 1 elsewhere ([.] = integer part; x_2 is the
    second coordinate).  Isolated high-permeability zones whose value grows with x_2."""
    c = (np.arange(n) + 0.5) / n
    cells = np.floor(10.0 * c).astype(np.int64)
    even = (cells % 2) == 0
    if dim == 2:
        ex, ey = np.meshgrid(even, even, indexing="xy")           # ex varies along x (fastest)
        _, cy = np.meshgrid(cells, cells, indexing="xy")
        zone = ex & ey
        k = np.where(zone, 1000.0 * (cy + 1), 1.0)
    else:
        ez, ey, ex = np.meshgrid(even, even, even, indexing="ij")  # index order (z, y, x): x fastest
        _, cy, _ = np.meshgrid(cells, cells, cells, indexing="ij")
        zone = ex & ey & ez
        k = np.where(zone, 1000.0 * (cy + 1), 1.0)
    return k.reshape(-1).astype(np.float64)


def dc_problem(n: int, dim: int, velocity: float = 0.0) -> GridProblem:
    """DC1 (velocity 0) and DCC1 / DCC2 (a = velocity in every direction; the paper
    uses 1000) on an n^dim grid, f = 1."""
    k = dc_kappa(n, dim)
    fx, fy, fz = constant_fluxes(dim, n, [velocity] * dim)
    name = ("dcc" if velocity else "dc1") + f"-{dim}d-{n}"
    return GridProblem(dim, n, n, n if dim == 3 else 1, k, k.copy(), k.copy(), fx, fy, fz,
                       np.ones(n ** dim), name=name)


# --------------------------------------------------------------------------
# the five workloads
# --------------------------------------------------------------------------

def c1_block_2d_64(seed: int = 1) -> GridProblem:
    """64x64 cells, 8x8 blocks of 10^U(-4,4), a = (1, 0.5), f = 1."""
    return block_kappa_grid(64, 2, 8, -4.0, 4.0, seed, velocity=("const", (1.0, 0.5)),
                            name="fv2d-64x64-blockkappa")


def c2_rotating_2d_1024(seed: int = 2, n: int = 1024) -> GridProblem:
    """1024^2 cells, 64x64 blocks of 10^U(-4,4), rotating velocity x10."""
    return block_kappa_grid(n, 2, max(1, n // 16), -4.0, 4.0,
                            seed, velocity=("rotating", 10.0), name=f"fv2d-{n}x{n}-rotating")


def c3_aniso_3d_128(seed: int = 3, n: int = 128) -> GridProblem:
    """128^3 cells, 16^3 blocks, each axis 10^U(-3,3), a = (1, 1, 1)."""
    return block_kappa_grid(n, 3, max(1, n // 8), -3.0, 3.0, seed, anisotropic=True,
                            velocity=("const", (1.0, 1.0, 1.0)), name=f"fv3d-{n}^3-aniso")


def c4_adjoint_2d(seed: int = 4, n: int = 512) -> Tuple[GridProblem, np.ndarray]:
    """512^2 block-kappa problem (32x32 blocks of 16^2) and its target field.

    x_target = sum_{m=1..4} c_m sin(p_m pi x + phi_m) sin(q_m pi y) at the
    cell centres, with c ~ N(0,1), p, q in {1,2,3}, phi ~ U(0, 2 pi).  The
    16^2 finite-difference instance uses 2x2 blocks of 8^2 (``n=16``).
    """
    blocks = max(1, n // 16)
    prob = block_kappa_grid(n, 2, blocks, -4.0, 4.0, seed, velocity=("const", (1.0, 0.5)),
                            name=f"fv2d-{n}x{n}-adjoint")
    rng = np.random.default_rng(seed + 1000)
    c = rng.standard_normal(4)
    p = rng.integers(1, 4, size=4)
    q = rng.integers(1, 4, size=4)
    phi = rng.uniform(0.0, 2.0 * np.pi, size=4)
    X, Y = prob.cell_centres()
    xt = np.zeros(prob.n)
    for m in range(4):
        xt += c[m] * np.sin(p[m] * np.pi * X + phi[m]) * np.sin(q[m] * np.pi * Y)
    return prob, xt


def rhs_normal(n: int, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal(n)


# --------------------------------------------------------------------------
# random geometric graph matrices (stand-ins for the paper's sparse collection)
# --------------------------------------------------------------------------

def rgg_matrix(n: int, nnz_per_row: int, seed: int, perturb: float = 0.1,
               shift: float = 1e-2) -> CsrMatrix:
    """Nonsymmetric sparse matrix A = L + K + delta*I from a random geometric graph.

    n points uniform in the unit cube are joined when closer than
    r = (3*dbar/(4*pi*n))^(1/3), dbar = nnz_per_row - 1 (expected degree in
    the interior).  L = D - W is the unit-weight graph Laplacian,
    K_ij = perturb*xi_ij*W_ij = -K_ji with xi ~ U(-1,1) for i < j, and
    delta = shift * mean(diag L).
    """
    from scipy.spatial import cKDTree

    rng = np.random.default_rng(seed)
    pts = rng.random((n, 3))
    dbar = max(1, nnz_per_row - 1)
    r = (3.0 * dbar / (4.0 * math.pi * n)) ** (1.0 / 3.0)
    pairs = cKDTree(pts).query_pairs(r, output_type="ndarray").astype(np.int64)
    if pairs.size:
        pairs = np.sort(pairs, axis=1)
        order = np.lexsort((pairs[:, 1], pairs[:, 0]))
        pairs = pairs[order]
    else:
        pairs = np.zeros((0, 2), dtype=np.int64)
    xi = rng.uniform(-1.0, 1.0, size=len(pairs))
    i, j = pairs[:, 0], pairs[:, 1]
    deg = np.bincount(np.concatenate([i, j]), minlength=n).astype(np.float64)
    delta = shift * float(deg.mean()) if n else 0.0
    if delta == 0.0:
        delta = shift
    rows = np.concatenate([i, j, np.arange(n)])
    cols = np.concatenate([j, i, np.arange(n)])
    vals = np.concatenate([-1.0 + perturb * xi, -1.0 - perturb * xi, deg + delta])
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=row_ptr[1:])
    return CsrMatrix(n, row_ptr, cols.astype(np.int32), vals.astype(np.float64),
                     name=f"rgg-{n}-d{nnz_per_row}")


# --------------------------------------------------------------------------
# batch of uneven systems
# --------------------------------------------------------------------------

@dataclasses.dataclass
class BatchSpec:
    """Recipe for one member of the uneven batch (generated lazily)."""

    kind: str          # "grid" or "rgg"
    size: int          # grid side, or RGG rows
    nnz_per_row: int   # RGG only
    seed: int


def c5_batch_specs(seed: int = 5, n_grid: int = 48, n_rgg: int = 16,
                   grid_side=(64, 512), rgg_rows=(10_000, 500_000),
                   rgg_nnz=(7, 30)) -> List[BatchSpec]:
    """48 block-kappa grids (side ~ U{64..512}) then 16 RGG matrices."""
    rng = np.random.default_rng(seed)
    sides = rng.integers(grid_side[0], grid_side[1] + 1, size=n_grid)
    rows = rng.integers(rgg_rows[0], rgg_rows[1] + 1, size=n_rgg)
    nnzr = rng.integers(rgg_nnz[0], rgg_nnz[1] + 1, size=n_rgg)
    specs = [BatchSpec("grid", int(s), 0, seed * 1000 + k) for k, s in enumerate(sides)]
    specs += [BatchSpec("rgg", int(r), int(d), seed * 1000 + n_grid + k)
              for k, (r, d) in enumerate(zip(rows, nnzr))]
    return specs


def batch_grid_problem(spec: BatchSpec) -> GridProblem:
    """Grid member of the batch: 8x8 blocks of 10^U(-4,4), a = (1, 0.5)."""
    return block_kappa_grid(spec.size, 2, 8, -4.0, 4.0, spec.seed,
                            velocity=("const", (1.0, 0.5)), name=f"batch-grid-{spec.size}")


def batch_rhs(spec: BatchSpec, n: int) -> np.ndarray:
    return rhs_normal(n, spec.seed + 7)
