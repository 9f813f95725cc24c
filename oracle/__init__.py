"""CPU oracle for the matching-aggregation two-grid AMG + FGMRES solver.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The product
path (``paper_1105_3468_gb300``) never imports it and never falls back to it.

The arithmetic lives in ``amg_oracle.c`` (plain single-threaded FP64 C,
``-O2 -ffp-contract=off``); this module compiles it on demand with gcc and
wraps it with ctypes and numpy.  Each wrapper names the paper passage its C
function follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from typing import NamedTuple, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "amg_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libamg_oracle.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, EBREAKDOWN, ENUMERIC, ENOTCONV, ELIMIT = 0, 1, 5, 6, 7, 8


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2 -ffp-contract=off)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-Wall", "-Wno-unused-function", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
            i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
            f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
            vp = C.c_void_p
            L.or_mix64.restype = C.c_uint64
            L.or_mix64.argtypes = [C.c_uint64]
            L.or_fv_assemble.restype = C.c_int64
            L.or_fv_assemble.argtypes = [C.c_int] * 4 + [f64p] * 7 + [i64p, i32p, f64p, f64p]
            L.or_fv_grad_logk.restype = C.c_int
            L.or_fv_grad_logk.argtypes = [C.c_int] * 4 + [f64p] * 5 + [f64p] * 3
            L.or_spmv.argtypes = [C.c_int, i64p, i32p, f64p, f64p, f64p]
            L.or_spmv_t.argtypes = [C.c_int, i64p, i32p, f64p, f64p, f64p]
            L.or_dot.restype = C.c_double
            L.or_dot.argtypes = [C.c_int, f64p, f64p]
            L.or_check_csr.restype = C.c_int
            L.or_check_csr.argtypes = [C.c_int, i64p, i32p]
            L.or_edge_weight.restype = C.c_double
            L.or_edge_weight.argtypes = [i64p, i32p, f64p, C.c_int, C.c_int]
            L.or_edge_hash.restype = C.c_uint64
            L.or_edge_hash.argtypes = [C.c_int, C.c_int, C.c_uint64]
            L.or_match.restype = C.c_int64
            L.or_match.argtypes = [C.c_int, i64p, i32p, f64p, C.c_uint64, C.c_int, i32p]
            L.or_edge_key_weight.restype = C.c_double
            L.or_edge_key_weight.argtypes = [i64p, i32p, f64p, C.c_int, C.c_int, C.c_int]
            L.or_aggregate.restype = C.c_int
            L.or_aggregate.argtypes = [C.c_int, i32p, i32p]
            L.or_galerkin.restype = C.c_int64
            L.or_galerkin.argtypes = [C.c_int, i64p, i32p, f64p, i32p, C.c_int, i64p, i32p, f64p]
            L.or_color.restype = C.c_int
            L.or_color.argtypes = [C.c_int, i64p, i32p, C.c_int, C.c_uint64, i32p]
            L.or_ilu0.restype = C.c_int
            L.or_ilu0.argtypes = [C.c_int, i64p, i32p, f64p, i32p, f64p]
            L.or_ilu_solve.argtypes = [C.c_int, i64p, i32p, f64p, i32p, f64p, f64p]
            L.or_ilu_solve_t.argtypes = [C.c_int, i64p, i32p, f64p, i32p, f64p, f64p]
            L.or_ilut.restype = vp
            L.or_ilut.argtypes = [C.c_int, i64p, i32p, f64p, C.c_double, C.POINTER(C.c_int)]
            L.or_ilut_nnz.restype = C.c_int64
            L.or_ilut_nnz.argtypes = [vp]
            L.or_ilut_get.argtypes = [vp, i64p, i32p, f64p]
            L.or_ilut_solve.argtypes = [vp, f64p, f64p]
            L.or_ilut_free.argtypes = [vp]
            L.or_setup.restype = vp
            L.or_setup.argtypes = [C.c_int, i64p, i32p, f64p, i32p, C.c_double, C.c_uint64,
                                   C.POINTER(C.c_int)]
            L.or_ilut_solve_t.argtypes = [vp, f64p, f64p]
            L.or_free.argtypes = [vp]
            L.or_hier_nlev.restype = C.c_int
            L.or_hier_nlev.argtypes = [vp]
            L.or_hier_level_info.argtypes = [vp, C.c_int, i32p]
            L.or_hier_nnz.restype = C.c_int64
            L.or_hier_nnz.argtypes = [vp, C.c_int]
            L.or_hier_matrix.argtypes = [vp, C.c_int, i64p, i32p, f64p]
            L.or_hier_agg.restype = C.c_int
            L.or_hier_agg.argtypes = [vp, C.c_int, C.c_int, i32p]
            L.or_hier_pass_n.restype = C.c_int
            L.or_hier_pass_n.argtypes = [vp, C.c_int, C.c_int]
            L.or_hier_mid_nnz.restype = C.c_int64
            L.or_hier_mid_nnz.argtypes = [vp, C.c_int, C.c_int]
            L.or_hier_mid.argtypes = [vp, C.c_int, C.c_int, i64p, i32p, f64p]
            L.or_hier_colors.argtypes = [vp, C.c_int, i32p]
            L.or_hier_lu.argtypes = [vp, C.c_int, f64p]
            L.or_restrict.argtypes = [vp, C.c_int, f64p, f64p]
            L.or_level_solve.argtypes = [vp, C.c_int, f64p, f64p, C.c_int]
            L.or_smooth.argtypes = [vp, C.c_int, f64p, f64p, C.c_int]
            L.or_precond_level.argtypes = [vp, C.c_int, f64p, f64p, C.c_int]
            L.or_precond.argtypes = [vp, f64p, f64p]
            L.or_precond_t.argtypes = [vp, f64p, f64p]
            L.or_fgmres.restype = C.c_int
            L.or_fgmres.argtypes = [vp, C.c_int, vp, vp, vp, f64p, f64p, C.c_double, C.c_int,
                                    C.c_int, C.c_int, f64p, C.c_int, i32p, f64p]
            _lib = L
    return _lib


class Csr(NamedTuple):
    n: int
    row_ptr: np.ndarray   # int64 [n+1]
    col: np.ndarray       # int32 [nnz]
    val: np.ndarray       # float64 [nnz]

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def dense(self) -> np.ndarray:
        D = np.zeros((self.n, self.n))
        for i in range(self.n):
            for e in range(self.row_ptr[i], self.row_ptr[i + 1]):
                D[i, self.col[e]] += self.val[e]
        return D


def as_csr(A) -> Csr:
    """Normalise any object with n/row_ptr/col/val (or a dense array)."""
    if isinstance(A, np.ndarray):
        n = A.shape[0]
        rows, cols = np.nonzero(A)
        rp = np.zeros(n + 1, np.int64)
        np.cumsum(np.bincount(rows, minlength=n), out=rp[1:])
        return Csr(n, rp, cols.astype(np.int32), A[rows, cols].astype(np.float64))
    return Csr(int(A.n), np.ascontiguousarray(A.row_ptr, dtype=np.int64),
               np.ascontiguousarray(A.col, dtype=np.int32),
               np.ascontiguousarray(A.val, dtype=np.float64))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------- O1
def fv_assemble(prob):
    """Cell-centred FV matrix and right-hand side of eq. (2) (Section 1)."""
    L = lib()
    n = prob.nx * prob.ny * prob.nz
    cap = (2 * prob.dim + 1) * n
    rp = np.zeros(n + 1, np.int64)
    ci = np.zeros(cap, np.int32)
    v = np.zeros(cap)
    b = np.zeros(n)
    fz = prob.fz if prob.dim == 3 else np.zeros(1)
    nnz = L.or_fv_assemble(prob.dim, prob.nx, prob.ny, prob.nz, _f64(prob.kx), _f64(prob.ky),
                           _f64(prob.kz), _f64(prob.fx), _f64(prob.fy), _f64(fz), _f64(prob.f),
                           rp, ci, v, b)
    if nnz < 0:
        raise ValueError("or_fv_assemble: invalid grid")
    return Csr(n, rp, ci[:nnz].copy(), v[:nnz].copy()), b


def fv_grad_logk(prob, lam, x):
    """dL/dlog(kappa_axis) per cell from the adjoint lambda and solution x."""
    L = lib()
    n = prob.nx * prob.ny * prob.nz
    gx, gy = np.zeros(n), np.zeros(n)
    gz = np.zeros(n) if prob.dim == 3 else np.zeros(1)
    kz = prob.kz if prob.dim == 3 else np.zeros(1)
    st = L.or_fv_grad_logk(prob.dim, prob.nx, prob.ny, prob.nz, _f64(prob.kx), _f64(prob.ky),
                           _f64(kz), _f64(lam), _f64(x), gx, gy, gz)
    assert st == OK
    return (gx, gy, gz) if prob.dim == 3 else (gx, gy)


# ---------------------------------------------------------------- sparse basics
def spmv(A, x, transpose=False):
    A = as_csr(A)
    y = np.zeros(A.n)
    (lib().or_spmv_t if transpose else lib().or_spmv)(A.n, A.row_ptr, A.col, A.val, _f64(x), y)
    return y


def dot(a, b) -> float:
    """Inner product of the Arnoldi process, as if in twice the working
    precision (Dot2 of Ogita, Rump and Oishi, 2005)."""
    a, b = _f64(a), _f64(b)
    assert a.shape == b.shape
    return float(lib().or_dot(len(a), a, b))


def check_csr(A) -> int:
    A = as_csr(A)
    return lib().or_check_csr(A.n, A.row_ptr, A.col)


def mix64(z: int) -> int:
    return int(lib().or_mix64(z & 0xFFFFFFFFFFFFFFFF))


def edge_weight(A, u, v) -> float:
    A = as_csr(A)
    return float(lib().or_edge_weight(A.row_ptr, A.col, A.val, u, v))


def edge_key_weight(A, u, v, scaled: int = 1) -> float:
    """Edge weight in the matching key (O2): plain, or divided by the
    geometric mean of the two endpoints' diagonal magnitudes."""
    A = as_csr(A)
    return float(lib().or_edge_key_weight(A.row_ptr, A.col, A.val, u, v, scaled))


def edge_hash(u, v, seed=0) -> int:
    return int(lib().or_edge_hash(u, v, seed))


# ---------------------------------------------------------------- O2-O4
MATCH_PLAIN, MATCH_SCALED = 0, 1


def match(A, seed: int = 0, weight: int = MATCH_SCALED):
    """Greedy heavy-edge matching (Section 2 aggregation by matching)."""
    A = as_csr(A)
    mate = np.zeros(A.n, np.int32)
    lib().or_match(A.n, A.row_ptr, A.col, A.val, seed, weight, mate)
    return mate


def aggregate(mate):
    """Aggregates from a matching, numbered by smallest member (eq. (4))."""
    mate = np.ascontiguousarray(mate, dtype=np.int32)
    agg = np.zeros(mate.size, np.int32)
    nc = lib().or_aggregate(mate.size, mate, agg)
    return agg, nc


def galerkin(A, agg, nc):
    """A_c = P^T A P, entrywise sum of Section 2, fixed summation order."""
    A = as_csr(A)
    agg = np.ascontiguousarray(agg, dtype=np.int32)
    rp = np.zeros(nc + 1, np.int64)
    ci = np.zeros(max(1, A.nnz), np.int32)
    v = np.zeros(max(1, A.nnz))
    m = lib().or_galerkin(A.n, A.row_ptr, A.col, A.val, agg, nc, rp, ci, v)
    return Csr(nc, rp, ci[:m].copy(), v[:m].copy())


# ---------------------------------------------------------------- O5
HASH_JP, FIRST_FIT = 0, 1


def color(A, mode: int = HASH_JP, seed: int = 0):
    A = as_csr(A)
    c = np.zeros(A.n, np.int32)
    nc = lib().or_color(A.n, A.row_ptr, A.col, mode, seed, c)
    return c, nc


def ilu0(A, colors):
    """ILU(0) in the colour-major order (Algorithm 1, smoother setup)."""
    A = as_csr(A)
    lu = np.zeros(max(1, A.nnz))
    st = lib().or_ilu0(A.n, A.row_ptr, A.col, A.val, np.ascontiguousarray(colors, dtype=np.int32), lu)
    return lu[:A.nnz].copy(), st


class Ilut:
    """ILUT(tau) factors of A in natural order (Section 2: the inexact
    coarse factorisation A~_c = L~_c U~_c): `F` holds row i's L~ part
    (unit diagonal implied) and then its U~ part, ascending columns."""

    def __init__(self, A, tau: float):
        A = as_csr(A)
        st = C.c_int(0)
        self._h = lib().or_ilut(A.n, A.row_ptr, A.col, A.val, float(tau), C.byref(st))
        self.status = st.value
        if not self._h:
            raise ValueError(f"or_ilut failed with status {st.value}")
        nnz = int(lib().or_ilut_nnz(self._h))
        rp = np.zeros(A.n + 1, np.int64)
        ci = np.zeros(max(1, nnz), np.int32)
        v = np.zeros(max(1, nnz))
        lib().or_ilut_get(self._h, rp, ci, v)
        self.F = Csr(A.n, rp, ci[:nnz].copy(), v[:nnz].copy())
        self.n = A.n

    def factors(self):
        """Dense (L~, U~)."""
        D = self.F.dense()
        Lf = np.tril(D, -1) + np.eye(self.n)
        return Lf, np.triu(D)

    def solve(self, z, transpose: bool = False):
        t = np.zeros(self.n)
        (lib().or_ilut_solve_t if transpose else lib().or_ilut_solve)(self._h, _f64(z), t)
        return t

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().or_ilut_free(h)
            self._h = None


def ilu_solve(A, lu, colors, z, transpose=False):
    A = as_csr(A)
    t = np.zeros(A.n)
    fn = lib().or_ilu_solve_t if transpose else lib().or_ilu_solve
    fn(A.n, A.row_ptr, A.col, _f64(lu), np.ascontiguousarray(colors, dtype=np.int32), _f64(z), t)
    return t


# ---------------------------------------------------------------- hierarchy + solve
ORDER_COLOR, ORDER_NATURAL = 0, 1
COARSE_RECURSIVE, COARSE_ILUT = 0, 1


class Options(NamedTuple):
    """Setup options (defaults: the configuration used throughout)."""
    passes: int = 2           # matching passes per level (aggregates <= 2^passes)
    coarse_inner: int = 5     # Richardson steps of the level-1 coarse solve
    deep_inner: int = 1       # Richardson steps on deeper levels
    dense_max: int = 4096     # a level this small is solved exactly (dense inverse)
    max_levels: int = 12
    order_fine: int = ORDER_NATURAL
    order_coarse: int = ORDER_COLOR
    coloring: int = HASH_JP
    coarse_solver: int = COARSE_RECURSIVE   # COARSE_ILUT: two-grid, ILUT on level 1 (Section 2)
    ilut_tau: float = 1e-6    # drop tolerance of the ILUT two-grid (the paper's choice)
    seed: int = 0
    match_weight: int = 1     # MATCH_SCALED (default) or MATCH_PLAIN edge weights


class Hierarchy:
    """Setup phase of Algorithm 1, applied level by level (matching passes,
    Galerkin products, ILU(0) smoothers, dense LU on the last level)."""

    def __init__(self, A, opts: Optional[Options] = None, **kw):
        opts = (opts or Options())._replace(**kw)
        self.opts = opts
        self.A = as_csr(A)
        st = C.c_int(0)
        o = np.array([opts.passes, opts.coarse_inner, opts.deep_inner, opts.dense_max,
                      opts.max_levels, opts.order_fine, opts.order_coarse, opts.coloring,
                      opts.coarse_solver, opts.match_weight], np.int32)
        self._h = lib().or_setup(self.A.n, self.A.row_ptr, self.A.col, self.A.val, o,
                                 float(opts.ilut_tau), opts.seed, C.byref(st))
        self.status = st.value
        if not self._h:
            raise ValueError(f"or_setup failed with status {st.value}")
        self.nlev = lib().or_hier_nlev(self._h)
        self.levels = []
        for l in range(self.nlev):
            info = np.zeros(8, np.int32)
            lib().or_hier_level_info(self._h, l, info)
            self.levels.append(dict(n=int(info[0]), nnz=int(lib().or_hier_nnz(self._h, l)),
                                    ncol=int(info[2]), dense=bool(info[3]), npass=int(info[4]),
                                    n_pass1=int(info[5]), n_next=int(info[6]), has_lu=bool(info[7])))
        self.n = self.levels[0]["n"]
        self.nc = self.levels[1]["n"] if self.nlev > 1 else self.n

    def __del__(self):
        if getattr(self, "_h", None):
            lib().or_free(self._h)
            self._h = None

    def matrix(self, l: int) -> Csr:
        n, nnz = self.levels[l]["n"], self.levels[l]["nnz"]
        rp = np.zeros(n + 1, np.int64)
        ci = np.zeros(max(1, nnz), np.int32)
        v = np.zeros(max(1, nnz))
        lib().or_hier_matrix(self._h, l, rp, ci, v)
        return Csr(n, rp, ci[:nnz], v[:nnz])

    def coarse(self) -> Csr:
        return self.matrix(1)

    def agg(self, l: int = 0, p: int = 0):
        n = self.levels[l]["n"] if p == 0 else lib().or_hier_pass_n(self._h, l, p - 1)
        out = np.zeros(n, np.int32)
        assert lib().or_hier_agg(self._h, l, p, out) == OK
        return out

    def mid(self, l: int, p: int) -> Csr:
        nnz = lib().or_hier_mid_nnz(self._h, l, p)
        n = lib().or_hier_pass_n(self._h, l, p)
        rp = np.zeros(n + 1, np.int64)
        ci = np.zeros(max(1, nnz), np.int32)
        v = np.zeros(max(1, nnz))
        lib().or_hier_mid(self._h, l, p, rp, ci, v)
        return Csr(n, rp, ci[:nnz], v[:nnz])

    def colors(self, l: int):
        out = np.zeros(self.levels[l]["n"], np.int32)
        lib().or_hier_colors(self._h, l, out)
        return out

    def lu(self, l: int):
        nnz = self.levels[l]["nnz"]
        out = np.zeros(max(1, nnz))
        lib().or_hier_lu(self._h, l, out)
        return out[:nnz]

    def restrict(self, l: int, r):
        out = np.zeros(self.levels[l + 1]["n"])
        lib().or_restrict(self._h, l, _f64(r), out)
        return out

    def level_solve(self, l: int, h, transpose=False):
        """C_l(h): the inexact solve of level l >= 1 (dense inverse on the last level)."""
        out = np.zeros(self.levels[l]["n"])
        lib().or_level_solve(self._h, l, _f64(h), out, int(transpose))
        return out

    def smooth(self, l: int, z, transpose=False):
        out = np.zeros(self.levels[l]["n"])
        lib().or_smooth(self._h, l, _f64(z), out, int(transpose))
        return out

    def precond(self, z, transpose=False, level: int = 0):
        """q = B~^{-1} z (Algorithm 1, the preconditioner application) at a level, or its transpose."""
        out = np.zeros(self.levels[level]["n"])
        lib().or_precond_level(self._h, level, _f64(z), out, int(transpose))
        return out

    def fgmres(self, b, x0=None, tol=1e-8, restart=30, maxit=600, transpose=False):
        return fgmres(None, b, x0, tol, restart, maxit, transpose, hier=self)


class SolveInfo(NamedTuple):
    status: int
    iters: int
    restarts: int
    relres: float
    hist: np.ndarray


def fgmres(A, b, x0=None, tol=1e-8, restart=30, maxit=600, transpose=False, hier=None):
    """Right-preconditioned FGMRES(m) (Algorithm 1 Krylov loop, Section 3 stop rule).

    ``hier=None`` runs with the identity preconditioner on ``A``.
    """
    b = _f64(b)
    n = b.size
    x = np.zeros(n) if x0 is None else _f64(x0).copy()
    cap = maxit + 2
    hist = np.zeros(cap)
    oi = np.zeros(3, np.int32)
    od = np.zeros(1)
    if hier is not None:
        st = lib().or_fgmres(hier._h, n, None, None, None, b, x, tol, restart, maxit,
                             int(transpose), hist, cap, oi, od)
    else:
        A = as_csr(A)
        st = lib().or_fgmres(None, A.n, A.row_ptr.ctypes.data, A.col.ctypes.data,
                             A.val.ctypes.data, b, x, tol, restart, maxit, int(transpose),
                             hist, cap, oi, od)
    return x, SolveInfo(st, int(oi[0]), int(oi[1]), float(od[0]), hist[:oi[2]].copy())
