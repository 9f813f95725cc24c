"""Pins of the oracle's smoother, preconditioner and Krylov solver.

Colouring / ILU(0) (Algorithm 1, smoother setup; orderings of
Section 3):
* colourings are proper and greedy (every vertex of colour c > 0 has a
  higher-priority neighbour of each colour below c); first-fit colouring of
  a 5-point (7-point) grid is the checkerboard (i+j(+k)) mod 2;
* ILU(0)'s defining property (LU)_ij = a_ij on the pattern of A, natural and
  colour-major orders; on a tridiagonal matrix ILU(0) = exact LU;
* the transposed solve is the transpose of the solve; a zero pivot reports
  a breakdown;
* for a symmetric M-matrix the ILU iteration converges (Theorem of Meijerink
  and van der Vorst quoted in Section 2.1): rho(I - S^{-1}A) < 1.
Preconditioner (eq. (5), Algorithm 1's preconditioner application):
* equals the paper's three-solve form t + f - q';
* with an exact coarse solve, (I - M^{-1}A) P = 0 (Theorem 1);
* the Richardson coarse solve equals sum_{k<m} (I - B^{-1}A)^k B^{-1};
* the transposed preconditioner is the transpose of the preconditioner;
* the dense final level solves exactly.
FGMRES (Algorithm 1 Krylov loop; stopping rule of Section 3):
* identity preconditioner with restart >= N reaches the dense solution in at
  most N steps; the least-squares residual estimate equals the true residual;
* residual estimates never increase within a cycle;
* the AMG-preconditioned solve matches dense LU; adjoint solves A^T;
* status codes: not converged, NaN input, zero right-hand side;
* inner products (Dot2): equal to the exact rational value rounded to
  nearest on well- and ill-conditioned cases, where a plain running sum is
  far off.
"""
import numpy as np
import pytest

from paper_1105_3468_gb300 import workloads as W


def _adj(A):
    D = A.dense()
    pat = (np.abs(D) > 0) | (np.abs(D.T) > 0)
    np.fill_diagonal(pat, False)
    return pat


@pytest.mark.parametrize("mode", [0, 1])
def test_colouring_proper_and_greedy(oracle_lib, mode):
    O = oracle_lib
    A, _ = O.fv_assemble(W.c3_aniso_3d_128(n=7))
    col, nc = O.color(A, mode)
    pat = _adj(A)
    n = A.n
    assert col.max() + 1 == nc
    if mode == 0:
        prio = [(O.mix64(i ^ (0 + 0x9E3779B97F4A7C15)), i) for i in range(n)]
    else:
        prio = [(0, -i) for i in range(n)]
    for u in range(n):
        nb = np.nonzero(pat[u])[0]
        assert np.all(col[nb] != col[u])
        higher = [v for v in nb if prio[v] > prio[u]]
        assert set(range(col[u])) <= set(col[higher].tolist())


def test_first_fit_is_checkerboard(oracle_lib):
    O = oracle_lib
    A, _ = O.fv_assemble(W.uniform_grid(9, 2))
    col, nc = O.color(A, O.FIRST_FIT)
    i, j = np.arange(81) % 9, np.arange(81) // 9
    assert nc == 2 and np.array_equal(col, (i + j) % 2)
    A, _ = O.fv_assemble(W.uniform_grid(5, 3))
    col, nc = O.color(A, O.FIRST_FIT)
    i, j, k = np.arange(125) % 5, (np.arange(125) // 5) % 5, np.arange(125) // 25
    assert nc == 2 and np.array_equal(col, (i + j + k) % 2)


def _factors(A, lu, colors):
    n = A.n
    order = np.lexsort((np.arange(n), colors))
    pos = np.empty(n, int)
    pos[order] = np.arange(n)
    L, U = np.eye(n), np.zeros((n, n))
    for i in range(n):
        for e in range(A.row_ptr[i], A.row_ptr[i + 1]):
            j = A.col[e]
            if pos[j] < pos[i]:
                L[i, j] = lu[e]
            else:
                U[i, j] = lu[e]
    return L, U


@pytest.mark.parametrize("order", ["natural", "colour"])
def test_ilu0_defining_property(oracle_lib, order):
    O = oracle_lib
    for p in (W.c1_block_2d_64(), W.c3_aniso_3d_128(n=6)):
        A, _ = O.fv_assemble(p)
        colors = np.zeros(A.n, np.int32) if order == "natural" else O.color(A)[0]
        lu, st = O.ilu0(A, colors)
        assert st == O.OK
        L, U = _factors(A, lu, colors)
        LU = L @ U
        D = A.dense()
        mask = D != 0
        scale = np.abs(D).max()
        assert np.abs((LU - D)[mask]).max() <= 1e-13 * scale
        # triangular structure in the elimination order
        n = A.n
        ordr = np.lexsort((np.arange(n), colors))
        assert np.allclose(np.triu(L[np.ix_(ordr, ordr)], 1), 0)
        assert np.allclose(np.tril(U[np.ix_(ordr, ordr)], -1), 0)
        z = np.random.default_rng(3).standard_normal(n)
        t = O.ilu_solve(A, lu, colors, z)
        assert np.allclose(LU @ t, z, rtol=1e-10, atol=1e-10 * np.abs(z).max())
        tt = O.ilu_solve(A, lu, colors, z, transpose=True)
        assert np.allclose(LU.T @ tt, z, rtol=1e-10, atol=1e-10 * np.abs(z).max())


def test_ilu0_exact_on_tridiagonal(oracle_lib):
    O = oracle_lib
    import scipy.linalg as sla
    rng = np.random.default_rng(5)
    n = 30
    D = np.diag(4 + rng.random(n)) + np.diag(-rng.random(n - 1), 1) + np.diag(-rng.random(n - 1), -1)
    A = O.as_csr(D)
    colors = np.zeros(n, np.int32)
    lu, st = O.ilu0(A, colors)
    L, U = _factors(A, lu, colors)
    P, Ls, Us = sla.lu(D)
    assert np.array_equal(P, np.eye(n))          # no pivoting needed
    assert np.allclose(L, Ls, rtol=1e-14, atol=1e-15) and np.allclose(U, Us, rtol=1e-14, atol=1e-15)
    z = rng.standard_normal(n)
    assert np.allclose(O.ilu_solve(A, lu, colors, z), np.linalg.solve(D, z), rtol=1e-12)


def test_ilu0_breakdown_reported(oracle_lib):
    O = oracle_lib
    D = np.array([[1.0, 1.0], [1.0, 1.0]])
    lu, st = O.ilu0(O.as_csr(D), np.zeros(2, np.int32))
    assert st == O.EBREAKDOWN


def test_ilu_iteration_converges_for_symmetric_m_matrix(oracle_lib):
    O = oracle_lib
    p = W.block_kappa_grid(10, 2, 2, -2, 2, 9, velocity=("const", (0.0, 0.0)))
    A, _ = O.fv_assemble(p)
    D = A.dense()
    for colors in (np.zeros(A.n, np.int32), O.color(A)[0]):
        lu, _ = O.ilu0(A, colors)
        Sinv = np.column_stack([O.ilu_solve(A, lu, colors, e) for e in np.eye(A.n)])
        rho = np.abs(np.linalg.eigvals(np.eye(A.n) - Sinv @ D)).max()
        assert rho < 1.0


def _dense_op(f, n):
    return np.column_stack([f(e) for e in np.eye(n)])


def _small_hier(O, **kw):
    p = W.block_kappa_grid(12, 2, 3, -2, 2, 21, velocity=("const", (1.0, 0.5)))
    A, b = O.fv_assemble(p)
    return A, b, O.Hierarchy(A, **kw)


def test_precond_equals_three_solve_form(oracle_lib):
    """Algorithm 1: S t = z; M~ f = z; M~ q' = A t; q = t + f - q'."""
    O = oracle_lib
    A, _, H = _small_hier(O, dense_max=40)
    assert H.nlev >= 3
    agg = H.agg(0)
    D = A.dense()

    def Minv(y):
        return H.level_solve(1, H.restrict(0, y))[agg]

    z = np.random.default_rng(2).standard_normal(A.n)
    t = H.smooth(0, z)
    f = Minv(z)
    qp = Minv(D @ t)
    q_paper = t + f - qp
    assert np.allclose(H.precond(z), q_paper, rtol=1e-12, atol=1e-12 * np.abs(q_paper).max())


def test_approximate_filtering_exact_coarse(oracle_lib):
    """Theorem 1: with the exact coarse solve, (I - P A_c^{-1} P^T A) P = 0."""
    O = oracle_lib
    A, _, H = _small_hier(O, dense_max=10 ** 6)
    assert H.nlev == 2 and H.levels[1]["dense"]
    agg = H.agg(0)
    D = A.dense()
    P = np.zeros((A.n, H.nc))
    P[np.arange(A.n), agg] = 1
    Minv = _dense_op(lambda y: H.level_solve(1, H.restrict(0, y))[agg], A.n)
    R = (np.eye(A.n) - Minv @ D) @ P
    assert np.abs(R).max() < 1e-10


def test_richardson_closed_form(oracle_lib):
    O = oracle_lib
    A, _, H = _small_hier(O, dense_max=40, coarse_inner=5)
    n1 = H.levels[1]["n"]
    A1 = H.matrix(1).dense()
    B1 = _dense_op(lambda v: H.precond(v, level=1), n1)
    C1 = _dense_op(lambda h: H.level_solve(1, h), n1)
    E = np.eye(n1) - B1 @ A1
    closed = sum(np.linalg.matrix_power(E, k) for k in range(5)) @ B1
    assert np.allclose(C1, closed, rtol=1e-9, atol=1e-9 * np.abs(closed).max())


def test_transposed_preconditioner(oracle_lib):
    O = oracle_lib
    A, _, H = _small_hier(O, dense_max=40)
    Bi = _dense_op(H.precond, A.n)
    BiT = _dense_op(lambda v: H.precond(v, transpose=True), A.n)
    assert np.allclose(BiT, Bi.T, rtol=1e-10, atol=1e-10 * np.abs(Bi).max())
    last = H.nlev - 1
    nL = H.levels[last]["n"]
    DL = H.matrix(last).dense()
    h = np.random.default_rng(4).standard_normal(nL)
    assert np.allclose(H.level_solve(last, h), np.linalg.solve(DL, h), rtol=1e-10)
    assert np.allclose(H.level_solve(last, h, transpose=True), np.linalg.solve(DL.T, h), rtol=1e-10)


def test_fgmres_identity_finite_termination(oracle_lib):
    O = oracle_lib
    rng = np.random.default_rng(8)
    n = 25
    D = np.diag(5 + rng.random(n)) + 0.5 * rng.standard_normal((n, n)) * (rng.random((n, n)) < 0.3)
    A = O.as_csr(D)
    b = rng.standard_normal(n)
    x, info = O.fgmres(A, b, tol=1e-13, restart=n, maxit=n)
    assert info.status == O.OK and info.iters <= n
    xe = np.linalg.solve(D, b)
    assert np.linalg.norm(x - xe) <= 1e-10 * np.linalg.norm(xe)


def test_fgmres_estimate_equals_true_residual(oracle_lib):
    O = oracle_lib
    A, b, H = _small_hier(O)
    D = A.dense()
    for k in (3, 7, 11):
        x, info = H.fgmres(b, tol=1e-30, restart=30, maxit=k)
        assert info.status == O.ENOTCONV and info.iters == k
        true = np.linalg.norm(b - D @ x) / np.linalg.norm(b)
        assert abs(info.hist[-1] - true) <= 1e-9 * true + 1e-13   # attainable: eps*||A|| ||x||/||b||
        assert abs(info.relres - true) <= 1e-10 * true + 1e-14


def test_fgmres_monotone_and_dense_agreement(oracle_lib):
    O = oracle_lib
    A, b, H = _small_hier(O, coarse_inner=1)
    x, info = H.fgmres(b, tol=1e-10, restart=4, maxit=400)
    assert info.status == O.OK
    h = info.hist
    for c in range(0, len(h) - 1, 4):     # within each 4-step cycle
        seg = h[c:c + 5]
        assert np.all(np.diff(seg) <= 1e-15 * seg[0])
    xe = np.linalg.solve(A.dense(), b)
    assert np.linalg.norm(x - xe) <= 1e-8 * np.linalg.norm(xe)


def test_fgmres_c1_converges(oracle_lib):
    O = oracle_lib
    A, b = O.fv_assemble(W.c1_block_2d_64())
    H = O.Hierarchy(A)
    x, info = H.fgmres(b, tol=1e-8)
    assert info.status == O.OK and info.iters < 60
    xe = np.linalg.solve(A.dense(), b)
    assert np.linalg.norm(x - xe) <= 1e-6 * np.linalg.norm(xe)
    assert np.linalg.norm(b - A.dense() @ x) <= 1e-8 * np.linalg.norm(b)


def test_adjoint_solve(oracle_lib):
    O = oracle_lib
    A, _, H = _small_hier(O)
    g = np.random.default_rng(6).standard_normal(A.n)
    lam, info = H.fgmres(g, tol=1e-12, transpose=True)
    assert info.status == O.OK
    le = np.linalg.solve(A.dense().T, g)
    assert np.linalg.norm(lam - le) <= 1e-9 * np.linalg.norm(le)


def test_status_codes(oracle_lib):
    O = oracle_lib
    A, b, H = _small_hier(O)
    x, info = H.fgmres(b, maxit=1)
    assert info.status == O.ENOTCONV and info.iters == 1
    bad = b.copy()
    bad[3] = np.nan
    _, info = H.fgmres(bad)
    assert info.status == O.ENUMERIC
    x, info = H.fgmres(np.zeros_like(b), x0=np.ones_like(b))
    assert info.status == O.OK and not x.any()


def _exact_dot_rounded(a, b):
    from fractions import Fraction
    ex = sum(Fraction(float(x)) * Fraction(float(y)) for x, y in zip(a, b))
    return float(ex), ex


def test_dot2_is_correctly_rounded(oracle_lib):
    O = oracle_lib
    rng = np.random.default_rng(17)
    for trial in range(60):
        n = int(rng.integers(1, 400))
        a, b = rng.standard_normal(n), rng.standard_normal(n) * 10.0 ** rng.integers(-8, 8)
        ref, _ = _exact_dot_rounded(a, b)
        assert O.dot(a, b) == ref, trial


def test_dot2_ill_conditioned(oracle_lib):
    """Sums that cancel to ~1e-12 of their terms: a plain running sum loses
    most digits, Dot2 still returns the exactly rounded value."""
    O = oracle_lib
    rng = np.random.default_rng(18)
    worst_plain = 0.0
    for trial in range(40):
        n = 200
        big = rng.standard_normal(n // 2) * 1e6
        a = np.concatenate([big, big])
        b = np.concatenate([rng.standard_normal(n // 2), np.zeros(n // 2)])
        b[n // 2:] = -b[:n // 2]                         # pairs cancel exactly ...
        b[n // 2:] += rng.standard_normal(n // 2) * 1e-12  # ... up to a small remainder
        perm = rng.permutation(n)
        a, b = a[perm], b[perm]
        ref, ex = _exact_dot_rounded(a, b)
        assert O.dot(a, b) == ref, trial
        plain = 0.0
        for x, y in zip(a, b):
            plain += x * y
        worst_plain = max(worst_plain, abs(plain - ref) / abs(ref))
    assert worst_plain > 1e-8          # the test cases are hard for a running sum
