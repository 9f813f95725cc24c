"""Pins of the oracle's ILUT(tau), the inexact factorisation of the coarse
operator (Section 2: A~_c = L~_c U~_c = ILUT(A_c); Algorithm 1 setup),
with Saad's dropping rule (tau_i = tau * ||a_i||_2) and no pivoting:

* tau = 0 keeps every nonzero: the complete LU factorisation without
  pivoting, so L~U~ reproduces A within the classical backward-error bound
  |A - L~U~| <= gamma_m |L~||U~| (Higham, Theorem 9.3; m the longest
  inner-product length), and solving with the factors solves A x = b;
* on a tridiagonal matrix (no fill) ILUT with tau = 0 equals ILU(0) in
  natural order bit for bit (same divisions and updates, in the same order);
* tau = inf keeps only the diagonal (L~ = I, U~ = diag A);
* structure and dropping rule: L~ strictly lower, U~ upper with its
  diagonal first in each row, every kept off-diagonal entry of row i at
  least tau_i in magnitude;
* the triangular solve with the factors equals the dense solve with L~U~;
* on the 64^2 block-kappa operator, fewer entries are kept and the relative
  factorisation error ||A - L~U~|| / ||A|| grows as tau grows (the trend
  of the paper's Table of ||LU - L~U~|| / ||LU||, context only);
* a hand-computed 3x3 case in which one fill entry is kept at tau = 0.01
  and dropped at tau = 0.02.
The two-grid form of Algorithm 1 with this coarse factorisation (one solve
with L~_c U~_c, level 1 the last level): with tau = 0 it equals the two-grid
preconditioner with the exact coarse inverse; its transpose is the
transpose; its coarse solve is the factor solve.
"""
import numpy as np
import pytest

from paper_1105_3468_gb300 import workloads as W


def _random_mmatrix(n, density, seed):
    rng = np.random.default_rng(seed)
    D = -rng.random((n, n)) * (rng.random((n, n)) < density)
    np.fill_diagonal(D, 0.0)
    np.fill_diagonal(D, np.abs(D).sum(axis=1) + 0.5 + rng.random(n))
    return D


def test_tau_zero_is_complete_lu(oracle_lib):
    O = oracle_lib
    for A in (O.as_csr(_random_mmatrix(60, 0.08, 1)), O.fv_assemble(W.c1_block_2d_64(seed=3))[0]):
        I = O.Ilut(A, 0.0)
        assert I.status == 0
        Lf, Uf = I.factors()
        D = A.dense()
        m = A.n
        gam = m * np.finfo(float).eps / (1 - m * np.finfo(float).eps)
        assert np.all(np.abs(D - Lf @ Uf) <= gam * (np.abs(Lf) @ np.abs(Uf)) + 1e-300)
        b = np.random.default_rng(4).standard_normal(A.n)
        x = I.solve(b)
        assert np.linalg.norm(D @ x - b) <= 1e-10 * np.linalg.norm(b) * np.linalg.cond(D)


def test_tridiagonal_equals_ilu0(oracle_lib):
    O = oracle_lib
    n = 50
    rng = np.random.default_rng(7)
    D = np.diag(3 + rng.random(n)) + np.diag(-rng.random(n - 1), 1) + np.diag(-rng.random(n - 1), -1)
    A = O.as_csr(D)
    lu, st = O.ilu0(A, np.zeros(n, np.int32))
    assert st == 0
    I = O.Ilut(A, 0.0)
    assert np.array_equal(I.F.row_ptr, A.row_ptr) and np.array_equal(I.F.col, A.col)
    assert np.array_equal(I.F.val, lu)


def test_tau_infinite_keeps_the_diagonal(oracle_lib):
    O = oracle_lib
    A = O.as_csr(_random_mmatrix(40, 0.2, 2))
    I = O.Ilut(A, 1e300)
    Lf, Uf = I.factors()
    assert np.array_equal(Lf, np.eye(A.n))
    assert np.array_equal(Uf, np.diag(np.diag(A.dense())))


@pytest.mark.parametrize("tau", [1e-6, 1e-4, 1e-2])
def test_structure_and_dropping_rule(oracle_lib, tau):
    O = oracle_lib
    A, _ = O.fv_assemble(W.c1_block_2d_64(seed=5))
    I = O.Ilut(A, tau)
    F = I.F
    for i in range(A.n):
        row = A.val[A.row_ptr[i]:A.row_ptr[i + 1]]
        ti = tau * np.sqrt(np.sum(row * row))
        cols = F.col[F.row_ptr[i]:F.row_ptr[i + 1]]
        vals = F.val[F.row_ptr[i]:F.row_ptr[i + 1]]
        assert np.all(np.diff(cols) > 0)
        assert i in cols
        off = cols != i
        assert np.all(np.abs(vals[off]) >= ti) and np.all(vals[off] != 0.0)
    z = np.random.default_rng(6).standard_normal(A.n)
    Lf, Uf = I.factors()
    ref = np.linalg.solve(Lf @ Uf, z)
    assert np.allclose(I.solve(z), ref, rtol=1e-9, atol=1e-9 * np.abs(ref).max())


def test_error_and_fill_trend(oracle_lib):
    O = oracle_lib
    A, _ = O.fv_assemble(W.c1_block_2d_64())
    D = A.dense()
    nnz, err = [], []
    for tau in (0.0, 1e-8, 1e-6, 1e-4, 1e-2):
        I = O.Ilut(A, tau)
        Lf, Uf = I.factors()
        nnz.append(I.F.nnz)
        err.append(np.linalg.norm(D - Lf @ Uf) / np.linalg.norm(D))
    assert all(a >= b for a, b in zip(nnz, nnz[1:]))
    assert err[0] < 1e-14 and all(a <= b * (1 + 1e-12) for a, b in zip(err, err[1:]))


@pytest.mark.parametrize("tau, kept", [(0.01, True), (0.02, False)])
def test_hand_computed_3x3(oracle_lib, tau, kept):
    """A = [[4,-1,-1],[-1,4,0],[-1,0,4]], by hand: row 2 gives l_10 = -1/4,
    u_11 = 4 - 1/4 = 15/4 and the fill u_12 = -1/4 (kept: tau_1 = tau sqrt 17
    < 1/4).  Row 3: l_20 = -1/4, fill w_1 = -1/4, w_2 = 4 - 1/4 = 15/4; then
    w_1 / u_11 = -1/15 against tau_2 = tau sqrt 17 (0.0412 at tau = 0.01:
    kept, u_22 = 15/4 - (1/15)(1/4); 0.0825 at tau = 0.02: dropped,
    u_22 = 15/4)."""
    O = oracle_lib
    A = O.as_csr(np.array([[4.0, -1, -1], [-1, 4, 0], [-1, 0, 4]]))
    Lf, Uf = O.Ilut(A, tau).factors()
    assert Lf[1, 0] == -0.25 and Lf[2, 0] == -0.25
    assert Uf[1, 1] == 3.75 and Uf[1, 2] == -0.25
    if kept:
        assert Lf[2, 1] == pytest.approx(-1 / 15, rel=1e-15)
        assert Uf[2, 2] == pytest.approx(3.75 - 1 / 60, rel=1e-15)
    else:
        assert Lf[2, 1] == 0.0 and Uf[2, 2] == 3.75


def _small(O):
    p = W.block_kappa_grid(16, 2, 4, -2, 2, 31, velocity=("const", (1.0, 0.5)))
    return O.fv_assemble(p)


def test_two_grid_with_ilut_tau0_is_the_exact_two_grid(oracle_lib):
    """The paper's two-grid form (Algorithm 1: A~_c = ILUT(A_c), one coarse
    solve): with tau = 0 the coarse factors are exact, so the preconditioner
    equals the two-grid one whose coarse level is solved by its inverse."""
    O = oracle_lib
    A, _ = _small(O)
    Hi = O.Hierarchy(A, coarse_solver=O.COARSE_ILUT, ilut_tau=0.0)
    He = O.Hierarchy(A, dense_max=10 ** 6, max_levels=2)
    assert Hi.nlev == He.nlev == 2 and He.levels[1]["dense"] and not Hi.levels[1]["dense"]
    z = np.random.default_rng(8).standard_normal(A.n)
    for tr in (False, True):
        qi, qe = Hi.precond(z, transpose=tr), He.precond(z, transpose=tr)
        assert np.allclose(qi, qe, rtol=1e-10, atol=1e-12 * np.abs(qe).max())


def test_two_grid_with_ilut_transpose_and_coarse_solve(oracle_lib):
    O = oracle_lib
    A, _ = _small(O)
    H = O.Hierarchy(A, coarse_solver=O.COARSE_ILUT, ilut_tau=1e-3)
    n = A.n
    Bi = np.column_stack([H.precond(e) for e in np.eye(n)])
    BiT = np.column_stack([H.precond(e, transpose=True) for e in np.eye(n)])
    assert np.allclose(BiT, Bi.T, rtol=1e-10, atol=1e-12 * np.abs(Bi).max())
    A1 = H.matrix(1)
    I = O.Ilut(A1, 1e-3)
    h = np.random.default_rng(9).standard_normal(A1.n)
    assert np.array_equal(H.level_solve(1, h), I.solve(h))
    assert np.array_equal(H.level_solve(1, h, transpose=True), I.solve(h, transpose=True))
    Lf, Uf = I.factors()
    assert np.allclose(I.solve(h, transpose=True), np.linalg.solve((Lf @ Uf).T, h), rtol=1e-9)
