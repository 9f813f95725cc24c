"""Pins of the oracle's coarsening: matching, aggregates, Galerkin product.

Matching (aggregation by graph matching, Section 2):
* the tie-break hash is SplitMix64's finaliser: the first three outputs of
  the SplitMix64 generator from state 0 are its published test vectors;
* validity (each vertex in at most one pair; every pair an edge, w > 0) and
  maximality (no edge joins two unmatched vertices);
* brute force on small graphs, for the plain and the scaled edge weight: the
  greedy matching equals the matching whose key multiset, sorted in
  decreasing order, is lexicographically largest (keys recomputed here from
  the dense matrix);
* the weight of a structurally one-sided entry is |a_uv|/2; A and A^T give
  the same matching;
* scaled weight, hand-computed: a vertex whose coupling is all of its
  diagonal pairs with its neighbour even against a heavier plain weight;
* scaled weight on the paper's DC1 2D case at 640^2: every level shrinks by
  at least 2x down to fewer than 200 rows, where the plain weight stalls
  (a level shrinking by less than 10%).
Aggregates (eq. (4) and the part map of Section 2): a partition; P*1 = 1;
rank P = N_c (Theorem 1); size <= 2^passes; ids ordered by smallest member.
Galerkin (eq. (3) and its entrywise form, Section 2): brute-force dense
P^T A P on dyadic values (exact); row sums A_c 1 = P^T A 1; symmetric ->
symmetric; SPD -> SPD (Theorem 2); diagonally dominant M-matrix -> the same
(Theorem of Kim et al. quoted in Section 2.1); the 4x4 counterexample of
Section 2.1 (tests/golden/counterexample_4x4.txt).
"""
import itertools
import os

import numpy as np
import pytest

from conftest import GOLDEN
from paper_1105_3468_gb300 import workloads as W


def test_splitmix64_published_vectors(oracle_lib):
    O = oracle_lib
    gamma = 0x9E3779B97F4A7C15
    expect = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    s = 0
    for e in expect:
        s = (s + gamma) & 0xFFFFFFFFFFFFFFFF
        assert O.mix64(s) == e


def _random_sparse(rng, n, density, sym_pattern=True, dyadic=False):
    D = np.zeros((n, n))
    mask = rng.random((n, n)) < density
    if sym_pattern:
        mask = mask | mask.T
    np.fill_diagonal(mask, True)
    if dyadic:
        vals = rng.integers(-8, 9, size=(n, n)) / 4.0
        vals[vals == 0] = 0.25
    else:
        vals = rng.standard_normal((n, n))
    D[mask] = vals[mask]
    np.fill_diagonal(D, np.abs(D).sum(axis=1) + 1.0)
    return D


def _edges(O, A, scaled=1):
    """Unordered structural edges with their keys (weight, hash, u, v); the
    weights are computed here from the dense matrix."""
    D = A.dense()
    n = A.n
    pat = (np.abs(D) > 0) | (np.abs(D.T) > 0)
    out = []
    for u in range(n):
        for v in range(u + 1, n):
            if pat[u, v]:
                w = (abs(D[u, v]) + abs(D[v, u])) * 0.5
                if scaled and w > 0:
                    w = w / np.sqrt(abs(D[u, u]) * abs(D[v, v]))
                if w > 0:
                    out.append(((w, O.edge_hash(u, v, 0), u, v), u, v))
    return out


def _check_matching(O, A, mate, scaled=1):
    n = A.n
    for u in range(n):
        if mate[u] >= 0:
            assert mate[mate[u]] == u and mate[u] != u
    for key, u, v in _edges(O, A, scaled):
        assert not (mate[u] < 0 and mate[v] < 0), "not maximal"
    pairs = {(min(u, int(mate[u])), max(u, int(mate[u]))) for u in range(n) if mate[u] >= 0}
    edge_set = {(u, v) for _, u, v in _edges(O, A, scaled)}
    assert pairs <= edge_set


@pytest.mark.parametrize("scaled", [0, 1])
@pytest.mark.parametrize("seed", range(12))
def test_matching_brute_force(oracle_lib, seed, scaled):
    O = oracle_lib
    rng = np.random.default_rng(seed)
    n = int(rng.integers(3, 9))
    D = _random_sparse(rng, n, 0.35, sym_pattern=bool(seed % 2))
    if seed % 3 == 0:   # ties in weight: the hash decides
        D[np.abs(D) > 0] = np.sign(D[np.abs(D) > 0])
        np.fill_diagonal(D, 10.0)
    elif scaled:        # unequal diagonals, so scaling reorders the keys
        np.fill_diagonal(D, np.diag(D) * rng.uniform(0.5, 4.0, n))
    A = O.as_csr(D)
    mate = O.match(A, weight=scaled)
    _check_matching(O, A, mate, scaled)
    E = _edges(O, A, scaled)
    best = None
    for r in range(0, n // 2 + 1):
        for combo in itertools.combinations(range(len(E)), r):
            used = set()
            ok = True
            for c in combo:
                _, u, v = E[c]
                if u in used or v in used:
                    ok = False
                    break
                used |= {u, v}
            if not ok:
                continue
            keyseq = sorted((E[c][0] for c in combo), reverse=True)
            if best is None or keyseq > best[0]:
                best = (keyseq, combo)
    greedy_pairs = {(min(u, int(mate[u])), max(u, int(mate[u]))) for u in range(n) if mate[u] >= 0}
    best_pairs = {(E[c][1], E[c][2]) for c in best[1]}
    assert greedy_pairs == best_pairs


def test_matching_one_sided_weight_and_transpose(oracle_lib):
    O = oracle_lib
    D = np.diag([4.0, 4.0, 4.0, 4.0])
    D[0, 1] = -3.0          # only a_01 stored: w(0,1) = 1.5
    D[2, 1] = -1.0
    D[1, 2] = -1.0          # w(1,2) = 1.0
    D[3, 2] = -2.5          # w(2,3) = 1.25
    A = O.as_csr(D)
    assert O.edge_weight(A, 0, 1) == 1.5
    assert O.edge_weight(A, 1, 0) == 1.5
    assert O.edge_key_weight(A, 0, 1, 0) == 1.5 and O.edge_key_weight(A, 0, 1, 1) == 1.5 / 4.0   # sqrt(4*4)
    for scaled in (0, 1):
        mate = O.match(A, weight=scaled)
        assert mate.tolist() == [1, 0, 3, 2]
        assert np.array_equal(O.match(O.as_csr(D.T.copy()), weight=scaled), mate)


def test_scaled_weight_pairs_a_dominated_vertex(oracle_lib):
    """Path 0 - 1 - 2: vertex 0's only coupling (1) is its whole diagonal,
    while 1 - 2 carries the heavier coupling 3 to a vertex with a large
    diagonal (100).  Plain weights (1 vs 3) pair {1, 2} and leave 0 single;
    scaled weights (1/sqrt(1*4) = 0.5 vs 3/sqrt(4*100) = 0.15) pair {0, 1}."""
    O = oracle_lib
    D = np.array([[1.0, -1.0, 0.0], [-1.0, 4.0, -3.0], [0.0, -3.0, 100.0]])
    A = O.as_csr(D)
    assert O.edge_key_weight(A, 0, 1, 1) == 0.5
    assert O.edge_key_weight(A, 1, 2, 1) == 3.0 / 20.0
    assert O.match(A, weight=0).tolist() == [-1, 2, 1]
    assert O.match(A, weight=1).tolist() == [1, 0, -1]


def test_scaled_weight_does_not_stall_on_dc1():
    """The paper's DC1 2D case (Section 4) at 640^2, coarsened without a
    dense level: with scaled weights each level of at least 200 rows is
    followed by one of at most half its size, down to fewer than 200 rows;
    with plain weights some level keeps more than 90% (the stall that ends
    the hierarchy)."""
    import oracle as O
    A, _ = O.fv_assemble(W.dc_problem(640, 2))
    for scaled in (1, 0):
        H = O.Hierarchy(A, dense_max=0, max_levels=24, match_weight=scaled)
        sizes = [L["n"] for L in H.levels]
        ratios = [b / a for a, b in zip(sizes, sizes[1:])]
        if scaled:
            big = [r for a, r in zip(sizes, ratios) if a >= 200]
            assert sizes[-1] < 200 and max(big) <= 0.5, sizes
        else:
            assert sizes[-1] > 1000, sizes          # the last level is the stalled one


def test_matching_on_grid_is_valid_and_maximal(oracle_lib):
    O = oracle_lib
    A, _ = O.fv_assemble(W.c1_block_2d_64())
    mate = O.match(A)
    _check_matching(O, A, mate)


def _P(agg, nc):
    P = np.zeros((agg.size, nc))
    P[np.arange(agg.size), agg] = 1.0
    return P


def test_aggregates_partition_and_numbering(oracle_lib):
    O = oracle_lib
    A, _ = O.fv_assemble(W.c3_aniso_3d_128(n=10))
    H = O.Hierarchy(A, dense_max=0, max_levels=3)
    for l in range(H.nlev - 1):
        agg = H.agg(l)
        nc = H.levels[l + 1]["n"]
        assert agg.min() == 0 and agg.max() == nc - 1
        sizes = np.bincount(agg, minlength=nc)
        assert sizes.min() >= 1 and sizes.max() <= 4          # 2 passes of pairs
        P = _P(agg, nc)
        assert np.array_equal(P @ np.ones(nc), np.ones(agg.size))     # P 1 = 1
        assert np.linalg.matrix_rank(P) == nc
        first = np.full(nc, agg.size)
        np.minimum.at(first, agg, np.arange(agg.size))
        assert np.all(np.diff(first) > 0)          # ordered by smallest member
        # composite map = pass-2 map after pass-1 map
        a1, a2 = H.agg(l, 1), H.agg(l, 2)
        assert np.array_equal(a2[a1], agg)


def test_galerkin_brute_force_dyadic(oracle_lib):
    O = oracle_lib
    rng = np.random.default_rng(7)
    for trial in range(6):
        n = int(rng.integers(5, 40))
        D = _random_sparse(rng, n, 0.2, sym_pattern=bool(trial % 2), dyadic=True)
        nc = int(rng.integers(1, n + 1))
        agg = np.sort(rng.integers(0, nc, size=n)).astype(np.int32)
        agg = np.unique(agg, return_inverse=True)[1].astype(np.int32)
        nc = int(agg.max()) + 1
        A = O.as_csr(D)
        Ac = O.galerkin(A, agg, nc)
        P = _P(agg, nc)
        assert np.array_equal(Ac.dense(), P.T @ D @ P)
        # structural pattern: every (I, J) reached by some a_kl is stored
        pat = (np.abs(P.T @ (np.abs(D) > 0) @ P) > 0)
        Dc = np.zeros((nc, nc), bool)
        for I in range(nc):
            Dc[I, Ac.col[Ac.row_ptr[I]:Ac.row_ptr[I + 1]]] = True
        assert np.array_equal(Dc, pat)


def test_galerkin_keeps_structural_zero(oracle_lib):
    O = oracle_lib
    D = np.array([[2.0, 1.0, 0.0], [1.0, 2.0, -1.0], [0.0, -1.0, 2.0]])
    Ac = O.galerkin(O.as_csr(D), np.array([0, 1, 1], np.int32), 2)
    assert Ac.nnz == 4
    assert Ac.dense()[0, 1] == 1.0 and Ac.dense()[1, 1] == 2.0


def test_galerkin_invariants_on_grid(oracle_lib):
    O = oracle_lib
    p = W.block_kappa_grid(16, 2, 4, -4, 4, 3, velocity=("const", (0.0, 0.0)))
    A, _ = O.fv_assemble(p)
    D = A.dense()
    H = O.Hierarchy(A, dense_max=0, max_levels=3)
    agg = H.agg(0)
    Ac = H.coarse().dense()
    P = _P(agg, H.nc)
    assert np.allclose(Ac, P.T @ D @ P, rtol=1e-14, atol=1e-14 * np.abs(D).max())
    assert np.allclose(Ac.sum(axis=1), P.T @ D.sum(axis=1), rtol=1e-13,
                       atol=1e-13 * np.abs(D).max())                   # row sums
    assert np.array_equal(Ac, Ac.T)                                    # symmetric
    assert np.linalg.eigvalsh(Ac).min() > 0                            # SPD (Theorem 2)
    off = Ac - np.diag(np.diag(Ac))
    assert np.all(off <= 0) and np.all(np.diag(Ac) > 0)                # M-matrix signs
    assert np.all(Ac.sum(axis=1) >= -1e-12 * np.abs(Ac).max())         # diagonal dominance


def test_counterexample_4x4(oracle_lib):
    O = oracle_lib
    rows = [l.split() for l in open(os.path.join(GOLDEN, "counterexample_4x4.txt"))
            if l.strip() and not l.startswith("#")]
    PT = np.array(rows[:2], float)
    x = np.array(rows[2], float)
    agg = np.array([0, 1, 0, 1], np.int32)      # G1 = {1,3}, G2 = {2,4} (1-based)
    assert np.array_equal(_P(agg, 2).T, PT)
    assert np.array_equal(PT @ x, np.zeros(2))
    # any SPD A: A_c = P^T A P is SPD, yet M = P A_c P^T annihilates x
    rng = np.random.default_rng(1)
    B = rng.standard_normal((4, 4))
    Aspd = B @ B.T + 4 * np.eye(4)
    Ac = O.galerkin(O.as_csr(Aspd), agg, 2).dense()
    assert np.allclose(Ac, PT @ Aspd @ PT.T)
    assert np.linalg.eigvalsh(Ac).min() > 0
    M = PT.T @ Ac @ PT
    assert abs(x @ M @ x) < 1e-12
