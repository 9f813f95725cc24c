"""Input generators: the paper's DC1 / DCC conductivity (Section 4, test
cases) evaluated point by point from its definition, and the shapes and
flux conventions of the generated problems."""
import math

import numpy as np

from paper_1105_3468_gb300 import workloads as W


def _kappa_point(x):
    """kappa(x) = 1000 ([10 x_2] + 1) if [10 x_i] is even for all i, else 1."""
    if all(math.floor(10.0 * xi) % 2 == 0 for xi in x):
        return 1000.0 * (math.floor(10.0 * x[1]) + 1)
    return 1.0


def test_dc_kappa_2d_matches_definition():
    n = 37
    k = W.dc_kappa(n, 2)
    for idx in range(0, n * n, 7):
        i, j = idx % n, idx // n
        x = ((i + 0.5) / n, (j + 0.5) / n)
        assert k[idx] == _kappa_point(x)


def test_dc_kappa_3d_matches_definition():
    n = 23
    k = W.dc_kappa(n, 3)
    for idx in range(0, n ** 3, 11):
        i, j, l = idx % n, (idx // n) % n, idx // (n * n)
        x = ((i + 0.5) / n, (j + 0.5) / n, (l + 0.5) / n)
        assert k[idx] == _kappa_point(x)


def test_dc_problems_shapes_and_velocity():
    p = W.dc_problem(40, 2)
    assert p.n == 1600 and not p.fx.any() and not p.fy.any()
    q = W.dc_problem(12, 3, velocity=1000.0)
    h = 1.0 / 12
    # constant velocity: every interior x-face carries a_x times the face area h^2
    assert np.allclose(q.fx, 1000.0 * h * h)
    assert np.unique(q.kx).tolist() == sorted(set(W.dc_kappa(12, 3).tolist()))
