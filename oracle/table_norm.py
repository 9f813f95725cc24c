"""Writes oracle/table_norm.json: the relative error ||LU - L~U~|| / ||LU|| of
the inexact coarse factorisation, the quantity of the paper's table comparing
exact and inexact coarse operators (Section 3), computed with the oracle only.

Readings (the paper leaves them open):
* the problem "JUMP3D" is the DC1 3D case (its convergence figure for the
  same comparison is titled DC3D 50^3);
* LU is the exact factorisation of the coarse operator, so LU = A_c, with
  A_c the Galerkin product of the default aggregation (two matching passes);
* L~U~ = ILUT(A_c) in natural order with the oracle's dropping rule (Saad's:
  a multiplier or entry of row i is dropped below tau * ||a_i||_2), at the
  drop tolerance 1e-4 of the paper's neighbouring table on the same problems
  and at 1e-6, the library's default;
* the norm is the Frobenius norm (the paper does not name it).
The sparse product L~U~ uses scipy.sparse (a library primitive).

    python oracle/table_norm.py [n ...]      (default: 30 40 50)
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import oracle as O  # noqa: E402
from paper_1105_3468_gb300 import workloads as W  # noqa: E402

TAUS = (1e-4, 1e-6)
PAPER_NO = {30: 7.5e-5, 40: 8.3e-5, 50: 7.0e-5}     # the paper's natural-ordering column


def factor_error(Ac, F):
    """||A_c - L~U~||_F / ||A_c||_F for ILUT factors F (rows: L~ part, then U~)."""
    import scipy.sparse as sp
    n = Ac.n
    rows = np.repeat(np.arange(n), np.diff(F.row_ptr))
    low = F.col < rows
    Lf = sp.csr_matrix((F.val[low], (rows[low], F.col[low])), shape=(n, n)) + sp.identity(n, format="csr")
    Uf = sp.csr_matrix((F.val[~low], (rows[~low], F.col[~low])), shape=(n, n))
    A = sp.csr_matrix((Ac.val, Ac.col, Ac.row_ptr), shape=(n, n))
    D = A - Lf @ Uf
    return float(sp.linalg.norm(D, "fro") / sp.linalg.norm(A, "fro"))


def coarse_operator(n):
    A, _ = O.fv_assemble(W.dc_problem(n, 3))
    H = O.Hierarchy(A, coarse_solver=O.COARSE_ILUT, ilut_tau=TAUS[0])
    return H.matrix(1)


def main(sizes):
    path = os.path.join(HERE, "table_norm.json")
    out = {"taus": list(TAUS), "norm": "frobenius", "problem": "DC1 3D (JUMP3D)", "rows": {}}
    for n in sizes:
        Ac = coarse_operator(n)
        row = {"n_c": Ac.n, "nnz_c": Ac.nnz, "paper_natural_order_tau_1e-4": PAPER_NO.get(n)}
        for tau in TAUS:
            F = O.Ilut(Ac, tau)
            assert F.status == O.OK
            row[f"tau_{tau:g}"] = {"nnz_factors": F.F.nnz, "rel_error": factor_error(Ac, F.F)}
        out["rows"][str(n)] = row
        print(n, row, flush=True)
    json.dump(out, open(path, "w"), indent=1)


if __name__ == "__main__":
    main([int(a) for a in sys.argv[1:]] or [30, 40, 50])
