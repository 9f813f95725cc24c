"""Writes oracle/ordering_iters.json: FGMRES(30) iterations of the oracle to
relative residual 1e-8 with the finest level's ILU(0) in natural order (the
paper's GMG-NO, Section 3) against colour-major order, on the 3D anisotropic
block-kappa recipe, with the exact two-grid form (level 1 solved by its
dense inverse) and with the default recursive hierarchy.  This is the
measurement behind keeping natural order on the finest level.

Runs only the oracle:  python oracle/ordering_iters.py [n ...]  (default 16 24)
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import oracle as O  # noqa: E402
from paper_1105_3468_gb300 import workloads as W  # noqa: E402


def main(sizes):
    out = {"tol": 1e-8, "restart": 30, "maxit": 600, "rows": {}}
    for n in sizes:
        A, b = O.fv_assemble(W.c3_aniso_3d_128(n=n))
        row = {}
        for form, kw in (("exact_two_grid", {"max_levels": 2}), ("default_hierarchy", {})):
            for order, name in ((O.ORDER_NATURAL, "natural"), (O.ORDER_COLOR, "colour_major")):
                H = O.Hierarchy(A, order_fine=order, **kw)
                _, info = H.fgmres(b, tol=1e-8, maxit=600)
                row[f"{form}/{name}"] = {"iters": info.iters, "status": info.status,
                                         "levels": [L["n"] for L in H.levels]}
        out["rows"][str(n)] = row
        print(n, row, flush=True)
    json.dump(out, open(os.path.join(HERE, "ordering_iters.json"), "w"), indent=1)


if __name__ == "__main__":
    main([int(a) for a in sys.argv[1:]] or [16, 24])
