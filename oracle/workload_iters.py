"""Writes oracle/workload_iters.json: FGMRES(30) iteration counts of the CPU
oracle (FP64, default options) to the stated tolerance on the full-size
benchmark workloads.  The benchmark's CPU-baseline legs scale a bounded
sample of oracle work (full setup + a few iterations) by these counts.

Runs only the oracle (tens of minutes for the 128^3 problem):
    python oracle/workload_iters.py [name ...]   (names: the keys of CASES)
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import oracle as O  # noqa: E402
from paper_1105_3468_gb300 import workloads as W  # noqa: E402

# (problem, tol, maxit, hierarchy options): the benchmark's settings per
# workload; the paper's own cases stop at its tolerance 1e-7 (Section 3)
CASES = {
    "c3": (lambda: W.c3_aniso_3d_128(), 1e-8, 3000, {}),
    "c2": (lambda: W.c2_rotating_2d_1024(), 1e-7, 600, {"order_fine": O.ORDER_COLOR,
                                                        "match_weight": O.MATCH_PLAIN}),
    "c1": (lambda: W.c1_block_2d_64(), 1e-8, 600, {}),
    "c4": (lambda: W.c4_adjoint_2d()[0], 1e-8, 600, {}),
    "dc1-2d": (lambda: W.dc_problem(1200, 2), 1e-7, 600, {}),
    "dcc1-2d": (lambda: W.dc_problem(1200, 2, velocity=1000.0), 1e-7, 600, {}),
    "dc1-3d": (lambda: W.dc_problem(120, 3), 1e-7, 600, {}),
    "dcc2-3d": (lambda: W.dc_problem(120, 3, velocity=1000.0), 1e-7, 600, {}),
}


def main(names):
    path = os.path.join(HERE, "workload_iters.json")
    for name in names:
        make, tol, maxit, opts = CASES[name]
        A, b = O.fv_assemble(make())
        t0 = time.perf_counter()
        H = O.Hierarchy(A, **opts)
        t1 = time.perf_counter()
        _, info = H.fgmres(b, tol=tol, maxit=maxit)
        t2 = time.perf_counter()
        out = json.load(open(path)) if os.path.exists(path) else {}     # other runs may have written
        out[name] = info.iters
        out[name + "_detail"] = {"status": info.status, "tol": tol, "maxit": maxit, "relres": info.relres,
                                 "setup_s": round(t1 - t0, 2), "solve_s": round(t2 - t1, 2)}
        json.dump(out, open(path, "w"), indent=1)
        print(name, out[name + "_detail"], flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or list(CASES))
