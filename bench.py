#!/usr/bin/env python
"""Benchmark: time to relative residual 1e-8 with the matching-aggregation
AMG preconditioner in FGMRES(30), mixed-precision V-cycle vs all-FP64, on one
GB300.

One step = one pass of the whole path over one system: amg_setup (matching
passes, aggregates, Galerkin products, colourings, ILU(0) factors, dense
last level, precision copies) + amg_solve to ||b - A x|| / ||b|| <= tol
(FGMRES(30) with the V-cycle preconditioner, true FP64 residual).  Inputs
(the assembled CSR matrix and right-hand side) are resident in HBM before the
timed region.  The default workload is the 128^3 anisotropic 3D
finite-volume problem (2,097,152 unknowns, 14.6 M nonzeros), whose matrix
alone (175 MB) exceeds L2, so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Under torchrun each rank solves its own copy (replicas: the single-system
path has no exchange step); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "time-to-rel-residual 1e-8 (mixed vs FP64, same GPU); SpMV/cycle HBM GB/s"


def workload(name, size=None):
    """(problem, tol, maxit, setup options, description).  size: a smaller
    instance of the 3D recipe (profiling captures only)."""
    from paper_1105_3468_gb300 import workloads as W
    if name == "c3" and size:
        return (W.c3_aniso_3d_128(n=size), 1e-8, 3000, {},
                f"fv3d-{size}^3-aniso-blockkappa (same recipe as the 128^3 workload, for profiling)")
    if name == "c3":
        return (W.c3_aniso_3d_128(), 1e-8, 3000, {},
                "fv3d-128^3-aniso-blockkappa (2,097,152 unknowns, 14,581,760 nnz, 7-point upwind, 16^3 blocks "
                "kappa_axis=10^U(-3,3), a=(1,1,1)); FGMRES(30) to true rel. residual 1e-8, maxit 3000; "
                "natural-order ILU(0) on level 0, colour-major below")
    if name == "c2":
        return (W.c2_rotating_2d_1024(), 1e-7, 600, {"order_fine": 0, "match_weight": 0},
                "fv2d-1024^2-rotating (1,048,576 unknowns), FGMRES(30), tol 1e-7 "
                "(1e-8 is below this matrix's FP64 attainable residual), colour-major ILU(0), "
                "unscaled matching weights")
    if name == "c1":
        return (W.c1_block_2d_64(), 1e-8, 600, {},
                "fv2d-64^2-blockkappa (4096 unknowns), FGMRES(30), tol 1e-8")
    if name in ("dc1-2d", "dcc1-2d", "dc1-3d", "dcc2-3d"):
        dim = 3 if name.endswith("3d") else 2
        n = 120 if dim == 3 else 1200
        a = 1000.0 if name.startswith("dcc") else 0.0
        return (W.dc_problem(n, dim, velocity=a), 1e-7, 600, {},
                f"paper test case {name.upper()} (Section 4): {n}^{dim} cells, kappa = 1000([10 x_2]+1) on "
                f"isolated zones else 1, a = {a:g} per axis; FGMRES(30) to true rel. residual 1e-7 (the "
                f"paper's stopping tolerance), maxit 600")
    if name == "c5":
        # dense_max 1024: the members' dense inverses dominate the batch's setup
        # (8.30 s per batch with 4096, 3.96 s with 1024, every member converging)
        return (W.c5_batch_specs(), 1e-8, 600, {"dense_max": 1024},
                "batch of 64 uneven systems: 48 block-kappa grids side U{64..512} + 16 random-geometric-graph "
                "matrices 10k..500k rows, 7..30 nnz/row (8.8 M rows); every member's loop in one graph, FP64 "
                "FGMRES(30), tol 1e-8, last levels of up to 1024 rows solved by their inverse")
    raise ValueError(name)


def batch_members(specs, amg, on_device=True):
    """Matrices (device CSR) and right-hand sides of the batch recipe."""
    import numpy as np
    from paper_1105_3468_gb300 import workloads as W
    mats, rhs = [], []
    for sp in specs:
        if sp.kind == "grid":
            A, _ = amg.assemble_fv(W.batch_grid_problem(sp))
        else:
            A = amg.CsrDevice.from_host(W.rgg_matrix(sp.size, sp.nnz_per_row, sp.seed))
        mats.append(A)
        rhs.append(W.batch_rhs(sp, A.n))
    return mats, np.concatenate(rhs)


def run_batch(args, amg, torch):
    """Batched path: setup + solve of the 64-system batch per step.  Under
    torchrun the members are split across ranks (longest-processing-time
    first by nonzeros, no data-path collective); the step time is the
    slowest rank's, so `value` is the time for the whole batch."""
    import torch.distributed as dist
    from paper_1105_3468_gb300 import shard
    rank, world, local = dist_env()
    specs, tol, maxit, sopts, desc = workload("c5")
    parts = shard.lpt_partition([shard.member_weight(s) for s in specs], world)
    mine = [specs[k] for k in parts[rank]]
    mats, rhs = batch_members(mine, amg)
    b = torch.tensor(rhs, device="cuda")
    vp = {"fp32": amg.AMG_FP32, "bf16": amg.AMG_BF16, "bf16all": amg.AMG_BF16_ALL, "fp64": amg.AMG_FP64}[args.prec]
    rows = sum(A.n for A in mats)
    nnz = sum(A.nnz for A in mats)

    def barrier():
        if world > 1:
            dist.barrier()

    extra_opts = dict(sopts)
    for kv in args.opt:
        k, v = kv.split("=", 1)
        extra_opts[k] = float(v) if k == "ilut_tau" else int(v)
    split = []

    def step(prec):
        extra = {"dot2": args.fp64_dot2} if prec == amg.AMG_FP64 and vp != amg.AMG_FP64 else {}
        t0 = time.perf_counter()
        h = amg.amg_setup_batched(mats, vcycle_prec=prec, maxit=maxit, **extra, **extra_opts)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        x = torch.zeros_like(b)
        st = amg.amg_solve_batched(h, b, x, tol)
        torch.cuda.synchronize()
        split.append((prec, 1e3 * (t1 - t0), 1e3 * (time.perf_counter() - t1)))
        h.close()
        return st

    for _ in range(args.warmup):
        step(vp)
    res = {}
    for prec in (vp, amg.AMG_FP64) if vp != amg.AMG_FP64 else (vp,):
        barrier()
        torch.cuda.synchronize()
        l0 = amg.amg_launch_counter()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            st = step(prec)
        e1.record()
        torch.cuda.synchronize()
        barrier()
        ms = e0.elapsed_time(e1) / args.steps
        if world > 1:
            t = torch.tensor([ms], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        res[prec] = (ms, st, amg.amg_launch_counter() - l0)
    ms, st, launches = res[vp]
    setup_each = sorted(((round(s.setup_ms, 1), A.n) for s, A in zip(st, mats)), reverse=True)
    summary = ([(s.iters, s.status) for s in st], rows, nnz, launches, setup_each)
    if world > 1:
        got = [None] * world
        dist.all_gather_object(got, summary)
    else:
        got = [summary]
    if rank != 0:
        return
    per_member = shard.merge(parts, [g[0] for g in got])
    rows = sum(g[1] for g in got)
    nnz = sum(g[2] for g in got)
    launches = sum(g[3] for g in got)
    out = {"metric": "batch time-to-rel-residual 1e-8 (64 uneven systems)", "value": round(ms, 2), "unit": "ms",
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 2),
           "higher_is_better": False, "scaling": "strong" if world > 1 else "weak", "vs_baseline": None,
           "dtype": {"fp32": "f32 V-cycle / f64 FGMRES", "bf16": "bf16 values, f32 V-cycle / f64 FGMRES",
                     "bf16all": "bf16 factors on every level, f32 V-cycle / f64 FGMRES", "fp64": "f64"}[args.prec], "data": "synthetic",
           "config": {"workload": desc, "rows": rows, "nnz": nnz,
                      "parallelism": f"members split over {world} ranks (LPT by nnz)" if world > 1 else "single GPU"},
           "rows_per_s": round(rows / (ms * 1e-3)),
           "iters_min_max": [min(i for i, _ in per_member), max(i for i, _ in per_member)],
           "all_converged": all(s == 0 for _, s in per_member), "gpu_launches": int(launches),
           "setup_solve_ms_last_step": [[round(a, 1), round(c, 1)] for p, a, c in split if p == vp][-1],
           "member_setup_ms": {"sum": round(sum(t for g in got for t, _ in g[4]), 1),
                               "largest_5_ms_rows": sorted((x for g in got for x in g[4]), reverse=True)[:5]},
           "options": extra_opts}
    if amg.AMG_FP64 in res and vp != amg.AMG_FP64:
        out["fp64_ms_per_step"] = round(res[amg.AMG_FP64][0], 2)
    print(json.dumps(out), flush=True)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


SMOOTHER_PROFILE = os.path.join(ROOT, "profiles", "smoother_dram_fv3d128_one_iteration.md")


def sweep_sources_sha256():
    """SHA-256 of the sweep kernels' sources (solve.cu, tiles.cu, devsync.cuh, in that order)."""
    import hashlib
    h = hashlib.sha256()
    for f in ("solve.cu", "tiles.cu", "devsync.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1105_3468_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def profiled_traffic(workload_name):
    """DRAM bytes per smoother application from the committed ncu summary,
    or None when the summary is for another workload or the sweep kernels'
    source changed since it was captured."""
    if workload_name != "c3":
        return None
    try:
        lines = open(SMOOTHER_PROFILE).read().splitlines()
    except OSError:
        return None
    vals = {}
    for ln in lines:
        if ":" in ln and ln.strip().startswith("- `"):
            k, v = ln.strip()[3:].split("`", 1)
            vals[k] = v.split(":", 1)[1].strip().strip("`")
    if vals.get("sweep_sources_sha256") != sweep_sources_sha256():
        return None
    try:
        return int(vals["dram_bytes_per_application"])
    except (KeyError, ValueError):
        return None


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return None


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def oracle_iterations(name):
    """(iterations, detail) of the oracle's own full FP64 solve of workload
    `name`, from oracle/workload_iters.json (written by
    oracle/workload_iters.py, which runs only the oracle), or (None, None)."""
    path = os.path.join(ROOT, "oracle", "workload_iters.json")
    try:
        d = json.load(open(path))
    except (OSError, ValueError):
        return None, None
    return d.get(name), d.get(name + "_detail")


class OracleSample:
    """The oracle (single-threaded C, as it stands) on a bounded sample of the
    workload: its full-size setup, timed once, and full FGMRES(m) restart
    cycles from x0 = 0, each timed on its own (m iterations, the Arnoldi
    steps j = 1..m and the cycle's update and true residual).  The time of
    the whole solve is projected as setup + iterations x (cycle time / m),
    with the iteration count of the oracle's own full solve."""

    def __init__(self, prob, sopts):
        import oracle as O
        self.O = O
        self.A, self.b = O.fv_assemble(prob)
        t0 = time.perf_counter()
        self.H = O.Hierarchy(self.A, **sopts)
        self.setup_s = time.perf_counter() - t0

    def cycle_s(self, m=30):
        t0 = time.perf_counter()
        self.H.fgmres(self.b, tol=0.0, restart=m, maxit=m)
        return (time.perf_counter() - t0) / m

    def describe(self, per_it, cycles, iters, detail, m=30):
        s = (f"full-size oracle setup ({self.setup_s:.1f} s) + {cycles} full FGMRES({m}) cycle(s) "
             f"({per_it:.2f} s/iteration averaged over the cycle), projected to the {iters} iterations of the "
             f"oracle's own full solve; 1 thread on a host with {os.cpu_count()} cores")
        if detail:
            s += (f"; cross-check: the oracle's full solve measured by oracle/workload_iters.py on its host took "
                  f"{detail.get('setup_s', 0) + detail.get('solve_s', 0):.0f} s (setup {detail.get('setup_s')} s)")
        return s


def cpu_baseline(prob, sopts, name):
    """Oracle timed on a bounded sample (setup + one full restart cycle),
    projected to the oracle's own iteration count for this workload."""
    iters, detail = oracle_iterations(name)
    if iters is None:
        return None
    S = OracleSample(prob, sopts)
    per_it = S.cycle_s()
    value_ms = 1e3 * (S.setup_s + per_it * iters)
    return {"value": round(value_ms, 1), "unit": "ms", "cores": 1, "kind": "oracle",
            "sample": S.describe(per_it, 1, iters, detail), "oracle_iters": iters,
            "setup_s": round(S.setup_s, 2), "s_per_iteration": round(per_it, 4)}


def companion_errors(amg, torch, opts, tol, n=64):
    """The 3D anisotropic recipe at n^3: each V-cycle precision of the GPU
    path against the oracle's FP64 solution, ||x - x_oracle|| / ||x_oracle||,
    all solved to the same true relative residual (run after the timed
    region)."""
    import numpy as np
    import oracle as O
    from paper_1105_3468_gb300 import workloads as W
    p = W.c3_aniso_3d_128(n=n)
    Ao, bo = O.fv_assemble(p)
    xo, info = O.Hierarchy(Ao).fgmres(bo, tol=tol, maxit=opts.get("maxit", 3000))
    A, b = amg.assemble_fv(p)
    out = {"workload": f"fv3d-{n}^3-aniso-blockkappa (same recipe)", "oracle_iters": info.iters}
    for name, prec in (("fp64", amg.AMG_FP64), ("fp32", amg.AMG_FP32), ("bf16", amg.AMG_BF16)):
        h = amg.amg_setup(A, vcycle_prec=prec, **opts)
        x = torch.zeros_like(b)
        st = amg.amg_solve(h, b, x, tol)
        h.close()
        out[name] = {"iters": st.iters, "rel_err": float(np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo))}
    return out


def run_reference(args):
    """Reference arm: the CPU oracle on the host cores.  Its setup is timed
    once; each timed step is one full FGMRES(30) restart cycle, and the step
    value is the projected solve time (setup + iterations x the cycle's
    average iteration time).  The oracle has no state that warms up, so
    warm-up steps are not run; timed steps stop early when the next one
    would take the whole run beyond four minutes (the line reports how many
    ran)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    prob, tol, maxit, sopts, desc = workload(args.workload)
    iters, detail = oracle_iterations(args.workload)
    if iters is None:
        print(json.dumps({"impl": "reference", "unavailable": f"no oracle iteration count for {args.workload}"}))
        return
    t_start = time.perf_counter()
    S = OracleSample(prob, sopts)
    per = []
    for k in range(args.steps):
        t0 = time.perf_counter()
        per.append(S.cycle_s())
        spent, last = time.perf_counter() - t_start, time.perf_counter() - t0
        if spent + last > 240.0:
            break
    vals = [1e3 * (S.setup_s + p * iters) for p in per]
    v = statistics.mean(vals)
    per_it = statistics.mean(per)
    bl = {"value": round(v, 1), "unit": "ms", "cores": 1, "kind": "oracle",
          "sample": S.describe(per_it, len(per), iters, detail), "oracle_iters": iters,
          "setup_s": round(S.setup_s, 2), "s_per_iteration": round(per_it, 4)}
    out = {"impl": "reference", "metric": METRIC, "value": round(v, 1), "unit": "ms", "n_gpus": world,
           "steps": len(per), "steps_requested": args.steps, "warmup": 0, "warmup_requested": args.warmup,
           "ms_per_step": round(v, 1), "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64", "data": "synthetic", "config": {"workload": desc, "tol": tol, "options": sopts},
           "cpu_baseline": bl, "e2e": {"value": round(v, 1), "unit": "ms", "h2d_bytes_per_step": 0,
                                       "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="c3", choices=["c3", "c2", "c1", "c5", "dc1-2d", "dcc1-2d", "dc1-3d",
                                                          "dcc2-3d"])
    ap.add_argument("--prec", default="fp32", choices=["fp32", "bf16", "bf16all", "fp64"])
    ap.add_argument("--roofline-class", type=int, default=2,
                    help="kernel class timed live for the roofline: 1 outer SpMV, 2 ILU(0) smoother, 3 CGS2")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--maxit", type=int, default=None, help="override the workload's iteration cap")
    ap.add_argument("--profile-run", action="store_true",
                    help="one setup + solve of the workload (for ncu captures), no timing output")
    ap.add_argument("--size", type=int, default=None,
                    help="with --profile-run: a smaller n^3 instance of the 3D recipe (small ncu captures)")
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--bf16-steps", type=int, default=1,
                    help="steps of each BF16-factor V-cycle leg (finest level / every level; fp32 runs)")
    ap.add_argument("--fp64-dot2", type=int, default=0, choices=[0, 1],
                    help="accurate (Dot2) inner products in the all-FP64 comparison leg (0: plain, as the mixed leg)")
    ap.add_argument("--persistent", type=int, default=None, choices=[0, 1, 2, 3, 4, 5],
                    help="ILU(0) sweep schedule: 0 per-level launches, 1 level barriers, 2 dataflow, "
                         "3 dataflow on the finest level only, 4 dataflow where the level does not fit "
                         "the shared-memory cluster kernel, 5 as 3 with a grid-stencil finest level in tiles")
    ap.add_argument("--orthog", type=int, default=None, choices=[0, 1], help="0 modified, 1 classical (2-pass) Gram-Schmidt")
    ap.add_argument("--dense-max", type=int, default=None,
                    help="largest level (rows) solved exactly by its dense inverse")
    ap.add_argument("--coarse-solver", type=int, default=None, choices=[0, 1],
                    help="0 recursive coarse solve (default), 1 two-grid with an ILUT-factored coarse level")
    ap.add_argument("--ilut-tau", type=float, default=None, help="drop tolerance of --coarse-solver 1")
    ap.add_argument("--deep-block-max", type=int, default=None,
                    help="levels >= 2 with at most this many rows run their V-cycle in one thread block")
    ap.add_argument("--opt", action="append", default=[], metavar="KEY=VALUE",
                    help="any other amg_options_t field, e.g. --opt coarse_inner=3 --opt coloring=1")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1105_3468_gb300 import build_lib
    build_lib.build()
    import paper_1105_3468_gb300 as amg

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    if args.workload == "c5":
        return run_batch(args, amg, torch)

    def barrier():
        if world > 1:
            dist.barrier()

    if args.size is not None and not args.profile_run:
        raise SystemExit("--size is for --profile-run captures only")
    prob, tol, maxit, sopts, desc = workload(args.workload, args.size)
    if args.maxit is not None:
        maxit = args.maxit
    A, b = amg.assemble_fv(prob)
    torch.cuda.synchronize()
    vp = {"fp32": amg.AMG_FP32, "bf16": amg.AMG_BF16, "bf16all": amg.AMG_BF16_ALL, "fp64": amg.AMG_FP64}[args.prec]
    opts = dict(sopts, maxit=maxit)
    for k in ("persistent", "orthog", "deep_block_max", "dense_max", "coarse_solver", "ilut_tau"):
        if getattr(args, k) is not None:
            opts[k] = getattr(args, k)
    for kv in args.opt:
        k, v = kv.split("=", 1)
        opts[k] = float(v) if k == "ilut_tau" else int(v)

    last_x = {}

    def step(prec, timing_class=0, acc=None):
        o = dict(opts)
        if prec == amg.AMG_FP64 and vp != amg.AMG_FP64:
            o.setdefault("dot2", args.fp64_dot2)      # the all-FP64 comparison leg
        h = amg.amg_setup(A, vcycle_prec=prec, **o)
        if timing_class:
            amg.amg_set_kernel_timing(h, timing_class)
        x = torch.zeros_like(b)
        st = amg.amg_solve(h, b, x, tol)
        if timing_class and acc is not None:
            acc.append(amg.amg_get_kernel_timing(h))
        h.close()
        last_x[prec] = x                              # kept for the accuracy report (outside the timing)
        return st

    if args.profile_run:
        st = step(vp)
        torch.cuda.synchronize()
        print(json.dumps({"profile_run": args.workload, "iters": st.iters, "status": st.status}))
        return

    for _ in range(args.warmup):
        step(vp)

    def timed(prec, timing_class=0, steps=None):
        steps = steps or args.steps
        stats, acc = [], []
        barrier()
        torch.cuda.synchronize()
        l0 = amg.amg_launch_counter()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            stats.append(step(prec, timing_class, acc))
        e1.record()
        torch.cuda.synchronize()
        barrier()
        ms = e0.elapsed_time(e1) / steps
        launches = amg.amg_launch_counter() - l0
        if world > 1:
            t = torch.tensor([ms], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        return ms, stats, acc, launches

    with ClockSampler(local) as clk:
        ms, stats, acc, launches = timed(vp, args.roofline_class)
    clocks = clk.summary()
    ms64, stats64, acc64, _ = (timed(amg.AMG_FP64, timing_class=1, steps=args.fp64_steps) if vp != amg.AMG_FP64
                               else (ms, stats, [], None))
    bf16 = bf16_all = None
    if args.prec == "fp32" and args.bf16_steps > 0:
        ms16, stats16, _, _ = timed(amg.AMG_BF16, steps=args.bf16_steps)
        bf16 = {"ms_per_step": round(ms16, 2), "iters": stats16[-1].iters,
                "rel_res_true": stats16[-1].rel_res_true, "speedup_vs_fp64": round(ms64 / ms16, 3)}
        ms16a, stats16a, _, _ = timed(amg.AMG_BF16_ALL, steps=args.bf16_steps)
        bf16_all = {"ms_per_step": round(ms16a, 2), "iters": stats16a[-1].iters,
                    "rel_res_true": stats16a[-1].rel_res_true, "speedup_vs_fp64": round(ms64 / ms16a, 3)}

    # distance of the mixed-precision solutions to the FP64 GPU solution
    def rel_to_fp64(prec):
        if prec not in last_x or amg.AMG_FP64 not in last_x or prec == amg.AMG_FP64:
            return None
        r = last_x[amg.AMG_FP64]
        return float(torch.linalg.vector_norm(last_x[prec] - r) / torch.linalg.vector_norm(r))
    err_vs_fp64 = {"fp32": rel_to_fp64(amg.AMG_FP32), "bf16": rel_to_fp64(amg.AMG_BF16),
                   "bf16_all_levels": rel_to_fp64(amg.AMG_BF16_ALL)}

    # end to end through the C ABI with host buffers (copies inside the region)
    Ah = amg.CsrDevice(A.n, A.row_ptr.cpu().numpy(), A.col.cpu().numpy(), A.val.cpu().numpy())
    bh = b.cpu().numpy()
    e2e = []
    for _ in range(max(1, args.e2e_steps)):
        xh = np.zeros(A.n)
        t0 = time.perf_counter()
        h = amg.amg_setup(Ah, vcycle_prec=vp, **opts)
        amg.amg_solve(h, bh, xh, tol)
        h.close()
        e2e.append(1e3 * (time.perf_counter() - t0))
    bi = Ah.row_ptr.nbytes + Ah.col.nbytes + Ah.val.nbytes + bh.nbytes + xh.nbytes
    bo = xh.nbytes

    tot_ms = sum(a[0] for a in acc)
    tot_n = sum(a[1] for a in acc)
    tot_b = sum(a[2] for a in acc)
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    roof = None
    if tot_n:
        achieved = tot_b / tot_n / (tot_ms / tot_n * 1e-3) / 1e9
        names = {1: "outer FP64 SpMV w = A z_j",
                 2: "ILU(0) smoother applications, all levels (k_sweep_tiles / k_sweep_pair / k_sweep_pair_dsm)",
                 3: "CGS2 pass"}
        roof = {"bound": "hbm", "kernel": names.get(args.roofline_class), "achieved": round(achieved, 1),
                "peak": peak, "peak_source": "measured" if peaks else "fallback", "unit": "GB/s",
                "frac": round(achieved / peak, 3),
                "traffic": profiled_traffic(args.workload) if args.roofline_class == 2 else None,
                "bytes_per_launch": round(tot_b / tot_n), "avg_launch_us": round(1e3 * tot_ms / tot_n, 2),
                "launches": tot_n}
    spmv_roof = None
    if acc64:
        n1 = sum(a[1] for a in acc64)
        if n1:
            ms1, b1 = sum(a[0] for a in acc64), sum(a[2] for a in acc64)
            ach = b1 / (ms1 * 1e-3) / 1e9
            spmv_roof = {"bound": "hbm", "kernel": "outer FP64 SpMV w = A z_j (FP64 V-cycle run)",
                         "achieved": round(ach, 1), "peak": peak, "unit": "GB/s", "frac": round(ach / peak, 3),
                         "bytes_per_launch": round(b1 / n1), "avg_launch_us": round(1e3 * ms1 / n1, 2),
                         "launches": n1}
    s0 = stats[-1]
    out = {
        "metric": METRIC, "value": round(ms, 2), "unit": "ms", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 2), "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp32": "f32 V-cycle / f64 FGMRES", "bf16": "bf16 values, f32 V-cycle / f64 FGMRES",
                                       "bf16all": "bf16 factors on every level, f32 V-cycle / f64 FGMRES",
                                       "fp64": "f64"}[args.prec],
        "data": "synthetic",
        "config": {"workload": desc,
                   "l2": (f"no flush: matrix {(12 * A.nnz + 8 * (A.n + 1)) / 1e6:.0f} MB and Krylov basis "
                          f"{8 * 31 * A.n / 1e6:.0f} MB per step against a 129 MB L2"),
                   "options": opts,
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "iters": s0.iters, "rel_res_true": s0.rel_res_true, "setup_ms": round(s0.setup_ms, 2),
        "solve_ms": round(s0.solve_ms, 2), "fp64_ms_per_step": round(ms64, 2), "fp64_iters": stats64[-1].iters,
        "speedup_vs_fp64": round(ms64 / ms, 3), "fp64_dot2": args.fp64_dot2, "bf16_vcycle": bf16, "bf16_all_levels_vcycle": bf16_all,
        "levels": s0.nlevels,
        "e2e": {"value": round(statistics.median(e2e), 2), "unit": "ms", "h2d_bytes_per_step": int(bi),
                "d2h_bytes_per_step": int(bo)},
        "gpu_launches": int(launches), "clocks": clocks, "roofline": roof, "spmv_roofline": spmv_roof,
        "err_vs_fp64_gpu": err_vs_fp64,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(prob, sopts, args.workload)
        if args.workload == "c3":
            out["err_vs_oracle"] = companion_errors(amg, torch, opts, tol)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
