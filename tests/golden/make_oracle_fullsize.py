"""Writes tests/golden/oracle_fullsize.json: the oracle's full-size solves of the benchmark
workloads, which take minutes on one core and so are stored instead of recomputed by every
GPU test run.  Calls only oracle/ (and the seeded input generators); nothing here comes from
the CUDA library.

For every case (solver, matrix) it records, at tol 1e-8 from x0 = 0:
  - iters, cycles, status of the oracle's solve;
  - iters_perturbed: the iteration counts of the same solve with b perturbed by about one ulp
    (b (1 + 2^-52 u), u = uniform_pm1(100 + s)), s = 0, 1 (s = 0 .. 7 for BiCGStab) -- the
    oracle's own rounding spread;
  - x_idx / x_vals: 64 sampled entries of the oracle's x after `iters` iterations, and
    x_fixed_spread: the largest change of those entries (relative to their largest magnitude)
    under the same perturbations, x taken after exactly `iters` iterations (tol = 0);
  - matrix_sha / b_sha: hashes of the generated matrix and right-hand side, so that a test on
    another machine can tell whether it regenerated exactly the same inputs.

Run:  python tests/golden/make_oracle_fullsize.py [--jobs N]   (about 15 min on 8 cores)
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import sys
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parents[2]
OUT = Path(__file__).resolve().parent / "oracle_fullsize.json"

# (solver, matrix name) -> the workload; GMRES restarts after 30 steps
CASES = [("cg", "lap3d_160"), ("cg", "lap2d_2048"),
         ("bicgstab", "convdiff_128"), ("gmres", "convdiff_128"),
         ("bicgstab", "powerlaw_1e5"), ("gmres", "powerlaw_1e5"),
         ("bicgstab", "powerlaw_1e6"), ("gmres", "powerlaw_1e6")]
TOL = 1e-8
MAXIT = 50_000
NSAMPLE = 64


def npert(solver):
    """One-ulp perturbations per case: BiCGStab's iteration count is the most rounding-sensitive
    (its spread on the power-law matrices is tens of iterations), so it gets more samples."""
    return 8 if solver == "bicgstab" else 2


def matrix(name):
    sys.path.insert(0, str(ROOT))
    from paper_1410_4054_gb300 import workloads as W
    return {"lap3d_160": lambda: W.laplace_3d(160), "lap2d_2048": lambda: W.laplace_2d(2048),
            "convdiff_128": lambda: W.convdiff_3d(128),
            "powerlaw_1e5": lambda: W.power_law(100_000, seed=0),
            "powerlaw_1e6": lambda: W.power_law(1_000_000, seed=0)}[name]()


def sha(*arrays) -> str:
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()[:24]


def run(solver, a, b, tol, maxit):
    sys.path.insert(0, str(ROOT))
    import oracle as O
    if solver == "cg":
        return O.cg(a, b, tol=tol, maxit=maxit, variant="pipelined", cap=1)
    if solver == "bicgstab":
        return O.bicgstab(a, b, tol=tol, maxit=maxit, variant="pipelined", cap=1)
    return O.gmres(a, b, tol=tol, maxit=maxit, m=30, variant="pipelined", cap=1)


def inputs(name, smp):
    """The matrix and b (smp = -1: unperturbed; else the one-ulp perturbation number smp)."""
    sys.path.insert(0, str(ROOT))
    from paper_1410_4054_gb300 import workloads as W
    a = matrix(name)
    _, b, _ = W.manufactured(a, seed=0)
    if smp >= 0:
        b = b * (1 + 2.0 ** -52 * W.uniform_pm1(100 + smp, a.n))
    return a, b


def job(spec):
    """One oracle solve: ('base', solver, name) / ('pert', solver, name, s) / ('fixed', solver,
    name, s, iters)."""
    kind, solver, name = spec[:3]
    if kind == "base":
        a, b = inputs(name, -1)
        r = run(solver, a, b, TOL, MAXIT)
        idx = np.sort(np.random.default_rng(12345).choice(a.n, NSAMPLE, replace=False))
        return spec, {"n": a.n, "nnz": a.nnz, "matrix_sha": sha(a.row_ptr, a.col, a.val), "b_sha": sha(b),
                      "iters": int(r["iters"]), "cycles": int(r.get("cycles", 0)), "status": int(r["status"]),
                      "x_idx": idx.tolist(), "x_vals": r["x"][idx].tolist(),
                      "x_norm": float(np.linalg.norm(r["x"]))}
    if kind == "pert":
        a, b = inputs(name, spec[3])
        return spec, int(run(solver, a, b, TOL, MAXIT)["iters"])
    a, b = inputs(name, spec[3])
    return spec, run(solver, a, b, 0.0, spec[4])["x"]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=8)
    ap.add_argument("--only", default=None, help="comma-separated solver:matrix keys")
    args = ap.parse_args()
    cases = CASES
    if args.only:
        keep = set(args.only.split(","))
        cases = [c for c in CASES if f"{c[0]}:{c[1]}" in keep]
    ctx = mp.get_context("spawn")
    out = json.loads(OUT.read_text())["cases"] if OUT.exists() else {}
    with ctx.Pool(args.jobs) as pool:
        first = [("base", s, m) for s, m in cases] + [("pert", s, m, k) for s, m in cases for k in range(npert(s))]
        res = dict(pool.map(job, first, chunksize=1))
        fixed = [("fixed", s, m, k, res[("base", s, m)]["iters"]) for s, m in cases for k in range(npert(s))]
        fres = dict(pool.map(job, fixed, chunksize=1))
    for s, m in cases:
        rec = res[("base", s, m)]
        rec["iters_perturbed"] = [res[("pert", s, m, k)] for k in range(npert(s))]
        idx = np.array(rec["x_idx"])
        xv = np.array(rec["x_vals"])
        scale = np.abs(xv).max()
        rec["x_fixed_spread"] = max(float(np.abs(fres[("fixed", s, m, k, rec["iters"])][idx] - xv).max() / scale)
                                    for k in range(npert(s)))
        rec["tol"] = TOL
        out[f"{s}:{m}"] = rec
        print(s, m, rec["iters"], rec["iters_perturbed"], rec["x_fixed_spread"], flush=True)
    OUT.write_text(json.dumps({"generated_by": "tests/golden/make_oracle_fullsize.py",
                               "perturbation": "b (1 + 2^-52 uniform_pm1(100 + s, n)), s = 0..1 (0..7 for BiCGStab)",
                               "sample": "64 indices from numpy default_rng(12345).choice(n, 64), sorted",
                               "cases": out}, indent=1) + "\n")


if __name__ == "__main__":
    main()
