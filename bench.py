#!/usr/bin/env python
"""Benchmark of the fused pipelined CG hot path on one GB300 (JSON line on stdout).

Workload (one "step"): a full pipelined-CG solve (Alg. 2, two fused kernels per iteration,
device-side convergence test in a CUDA-graph WHILE loop) of the 3D 7-point Dirichlet
Laplacian on a 160^3 grid (n = 4,096,000, nnz = 28,518,400), FP64 CSR with int32 indices,
b = A x* with x* ~ U[-1, 1) (splitmix64), x0 = 0, to ||r|| <= 1e-8 ||b||.  The working set
(~522 MB) is larger than the 129 MB L2, so no flush is needed between steps.

value     = algorithmic HBM bytes of the solve / device time of the solve (GB/s), summed
            over ranks (replicas; the solver itself does not shard);
e2e       = the same metric through the C ABI with pinned HOST b and x (the library copies
            them in and the solution out inside the call);
roofline  = the fused SpMV + inner-products kernel (K-CG-S) timed with CUDA events over
            30 fixed iterations (the paper's Sec. 4 methodology) against the measured HBM
            copy bandwidth in MEASURED_PEAKS.json;
cpu_baseline / --impl reference = the plain FP64 CPU oracle on the same matrix.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import shutil
import statistics
import subprocess
import sys
import tempfile
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

from paper_1410_4054_gb300 import workloads as W  # noqa: E402

METRIC = "pipelined CG: algorithmic HBM GB/s over the solve to 1e-8 (time-to-1e-8 beside it)"
UNIT = "GB/s"
K3D = 160


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--k", type=int, default=K3D, help="3D grid side of the timed workload")
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--mode", default="bench", choices=["bench", "kernels", "conv"],
                    help="kernels: run only --iters fixed pipelined-CG iterations (profiler driver); "
                         "conv: time the BF16 conv kernels on one 64^3 layer")
    ap.add_argument("--iters", type=int, default=30)
    ap.add_argument("--variant", default="pipelined")
    ap.add_argument("--solver", default="cg", choices=["cg", "bicgstab", "gmres", "batched"],
                    help="--mode kernels: cg on the Laplacian, bicgstab / gmres on convection-diffusion, "
                         "batched on the 512 shifted rectangles")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"],
                    help="--mode kernels, cg / batched: FP64 or FP32-inner mixed precision")
    ap.add_argument("--matrix", default="stencil", choices=["stencil", "powerlaw", "fe3d"],
                    help="--mode kernels: the stencil of --k, a power-law matrix with --n rows, or P1 "
                         "elasticity on --k^3 cubes")
    ap.add_argument("--sell", action="store_true", help="--mode kernels, cg: K-CG-S on the SELL-C-sigma copy")
    ap.add_argument("--n", type=int, default=1_000_000)
    ap.add_argument("--lanes", type=int, default=0,
                    help="--mode kernels, batched: the engine (0 row engine automatic, 1/2/4/8 lanes per "
                         "row, -1 tile engine, -2 cluster engine)")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the BiCGStab / GMRES / batched / mixed-precision lines")
    return ap.parse_args()


def run_kernels(args):
    """A fixed number of CG iterations on the --k^3 Laplacian, host-driven launches: the
    command that the committed ncu summaries under profiles/ profile."""
    import torch
    from paper_1410_4054_gb300 import pk

    if args.solver == "batched":
        mats = W.batched_rectangles(512, seed=0)
        As = [pk.CSRMatrix.from_workload(m) for m in mats]
        bs = [torch.from_numpy(W.manufactured(m, seed=k)[1]).cuda() for k, m in enumerate(mats)]
        xs = [torch.zeros(m.n, dtype=torch.float64, device="cuda") for m in mats]
        infos = pk.batched_solve(As, bs, xs, tol=0.0, maxit=args.iters, precision=args.precision,
                                 lanes=args.lanes)
        torch.cuda.synchronize()
        print(json.dumps({"mode": "kernels", "solver": "batched", "systems": len(mats),
                          "iters": infos[0]["iters"], "solve_ms": infos[0]["solve_ms"]}))
        return 0
    if args.matrix == "powerlaw":
        a = W.power_law(args.n, seed=0)
    elif args.matrix == "fe3d":
        a = W.fe_elasticity_3d(args.k)
    else:
        a = W.laplace_3d(args.k) if args.solver == "cg" else W.convdiff_3d(args.k)
    _, b, _ = W.manufactured(a, seed=0)
    A = pk.CSRMatrix.from_workload(a)
    bd = torch.from_numpy(b).cuda()
    xd = torch.zeros(a.n, dtype=torch.float64, device="cuda")
    fn = {"cg": pk.cg_solve, "bicgstab": pk.bicgstab_solve, "gmres": pk.gmres_solve}[args.solver]
    info = fn(A, bd, xd, tol=0.0, maxit=args.iters, variant=args.variant, loop="host",
              check_every=args.iters, flags=pk.FLAG_SELL if args.sell else 0,
              **({"precision": args.precision} if args.solver == "cg" else {}))
    torch.cuda.synchronize()
    print(json.dumps({"mode": "kernels", "solver": args.solver, "k": args.k, "n": a.n, "iters": info["iters"],
                      "launches": info["launches"], "solve_ms": info["solve_ms"]}))
    return 0


def bytes_per_solve(n: int, nnz: int, iters: int) -> int:
    """Compulsory HBM bytes of a pipelined CG solve, each vector read/written once per kernel.

    matrix pass A = 12 nnz + 4 (n + 1); setup r0 = b - A x0 (A + 32 n); per iteration
    K-CG-U 56 n (read x, r, p, Ap; write x, r, p) and K-CG-S A + 16 n (gather p once, write Ap);
    the setup K-CG-S plus (iters - 1) loop K-CG-S launches = iters matrix passes.
    """
    a = 12 * nnz + 4 * (n + 1)
    return (a + 32 * n) + iters * (56 * n + a + 16 * n)


def spmv_dots_bytes(n: int, nnz: int) -> int:
    return 12 * nnz + 4 * (n + 1) + 16 * n


def update_bytes(n: int) -> int:
    return 56 * n


def workload_name(k: int) -> str:
    return f"lap3d_{k}"


L2_BYTES = 129_000_000  # GB300 L2


def working_set_bytes(n: int, nnz: int) -> int:
    """Bytes a CG solve keeps touching: the CSR matrix and the five vectors b, x, r, p, Ap."""
    return 12 * nnz + 4 * (n + 1) + 40 * n


def config(k: int, a) -> dict:
    ws = working_set_bytes(a.n, a.nnz)
    fits = "working set ~%d MB <= 129 MB L2: algorithmic GB/s may exceed HBM speed" % (ws // 10**6)
    return {"workload": f"pipelined CG (Alg. 2), 3D 7-point Laplacian {k}^3, n={a.n}, nnz={a.nnz}, "
                        f"FP64 CSR int32, x*~U[-1,1), b=A x*, x0=0, tol 1e-8",
            "n": a.n, "nnz": a.nnz, "tol": 1e-8, "solver": "pipelined_cg",
            "l2": fits if ws <= L2_BYTES else
                  "inputs larger than L2 (working set ~%d MB > 129 MB), no flush" % (ws // 10**6)}


# ------------------------------------------------------------------ clocks

class Clocks:
    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        exe = shutil.which("nvidia-smi")
        if not exe:
            return
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        self.proc = subprocess.Popen([exe, f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                      "--format=csv,noheader,nounits", "-lms", "100"],
                                     stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        # let the sampler finish its start-up (NVML initialisation can hold driver locks)
        # before the timed region begins: wait for its first sample, at most 5 s
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < 5.0 and self.proc.poll() is None:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.02)

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in Path(self.path).read_text().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = max(mx, float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ helpers

def measured_peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


KERNEL_SOURCES = ("pk_cg.cu", "pk_tile.cuh", "pk_internal.cuh")


def kernel_source_sha() -> str:
    """Hash of the sources that define the profiled CG kernels."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        h.update((ROOT / "paper_1410_4054_gb300" / "csrc" / name).read_bytes())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on this source."""
    p = ROOT / "profiles" / "ncu_traffic.json"
    if not p.exists():
        return None
    d = json.loads(p.read_text()).get(f"{kernel}@{workload}")
    if not d or d.get("source_sha") != kernel_source_sha():
        return None
    return d.get("bytes_per_launch")


def dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, pg, device) -> float:
    """The job's time is the slowest replica's: all-reduce MAX over the process group (the
    replicas share nothing else; there is no data-path collective)."""
    if pg is None:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def job_value(ws: int, bytes_per_replica: float, seconds: float) -> float:
    """Whole-job GB/s: every replica moves the same algorithmic bytes in the job's time."""
    return ws * bytes_per_replica / seconds / 1e9


# ------------------------------------------------------------------ CPU oracle arm

def host_cores() -> int:
    return len(os.sched_getaffinity(0))


def oracle_sample(a, b, iters: int) -> tuple[float, float]:
    """Seconds for `iters` oracle pipelined-CG iterations (tol = 0) on the same system."""
    import oracle as O
    O.lib()  # build / load outside the timed region
    t0 = time.perf_counter()
    O.cg(a, b, tol=0.0, maxit=iters, variant="pipelined", cap=1)
    return time.perf_counter() - t0, iters


def oracle_omp_sample(a, b, iters: int):
    """Seconds for `iters` pipelined-CG iterations of the OpenMP copy of the oracle on every
    core this process may use (static schedule), or None without OpenMP."""
    import oracle as O
    if O.omp_lib() is None:
        return None
    t0 = time.perf_counter()
    O.cg_omp(a, b, tol=0.0, maxit=iters, threads=host_cores())
    return time.perf_counter() - t0


def oracle_gbs(a, seconds: float, iters: int) -> float:
    per_iter = 56 * a.n + 12 * a.nnz + 4 * (a.n + 1) + 16 * a.n
    return per_iter * iters / seconds / 1e9


def cpu_legs(a, b, k: int, it1: int, itp: int) -> dict:
    """The CPU baseline: (i) the sequential parity oracle on one core, (ii) its OpenMP copy on
    every core of the host (static schedule, cores from sched_getaffinity); the faster one is
    reported, as the paper's Sec. 4 reports the best of 1/2/4/8 CPU processes."""
    s1, _ = oracle_sample(a, b, it1)
    legs = {"one_core": {"value": oracle_gbs(a, s1, it1), "cores": 1, "iters": it1, "s": s1}}
    cores = host_cores()
    sp = oracle_omp_sample(a, b, itp)
    if sp is not None:
        legs["all_cores"] = {"value": oracle_gbs(a, sp, itp), "cores": cores, "iters": itp, "s": sp}
    best = max(legs.values(), key=lambda v: v["value"])
    return {"value": best["value"], "unit": UNIT, "cores": best["cores"], "kind": "oracle",
            "sample": f"pipelined-CG iterations (tol=0) of the same {k}^3 system: "
                      + "; ".join(f"{v['iters']} its on {v['cores']} core(s) in {v['s']:.2f} s "
                                  f"= {v['value']:.1f} GB/s" for v in legs.values())
                      + "; faster leg reported",
            "legs": {name: round(v["value"], 2) for name, v in legs.items()}}


def run_reference(args):
    """The oracle arm: each step runs a bounded sample of the same workload (12 pipelined-CG
    iterations of the --k^3 system) on one core and on every core (OpenMP copy); the faster
    leg's median step time is the value."""
    ws, rank, _ = dist()
    if rank != 0:
        return 0
    import oracle as O

    a = W.laplace_3d(args.k)
    _, b, _ = W.manufactured(a, seed=0)
    it = 12
    cores = host_cores()
    have_omp = O.omp_lib() is not None
    for _ in range(args.warmup):
        oracle_sample(a, b, 2)
        if have_omp:
            oracle_omp_sample(a, b, 2)
    t1, tp = [], []
    for _ in range(args.steps):
        t1.append(oracle_sample(a, b, it)[0])
        if have_omp:
            tp.append(oracle_omp_sample(a, b, it))
    legs = {"one_core": (statistics.median(t1), 1)}
    if tp:
        legs["all_cores"] = (statistics.median(tp), cores)
    name, (sec, used) = min(legs.items(), key=lambda kv: kv[1][0])
    val = oracle_gbs(a, sec, it)
    line = {"metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sec, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": config(args.k, a),
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": used, "kind": "oracle",
                             "sample": f"{it} pipelined-CG iterations of the {args.k}^3 system per step, "
                                       f"on 1 core and on {cores} cores (OpenMP copy); {name} reported",
                             "legs": {k: round(oracle_gbs(a, v[0], it), 2) for k, v in legs.items()}},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU arm

def run_ours(args):
    import torch
    from paper_1410_4054_gb300 import pk

    ws, rank, local = dist()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py: no CUDA device; the pk library runs only on the GPU")
    torch.cuda.set_device(local)
    pg = None
    if ws > 1:
        import torch.distributed as td
        td.init_process_group("nccl")
        pg = td
    dev = f"cuda:{local}"
    a = W.laplace_3d(args.k)
    _, b, _ = W.manufactured(a, seed=rank)
    A = pk.CSRMatrix.from_workload(a)
    bd = torch.from_numpy(b).to(dev)
    xd = torch.zeros(a.n, dtype=torch.float64, device=dev)
    kw = dict(tol=1e-8, maxit=50_000, variant="pipelined", loop="graph")
    stream = torch.cuda.current_stream()

    def step():
        xd.zero_()
        return pk.cg_solve(A, bd, xd, **kw)

    for _ in range(max(args.warmup, 3)):
        info = step()
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    clocks = Clocks(local)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    launches = 0
    iters = []
    for _ in range(args.steps):
        info = step()
        launches += info["launches"]
        iters.append(info["iters"])
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, pg, dev)
    if pg:
        pg.barrier()
    it = iters[-1]
    bps = bytes_per_solve(a.n, a.nnz, it)
    value = job_value(ws, bps, ms * 1e-3)

    # end to end through the C ABI with pinned host buffers
    bh = torch.from_numpy(b).pin_memory()
    xh = torch.zeros(a.n, dtype=torch.float64).pin_memory()
    for _ in range(2):
        xh.zero_()
        pk.cg_solve(A, bh, xh, **kw)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        xh.zero_()
        pk.cg_solve(A, bh, xh, **kw)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / args.steps, pg, dev)
    e2e = {"value": job_value(ws, bps, e2e_s), "unit": UNIT, "h2d_bytes_per_step": 16 * a.n,
           "d2h_bytes_per_step": 8 * a.n, "ms_per_step": 1e3 * e2e_s}

    if rank != 0:
        if pg:
            pg.destroy_process_group()
        return 0

    # roofline of the dominant kernel: 30 fixed iterations with per-launch CUDA events
    prof = pk.cg_solve(A, bd, xd.zero_(), tol=0.0, maxit=30, flags=pk.FLAG_TIMING)
    t_s = prof["kernel_ms"]["spmv_dots"] * 1e-3
    t_u = prof["kernel_ms"]["update"] * 1e-3
    peak, peak_kind = measured_peaks()
    ach = spmv_dots_bytes(a.n, a.nnz) / t_s / 1e9
    roofline = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                "traffic": ncu_traffic("k_cg_spmv_dots", workload_name(args.k)),
                "kernel": "k_cg_spmv_dots_tma (K-CG-S)",
                "peak_source": "of measured (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                               else "of fallback",
                "algorithmic_bytes_per_launch": spmv_dots_bytes(a.n, a.nnz), "launch_ms": 1e3 * t_s}
    update_roofline = {"kernel": "k_cg_update_tma (K-CG-U)", "launch_ms": 1e3 * t_u,
                       "algorithmic_bytes_per_launch": update_bytes(a.n),
                       "achieved": update_bytes(a.n) / t_u / 1e9, "peak": peak,
                       "frac": update_bytes(a.n) / t_u / 1e9 / peak,
                       "fp64_tflops_k_cg_s": (2 * a.nnz + 4 * a.n) / t_s / 1e12}
    emit_detail("roofline_kernels", update_roofline)

    if not args.no_sweep:
        for row in size_sweep(pk, torch, dev):
            emit_detail("sweep", row)

    if not args.no_forms:
        bench_forms(pk, torch, dev, args, emit=lambda name, val: emit_detail("form:" + name, val))

    cpu = None
    if not args.no_cpu:
        cpu = cpu_legs(a, b, args.k, it1=60, itp=240)

    line = headline(value=value, ws=ws, args=args, ms=ms, cfg=config(args.k, a), it=it, launches=launches,
                    e2e=e2e, roofline=roofline, cpu=cpu, clk=clk)
    print(line, flush=True)
    if pg:
        pg.destroy_process_group()
    return 0


HEADLINE_MAX = 2048


def emit_detail(name: str, data) -> None:
    """One JSON line per sweep row / form, printed BEFORE the headline (the last line)."""
    print(json.dumps({"detail": name, "data": data}), flush=True)


def headline(*, value, ws, args, ms, cfg, it, launches, e2e, roofline, cpu, clk) -> str:
    """The benchmark's result line: printed last, one line, under HEADLINE_MAX bytes."""
    r = lambda v, d=4: None if v is None else round(float(v), d)  # noqa: E731
    line = {"metric": METRIC, "value": r(value, 2), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r(ms), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
            "time_to_tol_ms": r(ms), "iters": it, "iters_per_s": r(it / (ms * 1e-3), 1),
            "gpu_launches": launches,
            "e2e": {k: (r(v, 3) if isinstance(v, float) else v) for k, v in e2e.items()},
            "roofline": {k: (r(v) if isinstance(v, float) else v) for k, v in roofline.items()},
            "cpu_baseline": cpu, "clocks": clk}
    if cpu is not None:
        line["cpu_baseline"] = dict(cpu, value=r(cpu["value"], 3))
    s = json.dumps(line)
    if len(s) >= HEADLINE_MAX:
        raise RuntimeError(f"bench.py: headline line is {len(s)} bytes (limit {HEADLINE_MAX})")
    return s


def size_sweep(pk, torch, dev):
    """Pipelined CG to 1e-8 against the unfused classical CG on the same GPU, both from x0 = 0,
    best of two solves, over the 3D k^3 and 2D k^2 Laplacians of the size sweep."""
    sweep = []
    cases = [("lap3d", k) for k in W.LAPLACE_3D_SWEEP] + [("lap2d", k) for k in W.LAPLACE_2D_SWEEP]
    for kind, k in cases:
        m = W.laplace_3d(k) if kind == "lap3d" else W.laplace_2d(k)
        _, mb, _ = W.manufactured(m, seed=0)
        M = pk.CSRMatrix.from_workload(m)
        mbd = torch.from_numpy(mb).to(dev)
        mx = torch.zeros(m.n, dtype=torch.float64, device=dev)
        ws_b = working_set_bytes(m.n, m.nnz)
        # below the L2 size, algorithmic GB/s may exceed HBM speed (L2 bandwidth)
        row = {"matrix": f"{kind}_{k}", "n": m.n, "nnz": m.nnz, "working_set_mb": ws_b / 1e6,
               "below_l2_size": ws_b <= L2_BYTES}
        for variant, loop in (("pipelined", "graph"), ("pipelined", "persistent"),
                              ("classical", "graph")):
            key = variant if variant == "classical" else f"{variant}_{loop}"
            best = None
            try:
                for rep in range(2):
                    mx.zero_()
                    inf = pk.cg_solve(M, mbd, mx, tol=1e-8, maxit=50_000, variant=variant, loop=loop)
                    best = inf if best is None or inf["solve_ms"] < best["solve_ms"] else best
            except pk.PkError:  # the persistent grid does not fit this n
                row[f"{key}_iters"] = row[f"{key}_ms"] = None
                continue
            row[f"{key}_iters"] = best["iters"]
            row[f"{key}_ms"] = best["solve_ms"]
        # what the default loop (PK_LOOP_AUTO) runs at this n
        auto = ("persistent" if m.n <= pk.PERSISTENT_AUTO_N and m.nnz <= pk.PERSISTENT_AUTO_NNZ
                and row["pipelined_persistent_ms"]
                else "graph")
        row["pipelined_loop"] = auto
        row["pipelined_iters"] = row[f"pipelined_{auto}_iters"]
        row["pipelined_ms"] = row[f"pipelined_{auto}_ms"]
        row["pipelined_gbs"] = bytes_per_solve(m.n, m.nnz, row["pipelined_iters"]) / (row["pipelined_ms"] * 1e-3) / 1e9
        row["speedup_vs_classical"] = row["classical_ms"] / row["pipelined_ms"]
        sweep.append(row)
        M.close()
    return sweep


def _best(fn, reps=2):
    best = None
    for _ in range(reps):
        info = fn()
        if best is None or info["solve_ms"] < best["solve_ms"]:
            best = info
    return best


def bench_forms(pk, torch, dev, args, emit=None):
    """The other solvers and forms, each timed after one warm-up run (device time of the call).

    bicgstab / gmres: 3D convection-diffusion 128^3 (cell Peclet 0.5), tol 1e-8, pipelined vs
    classical on the same GPU, plus per-kernel times over 30 fixed iterations.
    batched: 512 shifted 2D Laplacians on rectangles with sides log-uniform in [32, 256], tol
    1e-10, one persistent launch (FP64 and mixed precision) vs 512 sequential plain solves.
    mixed: the 160^3 Laplacian to 1e-8, mixed precision vs FP64, error of the mixed solution.
    nonsymmetric_sweep: BiCGStab and GMRES(30) to 1e-8, pipelined vs classical, on the
    convection-diffusion matrices 32^3, 64^3, 128^3 and the power-law matrices n = 1e4, 1e5, 1e6.
    fused_spmv_dot: q = A p with <p, q> fused into the SpMV (one launch) against SpMV then an
    inner-product kernel (Sec. 2.2), random matrices with 4 and 28 nonzeros per row.
    learned_warm_start: the transient heat sequence on 64^3 (300 implicit steps, CG to 1e-8),
    the network trained on steps 2-150 and evaluated on 151-300 against the x_{t-1} warm start
    (and the linear extrapolation alone), plus the BF16 convolution kernels' throughput.
    Each form is handed to `emit(name, value)` as soon as it is measured.
    """
    out = {}

    def put(name, val):
        out[name] = val
        if emit:
            emit(name, val)
    a = W.convdiff_3d(128)
    _, b, _ = W.manufactured(a, seed=0)
    A = pk.CSRMatrix.from_workload(a)
    bd = torch.from_numpy(b).to(dev)
    x = torch.zeros(a.n, dtype=torch.float64, device=dev)
    for solver, fn in (("bicgstab", pk.bicgstab_solve), ("gmres", pk.gmres_solve)):
        row = {"matrix": "convdiff3d_128", "n": a.n, "nnz": a.nnz, "tol": 1e-8}
        for variant in ("pipelined", "classical"):
            kw = dict(tol=1e-8, maxit=20_000, variant=variant)
            if solver == "gmres":
                kw["restart"] = 30
            fn(A, bd, x.zero_(), **kw)
            inf = _best(lambda: fn(A, bd, x.zero_(), **kw))
            row[f"{variant}_ms"] = inf["solve_ms"]
            row[f"{variant}_iters"] = inf["iters"]
            row[f"{variant}_status"] = inf["status_name"]
        prof = fn(A, bd, x.zero_(), tol=0.0, maxit=30, flags=pk.FLAG_TIMING,
                  **({"restart": 30} if solver == "gmres" else {}))
        row["kernel_ms_30_fixed_iterations"] = prof["kernel_ms"]
        row["roofline"] = solver_rooflines(solver, a.n, a.nnz, prof["kernel_ms"])
        row["speedup_vs_classical"] = row["classical_ms"] / row["pipelined_ms"]
        put(solver, row)
    A.close()

    mats = W.batched_rectangles(512, seed=0)
    rhs = [W.manufactured(m, seed=k)[1] for k, m in enumerate(mats)]
    As = [pk.CSRMatrix.from_workload(m) for m in mats]
    bs = [torch.from_numpy(v).to(dev) for v in rhs]
    xs = [torch.zeros(m.n, dtype=torch.float64, device=dev) for m in mats]
    brow = {"systems": len(mats), "rows": int(sum(m.n for m in mats)),
            "nnz": int(sum(m.nnz for m in mats)), "tol": 1e-10}
    res = {}
    for prec in ("fp64", "mixed"):
        kw = dict(tol=1e-10, maxit=20_000, precision=prec, flags=pk.FLAG_AUTOTUNE)
        pk.batched_solve(As, bs, [v.zero_() for v in xs], **kw)   # tunes, then warm
        times = []
        for _ in range(3):
            infos = pk.batched_solve(As, bs, [v.zero_() for v in xs], **kw)
            times.append(infos[0]["solve_ms"])
        ms = min(times)
        brow[f"{prec}_ms"] = ms
        brow[f"{prec}_solves_per_s"] = len(mats) / (ms * 1e-3)
        brow[f"{prec}_all_converged"] = all(i["status"] == pk.PK_OK for i in infos)
        brow[f"{prec}_config"] = list(pk.batched_last_config()) + [pk.batched_last_lanes()]
        # algorithmic bytes of every system's iterations (FP64: 12 nnz + 76 n per iteration;
        # mixed: the FP32 inner iteration, 8 nnz + 40 n) over the launch time
        per_it = [(12 * m.nnz + 76 * m.n) if prec == "fp64" else (8 * m.nnz + 40 * m.n) for m in mats]
        moved = sum(i["iters"] * b_ for i, b_ in zip(infos, per_it))
        gbs = moved / (ms * 1e-3) / 1e9
        brow[f"{prec}_roofline"] = {"bound": "hbm", "achieved": gbs, "peak": measured_peaks()[0],
                                    "unit": "GB/s", "frac": gbs / measured_peaks()[0],
                                    "note": "sum over systems of iterations x algorithmic bytes per iteration"}
        res[prec] = [v.clone() for v in xs]
    errs = [float(torch.linalg.norm(xm - x64) / torch.linalg.norm(x64))
            for xm, x64 in zip(res["mixed"], res["fp64"]) if float(torch.linalg.norm(x64)) > 0]
    brow["mixed_max_rel_error_vs_fp64"] = max(errs)
    # sequential plain FP64 solves (CUDA-graph loop per system), the same systems
    for k in range(4):
        pk.cg_solve(As[k], bs[k], xs[k].zero_(), tol=1e-10, maxit=20_000)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(len(mats)):
        pk.cg_solve(As[k], bs[k], xs[k].zero_(), tol=1e-10, maxit=20_000)
    torch.cuda.synchronize()
    seq = time.perf_counter() - t0
    brow["sequential_plain_ms"] = 1e3 * seq
    brow["sequential_plain_solves_per_s"] = len(mats) / seq
    brow["speedup_fp64_batched_vs_sequential"] = brow["sequential_plain_ms"] / brow["fp64_ms"]
    put("batched", brow)
    for M in As:
        M.close()
    put("batched_fe", batched_fe(pk, torch, dev))

    a = W.laplace_3d(args.k)
    _, b, _ = W.manufactured(a, seed=0)
    A = pk.CSRMatrix.from_workload(a)
    bd = torch.from_numpy(b).to(dev)
    x64 = torch.zeros(a.n, dtype=torch.float64, device=dev)
    xm = torch.zeros(a.n, dtype=torch.float64, device=dev)
    pk.cg_solve(A, bd, xm.zero_(), tol=1e-8, maxit=50_000, precision="mixed")
    i64 = _best(lambda: pk.cg_solve(A, bd, x64.zero_(), tol=1e-8, maxit=50_000))
    im = _best(lambda: pk.cg_solve(A, bd, xm.zero_(), tol=1e-8, maxit=50_000, precision="mixed",
                                   flags=pk.FLAG_TRUE_RES))
    mixed = {"matrix": f"lap3d_{args.k}", "tol": 1e-8, "fp64_ms": i64["solve_ms"],
                    "mixed_ms": im["solve_ms"], "speedup": i64["solve_ms"] / im["solve_ms"],
                    "refinement_steps": im["cycles"], "inner_iters": im["iters"],
                    "fp64_iters": i64["iters"], "mixed_rel_res_true": im["rel_res_true"],
                    "rel_error_vs_fp64": float(torch.linalg.norm(xm - x64) / torch.linalg.norm(x64)),
                    "inner_bytes_per_iter": 8 * a.nnz + 40 * a.n}
    mixed_bytes = im["iters"] * (8 * a.nnz + 40 * a.n) + (im["cycles"] + 1) * (12 * a.nnz + 4 * (a.n + 1) + 16 * a.n)
    gbs = mixed_bytes / (im["solve_ms"] * 1e-3) / 1e9
    mixed["roofline"] = {"bound": "hbm", "achieved": gbs, "peak": measured_peaks()[0], "unit": "GB/s",
                         "frac": gbs / measured_peaks()[0],
                         "note": "inner FP32 iterations x (8 nnz + 40 n) + FP64 residuals, over the solve"}
    put("mixed", mixed)
    A.close()

    put("jacobi_pcg", jacobi_pcg(pk, torch, dev, args.k))
    put("jacobi_right", jacobi_right(pk, torch, dev))
    put("gmres_variants", gmres_variants(pk, torch, dev))
    put("fe_sweep", fe_sweep(pk, torch, dev))
    put("sell", sell_compare(pk, torch, dev, args.k))
    put("nonsymmetric_sweep", nonsymmetric_sweep(pk, torch, dev))
    put("fused_spmv_dot", fused_spmv_dot(pk, torch, dev))

    from paper_1410_4054_gb300 import warmstart as WS

    res = WS.run_transient(k=64, steps=300, train_last=150, epochs=30)
    lw = {k: v for k, v in res.items() if not isinstance(v, list)}
    lw["train_ms_per_sample"] = 1e3 * res["train_s"] / (res["epochs"] * res["train_samples"])
    lw["iteration_gain_vs_plain_warm_start"] = res["baseline_mean_iters"] - res["learned_mean_iters"]
    lw["relaxed_iteration_gain_vs_extrapolation"] = res["extrap_mean_iters"] - res["learned_relaxed_mean_iters"]
    lw["conv"] = conv_throughput(pk, torch, dev, (64, 64, 64))
    bf16_peak = bf16_peak_tflops()
    lw["conv"]["roofline"] = {"bound": "tensor", "peak": bf16_peak, "unit": "TFLOP/s",
                              "peak_source": "measured (MEASURED_PEAKS.json bf16_tflops)",
                              **{f"{k}_frac": lw["conv"][f"{k}_tflops"] / bf16_peak
                                 for k in ("fwd", "bwd_data", "wgrad")}}
    put("learned_warm_start", lw)
    return out


FP64_NOMINAL_TFLOPS = 1.25  # GB300 FP64 (vector and tensor), nominal


def bf16_peak_tflops():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        return float(json.loads(p.read_text())["bf16_tflops"])
    return 1900.0


def solver_rooflines(solver, n, nnz, km):
    """Per-kernel achieved GB/s (algorithmic bytes per launch / mean launch time of 30 fixed
    iterations) against the measured HBM copy bandwidth; the Gram-Schmidt kernels also
    against the nominal FP64 rate, which bounds them on GB300."""
    peak = measured_peaks()[0]
    spmv = 12 * nnz + 4 * (n + 1) + 24 * n
    out = {}

    def hbm(name, bytes_, ms):
        if ms:
            gbs = bytes_ / (ms * 1e-3) / 1e9
            out[name] = {"bound": "hbm", "bytes_per_launch": bytes_, "launch_ms": ms, "achieved_gbs": gbs,
                         "peak_gbs": peak, "frac": gbs / peak}

    if solver == "bicgstab":
        hbm("K-BI-1/3 (SpMV + dots)", spmv, km.get("spmv_dots"))
        hbm("K-BI-2/4 (updates + dots), mean of 24n and 72n", 48 * n, km.get("update"))
    else:
        hbm("K-GM-1 (SpMV + <v_{i-1}, v_i>)", spmv, km.get("spmv_dots"))
        hbm("K-GM-4 (normalise + xi)", 24 * n, km.get("update"))
        steps = range(1, 31)
        for name, slot, vecs, fmas in (("K-GM-2 (inner products)", "multidot",
                                        lambda i: i - 1 if i >= 3 else 0, lambda i: max(i - 2, 0)),
                                       ("K-GM-3 (CGS update + norm)", "ortho",
                                        lambda i: i + 1, lambda i: i)):
            ms = km.get(slot)
            if not ms:
                continue
            b_ = 8 * n * sum(vecs(i) for i in steps) / 30
            f_ = 2 * n * sum(fmas(i) for i in steps) / 30
            gbs = b_ / (ms * 1e-3) / 1e9
            tf = f_ / (ms * 1e-3) / 1e12
            out[name] = {"bound": "fp64", "bytes_per_launch_mean": b_, "launch_ms": ms, "achieved_gbs": gbs,
                         "frac_hbm": gbs / peak, "fp64_tflops": tf, "fp64_peak_tflops": FP64_NOMINAL_TFLOPS,
                         "frac": tf / FP64_NOMINAL_TFLOPS, "peak_source": "nominal FP64"}
    return out


def batched_fe(pk, torch, dev, nsys=256):
    """Batched FP64 pipelined CG on 256 uneven P1 elasticity systems (k = 3..7 cubes: 144 to
    1,536 rows, up to 45 nonzeros per row) to 1e-10: solves/s with the autotuned block shape
    and lanes per row, against one thread per row (lanes = 1, its best block shape)."""
    ks = 3 + (W.splitmix64(7, nsys) % np.uint64(5)).astype(int)
    mats = [W.fe_elasticity_3d(int(k), seed=i) for i, k in enumerate(ks)]
    rhs = [W.manufactured(m, seed=i)[1] for i, m in enumerate(mats)]
    As = [pk.CSRMatrix.from_workload(m) for m in mats]
    bs = [torch.from_numpy(v).to(dev) for v in rhs]
    xs = [torch.zeros(m.n, dtype=torch.float64, device=dev) for m in mats]
    row = {"systems": nsys, "rows": int(sum(m.n for m in mats)), "nnz": int(sum(m.nnz for m in mats)), "tol": 1e-10}
    for key, lanes in (("tuned", 0), ("one_lane", 1)):
        kw = dict(tol=1e-10, maxit=20_000, flags=pk.FLAG_AUTOTUNE, lanes=lanes)
        pk.batched_solve(As, bs, [v.zero_() for v in xs], **kw)
        ms = min(pk.batched_solve(As, bs, [v.zero_() for v in xs], **kw)[0]["solve_ms"] for _ in range(3))
        infos = pk.batched_solve(As, bs, [v.zero_() for v in xs], **kw)
        row[f"{key}_ms"] = ms
        row[f"{key}_solves_per_s"] = nsys / (ms * 1e-3)
        row[f"{key}_all_converged"] = all(i["status"] == pk.PK_OK for i in infos)
        row[f"{key}_config"] = list(pk.batched_last_config()) + [pk.batched_last_lanes()]
    row["speedup_tuned_vs_one_lane"] = row["one_lane_ms"] / row["tuned_ms"]
    for M in As:
        M.close()
    return row


def jacobi_pcg(pk, torch, dev, k):
    """Jacobi-preconditioned pipelined CG against plain pipelined CG, tol 1e-8, on two badly
    scaled SPD matrices D A D (ln d uniform on [0, ln 100)): the k^3 Laplacian and the SPD
    power-law matrix with 10^6 rows.  Best of two solves after a warm-up; per-kernel
    rooflines from 30 fixed iterations."""
    peak = measured_peaks()[0]
    rows = []
    for a in (W.diag_scaled(W.laplace_3d(k), seed=0, spread=100.0),
              W.diag_scaled(W.spd_power_law(1_000_000, seed=1), seed=1, spread=100.0)):
        _, b, _ = W.manufactured(a, seed=0)
        A = pk.CSRMatrix.from_workload(a)
        bd = torch.from_numpy(b).to(dev)
        x = torch.zeros(a.n, dtype=torch.float64, device=dev)
        row = {"matrix": a.name, "n": a.n, "nnz": a.nnz, "tol": 1e-8}
        for pre in ("jacobi", "none"):
            kw = dict(tol=1e-8, maxit=50_000, precond=pre, loop="graph")
            pk.cg_solve(A, bd, x.zero_(), **kw)
            inf = _best(lambda: pk.cg_solve(A, bd, x.zero_(), flags=pk.FLAG_TRUE_RES, **kw))
            row[f"{pre}_ms"] = inf["solve_ms"]
            row[f"{pre}_iters"] = inf["iters"]
            row[f"{pre}_status"] = inf["status_name"]
            row[f"{pre}_rel_res_true"] = inf["rel_res_true"]
        row["speedup_vs_plain_cg"] = row["none_ms"] / row["jacobi_ms"]
        per_it = 12 * a.nnz + 92 * a.n + 4
        row["bytes_per_iteration"] = per_it
        gbs = per_it * row["jacobi_iters"] / (row["jacobi_ms"] * 1e-3) / 1e9
        row["solve_roofline"] = {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                                 "frac": gbs / peak}
        prof = pk.cg_solve(A, bd, x.zero_(), tol=0.0, maxit=30, precond="jacobi", flags=pk.FLAG_TIMING)
        km = prof["kernel_ms"]
        for name, slot, bytes_ in (("K-PCG-S (SpMV + <p,Ap>, <Ap,M^-1 Ap>)", "spmv_dots", 12 * a.nnz + 28 * a.n + 4),
                                   ("K-PCG-U (x, r, p updates + <r,M^-1 r>, <r,r>)", "update", 64 * a.n)):
            ms = km.get(slot)
            if ms:
                g = bytes_ / (ms * 1e-3) / 1e9
                row.setdefault("kernel_rooflines", {})[name] = {
                    "bytes_per_launch": bytes_, "launch_ms": ms, "achieved_gbs": g, "frac": g / peak}
        rows.append(row)
        A.close()
    return rows


def jacobi_right(pk, torch, dev, k=128):
    """Right-Jacobi BiCGStab and GMRES(30) against the plain solvers, tol 1e-8, pipelined, on
    the badly scaled convection-diffusion matrix D A D (k^3, ln d uniform on [0, ln 100)).
    Best of two solves after a warm-up.  The preconditioned solve runs the same kernels on the
    column-scaled values, so its time per iteration should equal the plain one's."""
    a = W.diag_scaled(W.convdiff_3d(k), seed=0, spread=100.0)
    _, b, _ = W.manufactured(a, seed=0)
    A = pk.CSRMatrix.from_workload(a)
    bd = torch.from_numpy(b).to(dev)
    x = torch.zeros(a.n, dtype=torch.float64, device=dev)
    out = {}
    for solver, fn, extra in (("bicgstab", pk.bicgstab_solve, {}), ("gmres", pk.gmres_solve, {"restart": 30})):
        row = {"matrix": a.name, "n": a.n, "nnz": a.nnz, "tol": 1e-8}
        for pre in ("jacobi", "none"):
            kw = dict(tol=1e-8, maxit=20_000, precond=pre, **extra)
            fn(A, bd, x.zero_(), **kw)
            inf = _best(lambda: fn(A, bd, x.zero_(), flags=pk.FLAG_TRUE_RES, **kw))
            row[f"{pre}_ms"] = inf["solve_ms"]
            row[f"{pre}_iters"] = inf["iters"]
            row[f"{pre}_status"] = inf["status_name"]
            row[f"{pre}_rel_res_true"] = inf["rel_res_true"]
            row[f"{pre}_us_per_iter"] = 1e3 * inf["solve_ms"] / max(inf["iters"], 1)
        row["speedup_vs_plain"] = row["none_ms"] / row["jacobi_ms"]
        out[solver] = row
    A.close()
    return out


def sell_compare(pk, torch, dev, k, reps=20):
    """Fused SpMV + inner products on the SELL-C-sigma copy against the CSR kernels.
    spmv_dot: q = A p, <p, q> as one launch, CSR thread-per-row (the paper's design) and
    SELL-C-sigma (warp per 32-row slice), CUDA events over `reps` calls; bytes 12 nnz + 4 (n+1)
    + 16 n (the SELL copy reads its padding and no row pointers: its own bytes are reported too).
    CG (SPD matrices): K-CG-S on the CSR tiles and on SELL, mean launch time over 30 fixed
    iterations (PK_FLAG_TIMING)."""
    out = []
    for a, spd in ((W.laplace_3d(k), True), (W.fe_elasticity_3d(47), True),
                   (W.spd_power_law(1_000_000, seed=1), True), (W.random_uniform(1_000_000, 28, seed=1), False)):
        A = pk.CSRMatrix.from_workload(a)
        p = torch.from_numpy(W.uniform_pm1(3, a.n)).to(dev)
        q = torch.empty_like(p)
        res = torch.zeros(1, dtype=torch.float64, device=dev)
        row = {"matrix": a.name, "n": a.n, "nnz": a.nnz, "csr_bytes": 12 * a.nnz + 4 * (a.n + 1) + 16 * a.n}
        for key, kw in (("csr_thread", {"fused": True}), ("sell", {"sell": True})):
            for _ in range(3):
                pk.spmv_dot(A, p, q, res, **kw)
            st, en = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            st.record()
            for _ in range(reps):
                pk.spmv_dot(A, p, q, res, **kw)
            en.record()
            torch.cuda.synchronize()
            us = 1e3 * st.elapsed_time(en) / reps
            row[f"spmv_dot_{key}_us"] = us
            row[f"spmv_dot_{key}_gbs"] = row["csr_bytes"] / (us * 1e-6) / 1e9
        if spd:
            _, b, _ = W.manufactured(a, seed=0)
            bd = torch.from_numpy(b).to(dev)
            x = torch.zeros(a.n, dtype=torch.float64, device=dev)
            for key, fl in (("tiles", 0), ("sell", pk.FLAG_SELL)):
                best = None
                for _ in range(2):
                    inf = pk.cg_solve(A, bd, x.zero_(), tol=0.0, maxit=30, flags=pk.FLAG_TIMING | fl)
                    ms = inf["kernel_ms"]["spmv_dots"]
                    best = ms if best is None else min(best, ms)
                row[f"k_cg_s_{key}_us"] = 1e3 * best
                row[f"k_cg_s_{key}_gbs"] = (12 * a.nnz + 4 * (a.n + 1) + 16 * a.n) / (best * 1e-3) / 1e9
        out.append(row)
        A.close()
    return out


def fe_sweep(pk, torch, dev):
    """Time per iteration against system size on finite-element matrices (the shape of the
    paper's Sec. 4.1 / 4.2 benchmarks): P1 Poisson on irregular triangulations of the unit
    square, 225 ... 261,121 unknowns (~7 per row), and P1 elasticity on jittered Kuhn
    tetrahedra, 540 ... 324,864 unknowns (3 x 3 blocks, ~43 per row).  CG, BiCGStab and
    GMRES(30), pipelined and classical, a fixed number of iterations (tol 0) through the graph
    loop; CG, BiCGStab and GMRES also through PK_LOOP_AUTO (the cluster-resident loop for
    small systems), GMRES also in the three-kernel form.  Best of two after a warm-up, microseconds
    per iteration (solve time / iterations)."""
    mats = [("fe2d", lv, lambda lv=lv: W.fe_poisson_2d(lv)) for lv in range(4, 10)]
    mats += [("fe3d", k, lambda k=k: W.fe_elasticity_3d(k)) for k in (5, 11, 23, 47)]
    forms = [("cg", pk.cg_solve, "pipelined", "graph", 300, {}), ("cg", pk.cg_solve, "classical", "graph", 300, {}),
             ("cg", pk.cg_solve, "pipelined", "auto", 300, {}),
             ("bicgstab", pk.bicgstab_solve, "pipelined", "graph", 150, {}),
             ("bicgstab", pk.bicgstab_solve, "classical", "graph", 150, {}),
             ("bicgstab", pk.bicgstab_solve, "pipelined", "auto", 150, {}),
             ("gmres", pk.gmres_solve, "pipelined", "graph", 120, {"restart": 30, "flags": pk.FLAG_GM_SHIFT}),
             ("gmres", pk.gmres_solve, "pipelined", "auto", 120, {"restart": 30}),
             ("gmres", pk.gmres_solve, "pipelined", "graph", 120, {"restart": 30}),
             ("gmres", pk.gmres_solve, "classical", "graph", 120, {"restart": 30})]
    rows = []
    for kind, size, make in mats:
        a = make()
        _, b, _ = W.manufactured(a, seed=0)
        A = pk.CSRMatrix.from_workload(a)
        bd = torch.from_numpy(b).to(dev)
        x = torch.zeros(a.n, dtype=torch.float64, device=dev)
        row = {"matrix": a.name, "n": a.n, "nnz": a.nnz}
        for solver, fn, variant, loop, its, extra in forms:
            kw = dict(tol=0.0, maxit=its, variant=variant, loop=loop, **extra)
            fn(A, bd, x.zero_(), **kw)
            inf = _best(lambda: fn(A, bd, x.zero_(), **kw))
            key = f"{solver}_{variant}" + ("_auto" if loop == "auto" else "") + ("_shift3" if extra.get("flags") else "")
            row[f"{key}_us_per_iter"] = 1e3 * inf["solve_ms"] / max(inf["iters"], 1)
        rows.append(row)
        A.close()
        del a
    return rows


def gmres_variants(pk, torch, dev):
    """Pipelined GMRES(30) to 1e-8 in three forms: four kernels per step with one
    Gram-Schmidt pass ('cgs', Alg. 6), two passes (PK_FLAG_CGS2, six kernels), and the
    shift-invariant three-kernel form (PK_FLAG_GM_SHIFT): iterations, cycles, time per step
    and solve time, on the 32^3 and 128^3 convection-diffusion matrices, the 128^3 one
    diagonally scaled (spread 100, right Jacobi) and the power-law matrix with 10^6 rows.
    Best of two after a warm-up."""
    out = []
    for a, pre in ((W.convdiff_3d(32), "none"), (W.convdiff_3d(128), "none"),
                   (W.diag_scaled(W.convdiff_3d(128), seed=0, spread=100.0), "jacobi"),
                   (W.power_law(1_000_000, seed=0), "none")):
        _, b, _ = W.manufactured(a, seed=0)
        A = pk.CSRMatrix.from_workload(a)
        bd = torch.from_numpy(b).to(dev)
        x = torch.zeros(a.n, dtype=torch.float64, device=dev)
        row = {"matrix": a.name, "n": a.n, "nnz": a.nnz, "precond": pre, "tol": 1e-8}
        for key, fl in (("cgs", 0), ("cgs2", pk.FLAG_CGS2), ("shift3", pk.FLAG_GM_SHIFT)):
            kw = dict(tol=1e-8, maxit=20_000, restart=30, precond=pre)
            pk.gmres_solve(A, bd, x.zero_(), flags=fl, **kw)
            inf = _best(lambda: pk.gmres_solve(A, bd, x.zero_(), flags=fl | pk.FLAG_TRUE_RES, **kw))
            row[f"{key}_ms"] = inf["solve_ms"]
            row[f"{key}_iters"] = inf["iters"]
            row[f"{key}_cycles"] = inf["cycles"]
            row[f"{key}_status"] = inf["status_name"]
            row[f"{key}_rel_res_true"] = inf["rel_res_true"]
            row[f"{key}_us_per_step"] = 1e3 * inf["solve_ms"] / max(inf["iters"], 1)
        out.append(row)
        A.close()
    return out


def nonsymmetric_sweep(pk, torch, dev):
    """BiCGStab and GMRES(30) solve times (best of two after a warm-up) on the paper's
    nonsymmetric workload shapes."""
    rows = []
    mats = [("convdiff3d", k, lambda k=k: W.convdiff_3d(k)) for k in (32, 64, 128)] + \
           [("powerlaw", n, lambda n=n: W.power_law(n, seed=0)) for n in (10_000, 100_000, 1_000_000)]
    for kind, size, make in mats:
        a = make()
        _, b, _ = W.manufactured(a, seed=0)
        A = pk.CSRMatrix.from_workload(a)
        bd = torch.from_numpy(b).to(dev)
        x = torch.zeros(a.n, dtype=torch.float64, device=dev)
        row = {"matrix": f"{kind}_{size}", "n": a.n, "nnz": a.nnz}
        for solver, fn in (("bicgstab", pk.bicgstab_solve), ("gmres", pk.gmres_solve)):
            for variant in ("pipelined", "classical"):
                kw = dict(tol=1e-8, maxit=20_000, variant=variant)
                if solver == "gmres":
                    kw["restart"] = 30
                fn(A, bd, x.zero_(), **kw)
                inf = _best(lambda: fn(A, bd, x.zero_(), **kw))
                row[f"{solver}_{variant}_ms"] = inf["solve_ms"]
                row[f"{solver}_{variant}_iters"] = inf["iters"]
                row[f"{solver}_{variant}_status"] = inf["status_name"]
            row[f"{solver}_speedup"] = row[f"{solver}_classical_ms"] / row[f"{solver}_pipelined_ms"]
        rows.append(row)
        A.close()
    return rows


def fused_spmv_dot(pk, torch, dev, reps=20):
    """Sec. 2.2 experiment: fused q = A p, <p, q> (one kernel) against the unfused pair, CUDA
    events over `reps` calls after a warm-up.  Bytes per call: 12 nnz + 4 (n + 1) + 16 n."""
    out = []
    for per_row, sizes in ((4, (1_000, 10_000, 100_000, 1_000_000, 10_000_000)),
                           (28, (1_000, 10_000, 100_000, 1_000_000))):
        for n in sizes:
            a = W.random_uniform(n, per_row, seed=1)
            A = pk.CSRMatrix.from_workload(a)
            p = torch.from_numpy(np.random.default_rng(2).uniform(-1, 1, a.n)).to(dev)
            q = torch.empty_like(p)
            res = torch.zeros(1, dtype=torch.float64, device=dev)
            row = {"per_row": per_row, "n": n, "nnz": a.nnz}
            for fused in (True, False):
                for _ in range(3):
                    pk.spmv_dot(A, p, q, res, fused=fused)
                st, en = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                st.record()
                for _ in range(reps):
                    pk.spmv_dot(A, p, q, res, fused=fused)
                en.record()
                torch.cuda.synchronize()
                us = 1e3 * st.elapsed_time(en) / reps
                key = "fused" if fused else "unfused"
                row[f"{key}_us"] = us
                row[f"{key}_gbs"] = (12 * a.nnz + 4 * (a.n + 1) + 16 * a.n) / (us * 1e-6) / 1e9
            row["speedup"] = row["unfused_us"] / row["fused_us"]
            out.append(row)
            A.close()
    return out


def conv_throughput(pk, torch, dev, dims, reps=20):
    """CUDA-event times of the BF16 conv kernels on a 16 -> 16 channel layer: forward (ReLU,
    BF16 out), backward-data (flipped weights, ReLU mask) and weight gradient.  FLOPs are those
    of the padded implicit GEMM, 2 x 27 x 16 x 16 per voxel."""
    nvox = int(np.prod(dims))
    g = torch.Generator(device=dev).manual_seed(0)
    X = torch.randn(dims + (16,), generator=g, device=dev).to(torch.bfloat16)
    Gr = torch.randn(dims + (16,), generator=g, device=dev).to(torch.bfloat16)
    Wt = (0.1 * torch.randn((27, 16, 16), generator=g, device=dev)).to(torch.bfloat16)
    Wf = torch.empty_like(Wt)
    pk.conv3d_flip(Wt, Wf)
    bias = torch.zeros(16, device=dev)
    Y = torch.empty_like(X)
    dX = torch.empty_like(X)
    scratch = torch.zeros(pk.conv3d_wgrad_scratch_floats(dims), device=dev)
    dW = torch.zeros((27, 16, 16), device=dev)
    db = torch.zeros(16, device=dev)
    calls = {"fwd": lambda: pk.conv3d_fwd(X, Wt, bias, Y, dims, relu=True),
             "bwd_data": lambda: pk.conv3d_fwd(Gr, Wf, None, dX, dims, relu=False, mask=X),
             "wgrad": lambda: pk.conv3d_wgrad(X, Gr, scratch, dW, db, dims)}
    flops = 2 * 27 * 16 * 16 * nvox
    out = {"dims": list(dims), "gflop_per_call": flops / 1e9}
    for name, fn in calls.items():
        for _ in range(3):
            fn()
        st, en = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        st.record()
        for _ in range(reps):
            fn()
        en.record()
        torch.cuda.synchronize()
        us = 1e3 * st.elapsed_time(en) / reps
        out[f"{name}_us"] = us
        out[f"{name}_tflops"] = flops / (us * 1e-6) / 1e12
    return out


def main():
    args = parse()
    if args.mode == "kernels":
        return run_kernels(args)
    if args.mode == "conv":
        import torch
        from paper_1410_4054_gb300 import pk

        print(json.dumps({"mode": "conv", **conv_throughput(pk, torch, "cuda", (64, 64, 64))}))
        pk.conv3d_check()
        return 0
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
