"""GPU parity of restarted GMRES(m) (pipelined Alg. 6, classical Alg. 5) against the oracle.

Per step the solver traces R_{i-1,i}, R_{i,i}, xi_i and the residual estimate; the first
cycle's values are compared with the oracle's R and xi relative to max |R| (the scalars of
this method, R14), iterations to tol within +-2, x at the oracle's iteration count within
1e-9, and the true residual at exit within tol.
"""
import numpy as np
import pytest

import oracle as O
from _parity import record
from paper_1410_4054_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1410_4054_gb300 import pk  # noqa: E402

DEV = "cuda:0"


def dev(v):
    return torch.from_numpy(np.ascontiguousarray(v, dtype=np.float64)).to(DEV)


def solve(a, b, x0=None, A=None, trace_cap=256, **kw):
    A = A or pk.CSRMatrix.from_workload(a)
    x = dev(np.zeros(a.n) if x0 is None else x0)
    tr = torch.full((trace_cap, 4), float("nan"), dtype=torch.float64, device=DEV)
    info = pk.gmres_solve(A, dev(b), x, trace=tr, **kw)
    torch.cuda.synchronize()
    return info, x.cpu().numpy(), tr.cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


MATRICES = {
    "dense_rows_1e4": lambda: W.spd_dense_rows(),
    "fe2d_p1_961": lambda: W.fe_poisson_2d(5),
    "fe3d_elast_540": lambda: W.fe_elasticity_3d(5),
    "convdiff_16": lambda: W.convdiff_3d(16),
    "convdiff_23": lambda: W.convdiff_3d(23),
    "powerlaw_1e4": lambda: W.power_law(10_000, seed=1),
    "rand28": lambda: W.random_uniform(4000, 28, seed=2),
    "lap2d_ragged": lambda: W.laplace_2d(97, 41),
}


def oracle_sensitivity(a, b, variant, m, tol, maxit, nsamp=3, precond="none", cgs2=False, shift3=False):
    """The oracle's own rounding sensitivity: rerun it with b perturbed by about one ulp
    (relative 2^-52, three seeds); running maxima of the change of R (relative to max |R|)
    and xi per step of the first cycle, of the iteration count and of x at a fixed count."""
    kw = dict(m=m, variant=variant, precond=precond, cgs2=cgs2, shift3=shift3)
    base = O.gmres(a, b, tol=tol, maxit=maxit, **kw)
    fixed = O.gmres(a, b, tol=0.0, maxit=max(base["iters"], 1), **kw)
    k = min(m, max(base["iters"], 1))
    sR = np.zeros(k)
    sX = np.zeros(k)
    it_spread, x_spread = 0, 0.0
    scale = np.abs(base["R"][:k, :k]).max()
    for smp in range(nsamp):
        bp = b * (1 + 2.0 ** -52 * W.uniform_pm1(100 + smp, a.n))
        r = O.gmres(a, bp, tol=tol, maxit=maxit, **kw)
        dR = np.abs(r["R"][:k, :k] - base["R"][:k, :k]).max(axis=0) / scale
        sR = np.fmax(sR, dR)
        sX = np.fmax(sX, np.abs(r["xi"][:k] - base["xi"][:k]))
        it_spread = max(it_spread, abs(r["iters"] - base["iters"]))
        rf = O.gmres(a, bp, tol=0.0, maxit=max(base["iters"], 1), **kw)
        x_spread = max(x_spread, rel(rf["x"], fixed["x"]))
    return base, fixed, np.maximum.accumulate(sR), np.maximum.accumulate(sX), it_spread, x_spread


def first_cycle_lengths(tr, ref, steps):
    """Length of the first cycle: the oracle's nonzero R diagonal; on the GPU the trace of a
    cycle's first step has R_{0,1} = 0."""
    k_orc = int(np.count_nonzero(np.diag(ref["R"])))
    nxt = [j for j in range(1, steps) if tr[j, 0] == 0.0]
    return k_orc, (nxt[0] if nxt else steps)


def full_R_check(A, a, b, ref, sR, sX, k, case, m=30, **kw):
    """Every entry R_{j,i}, j <= i <= k, of the first cycle (K-GM-2 forms R_{j,i} for
    j <= i - 2, K-GM-1 R_{i-1,i}, K-GM-3 R_{i,i}) and xi_1..xi_k, read back after a solve of
    exactly k steps, against the oracle's first cycle: column i within max(1e-12, 100 x the
    oracle's own one-ulp spread of that column) relative to max |R|, xi as in the trace."""
    info, _, _ = solve(a, b, A=A, tol=0.0, maxit=k, restart=m, **kw)
    assert info["iters"] == k and info["cycles"] == 1
    R, xi = pk.gmres_cycle_factors(A, m)
    Ro = ref["R"][:k, :k]
    scale = np.abs(Ro).max()
    dcol = np.abs(np.triu(R[:k, :k]) - np.triu(Ro)).max(axis=0) / scale
    bars = np.maximum(1e-12, 100 * sR[:k])
    record("gmres_full_R", case, f"R_(j,i), i <= {k} (rel. max|R|)", float(dcol.max()), 1e-12, float(bars.max()),
           oracle_spread=float(sR[:k].max()))
    assert np.all(dcol <= bars), (dcol, bars)
    dxi = np.abs(xi[:k] - ref["xi"][:k])
    barx = np.maximum(1e-12, 100 * sX[:k])
    record("gmres_full_R", case, f"xi_i, i <= {k}", float(dxi.max()), 1e-12, float(barx.max()),
           oracle_spread=float(sX[:k].max()))
    assert np.all(dxi <= barx), (dxi, barx)
    assert np.all(np.tril(R[:k, :k], -1) == 0.0)


def first_cycle_check(tr, ref, sR, sX, steps, case=""):
    """R_{i-1,i}, R_{i,i} (relative to max |R|) and xi_i (absolute, |xi| <= 1) within
    max(1e-12, 100 x the oracle's own one-ulp spread) at every step of the first cycle; the
    steps where the oracle itself is insensitive meet 1e-12 outright."""
    R, xi = ref["R"], ref["xi"]
    # The end-of-cycle test compares 1 - sum xi^2 with a floor, so rounding may move the
    # boundary by one step: compare the steps both took.
    k_orc, k_gpu = first_cycle_lengths(tr, ref, steps)
    assert abs(k_orc - k_gpu) <= 1, (k_orc, k_gpu)
    k = min(len(sR), steps, k_orc, k_gpu)
    scale = np.abs(R[:k, :k]).max()
    dR = max(abs(tr[i - 1, 1] - R[i - 1, i - 1]) for i in range(1, k + 1)) / scale
    dX = max(abs(tr[i - 1, 2] - xi[i - 1]) for i in range(1, k + 1))
    record("gmres_trace", f"{case} k={k}", "R_(i-1,i), R_(i,i) (rel. max|R|)", dR, 1e-12,
           float(max(1e-12, 100 * sR[k - 1])), oracle_spread=float(sR[k - 1]))
    record("gmres_trace", f"{case} k={k}", "xi_i", dX, 1e-12, float(max(1e-12, 100 * sX[k - 1])),
           oracle_spread=float(sX[k - 1]))
    for i in range(1, k + 1):
        barR = max(1e-12, 100 * sR[i - 1]) * scale
        barX = max(1e-12, 100 * sX[i - 1])
        if i >= 2:
            assert abs(tr[i - 1, 0] - R[i - 2, i - 1]) <= barR, (i, "R_{i-1,i}")
        assert abs(tr[i - 1, 1] - R[i - 1, i - 1]) <= barR, (i, "R_ii")
        assert abs(tr[i - 1, 2] - xi[i - 1]) <= barX, (i, "xi")
    assert (sX[: min(3, k)] < 1e-14).all()


JACOBI_MATRICES = {
    "convdiff_16_scaled": lambda: W.diag_scaled(W.convdiff_3d(16), seed=1, spread=100.0),
    "powerlaw_1e4_scaled": lambda: W.diag_scaled(W.power_law(10_000, seed=1), seed=2, spread=100.0),
    "lap2d_ragged_scaled": lambda: W.diag_scaled(W.laplace_2d(97, 41), seed=4, spread=10.0),
}


CGS2_MATRICES = {
    "convdiff_16": lambda: W.convdiff_3d(16),
    "powerlaw_1e4": lambda: W.power_law(10_000, seed=1),
    "fe3d_elast_540": lambda: W.fe_elasticity_3d(5),
    "convdiff10_scaled": lambda: W.diag_scaled(W.convdiff_3d(10), seed=3, spread=100.0),
}


# the shift-invariant three-kernel form (pipelined only)
SHIFT3_MATRICES = {
    "convdiff_16": lambda: W.convdiff_3d(16),
    "convdiff_23": lambda: W.convdiff_3d(23),
    "powerlaw_1e4": lambda: W.power_law(10_000, seed=1),
    "fe3d_elast_540": lambda: W.fe_elasticity_3d(5),
    "lap2d_ragged": lambda: W.laplace_2d(97, 41),
    "rand28": lambda: W.random_uniform(4000, 28, seed=2),
    "dense_rows_1e4": lambda: W.spd_dense_rows(),
}

PARITY_CASES = ([(n, v, lp) for n in sorted(MATRICES) + [f"jacobi:{k}" for k in sorted(JACOBI_MATRICES)]
                 for v, lp in (("classical", "graph"), ("pipelined", "graph"), ("pipelined", "persistent"))]
                + [(f"cgs2:{k}", v, "graph") for k in sorted(CGS2_MATRICES) for v in ("classical", "pipelined")]
                + [(f"shift3:{k}", "pipelined", "graph") for k in sorted(SHIFT3_MATRICES)]
                + [("shift3:jacobi:convdiff_16_scaled", "pipelined", "graph")])


@pytest.mark.parametrize("name,variant,loop", PARITY_CASES)
def test_gmres_parity(name, variant, loop):
    """'jacobi:' cases: right preconditioning with M = diag(A) on both sides; 'cgs2:' cases:
    Gram-Schmidt applied twice per step on both sides; 'shift3:' cases: the shift-invariant
    three-kernel form on both sides.  loop 'graph': the kernels of a step launched from a CUDA
    graph; 'persistent': the whole restarted loop on one thread-block cluster."""
    shift3 = name.startswith("shift3:")
    if shift3:
        name = name[7:]
    precond = "jacobi" if name.startswith("jacobi:") else "none"
    cgs2 = name.startswith("cgs2:")
    if precond == "jacobi":
        a = JACOBI_MATRICES[name[7:]]()
    elif cgs2:
        a = CGS2_MATRICES[name[5:]]()
    elif shift3:
        a = SHIFT3_MATRICES[name]()
    else:
        a = MATRICES[name]()
    _, b, _ = W.manufactured(a, seed=0)
    m = 30
    ref, fixed, sR, sX, it_spread, x_spread = oracle_sensitivity(a, b, variant, m, 1e-8, 20_000,
                                                                 precond=precond, cgs2=cgs2, shift3=shift3)
    assert ref["status"] == O.OK
    fl = pk.FLAG_CGS2 if cgs2 else pk.FLAG_GM_SHIFT if shift3 else 0
    if shift3:
        name = "shift3:" + name
    A = pk.CSRMatrix.from_workload(a)
    info, x, tr = solve(a, b, A=A, tol=1e-8, maxit=20_000, restart=m, variant=variant,
                        flags=pk.FLAG_TRUE_RES | fl, trace_cap=max(256, ref["iters"] + 8), precond=precond, loop=loop)
    assert info["status"] == pk.PK_OK, info
    assert info["rel_res_true"] <= 1.5e-8
    if loop == "persistent":
        assert info["launches"] <= 4 + (2 if precond == "jacobi" else 0), info["launches"]
    case = f"{name} {variant} {loop}"
    first_cycle_check(tr, ref, sR, sX, ref["iters"], case)
    k_orc, k_gpu = first_cycle_lengths(tr, ref, ref["iters"])
    full_R_check(A, a, b, ref, sR, sX, min(k_orc, k_gpu, len(sR)), case, m=m, variant=variant,
                 precond=precond, flags=fl, loop=loop)
    if k_orc == k_gpu or ref["iters"] <= min(k_orc, k_gpu):
        d_it = abs(info["iters"] - ref["iters"])
        record("gmres_parity", case, "iterations", d_it, 2, max(2, 2 * it_spread), oracle_spread=it_spread)
        assert d_it <= max(2, 2 * it_spread)
        info2, x2, _ = solve(a, b, tol=0.0, maxit=ref["iters"], restart=m, variant=variant, precond=precond,
                             flags=fl, loop=loop)
        assert info2["iters"] == ref["iters"] and info2["cycles"] == fixed["cycles"]
        d_x = rel(x2, fixed["x"])
        record("gmres_parity", case, "x at the oracle's count", d_x, 1e-9, max(1e-9, 10 * x_spread),
               oracle_spread=x_spread)
        assert d_x <= max(1e-9, 10 * x_spread)
    else:
        # rounding moved the end of the first cycle by one step (R17): the restart points
        # differ, so the totals may differ by up to one cycle; x is compared over the steps
        # both took (a fixed count that ends the first cycle on both sides)
        record("gmres_parity", case, "iterations (first cycle ended one step apart)",
               abs(info["iters"] - ref["iters"]), 2, m, oracle_spread=it_spread)
        assert info["iters"] <= ref["iters"] + m
        k = min(k_orc, k_gpu)
        _, fixed_k, _, _, _, xs_k = oracle_sensitivity(a, b, variant, m, 0.0, k, precond=precond, cgs2=cgs2,
                                                       shift3=shift3)
        info2, x2, _ = solve(a, b, tol=0.0, maxit=k, restart=m, variant=variant, precond=precond, flags=fl,
                             loop=loop)
        assert info2["iters"] == k and info2["cycles"] == fixed_k["cycles"]
        assert rel(x2, fixed_k["x"]) <= max(1e-9, 10 * xs_k)


def test_gmres_jacobi_unit_diagonal_and_clean_handle():
    a = W.convdiff_3d(12)
    u = W.CSR(a.n, a.row_ptr, a.col, a.val / 9.0, "convdiff_unit_diag")
    _, b, _ = W.manufactured(u, seed=1)
    for variant in ("pipelined", "classical"):
        A = pk.CSRMatrix.from_workload(u)
        i1, x1, t1 = solve(u, b, A=A, variant=variant, restart=20)
        i2, x2, t2 = solve(u, b, A=A, variant=variant, restart=20, precond="jacobi")
        assert i1["iters"] == i2["iters"] and np.array_equal(x1, x2)
        assert np.array_equal(t1, t2, equal_nan=True)
    s = W.diag_scaled(a, seed=5, spread=100.0)
    _, b, _ = W.manufactured(s, seed=2)
    A = pk.CSRMatrix.from_workload(s)
    i1, x1, _ = solve(s, b, A=A, tol=1e-8, maxit=20_000, restart=30)
    ij, _, _ = solve(s, b, A=A, tol=1e-8, maxit=20_000, restart=30, precond="jacobi", flags=pk.FLAG_TRUE_RES)
    i3, x3, _ = solve(s, b, A=A, tol=1e-8, maxit=20_000, restart=30)
    assert i1["iters"] == i3["iters"] and np.array_equal(x1, x3)
    assert ij["status"] == pk.PK_OK and ij["rel_res_true"] <= 1.5e-8 and ij["iters"] < i1["iters"]


@pytest.mark.parametrize("loop", ["graph", "host", "persistent"])
@pytest.mark.parametrize("m", [1, 5, 30, 64])
def test_gmres_restart_lengths_and_loops(m, loop):
    a = W.convdiff_3d(12)
    _, b, _ = W.manufactured(a, seed=3)
    ref = O.gmres(a, b, tol=1e-9, maxit=5000, m=m)
    info, x, _ = solve(a, b, tol=1e-9, maxit=5000, restart=m, loop=loop, check_every=1,
                       flags=pk.FLAG_TRUE_RES)
    assert info["status"] == pk.PK_OK and abs(info["iters"] - ref["iters"]) <= 2
    assert abs(info["cycles"] - ref["cycles"]) <= 1
    assert info["rel_res_true"] <= 1.5e-9


def test_gmres_launch_counts():
    """Sec. 3.3: four kernels per pipelined Arnoldi step (the classical form here: seven);
    CGS2 adds a second K-GM-2 / K-GM-3 pair; the shift-invariant form takes three."""
    a = W.convdiff_3d(10)
    _, b, _ = W.manufactured(a)
    per = {}
    for variant in ("pipelined", "classical"):
        for fl, tag in ((0, ""), (pk.FLAG_CGS2, "+cgs2"), (pk.FLAG_GM_SHIFT, "+shift")):
            if variant == "classical" and fl == pk.FLAG_GM_SHIFT:
                continue
            i10, _, _ = solve(a, b, tol=0.0, maxit=10, restart=30, variant=variant, flags=fl, loop="graph")
            i20, _, _ = solve(a, b, tol=0.0, maxit=20, restart=30, variant=variant, flags=fl, loop="graph")
            per[variant + tag] = (i20["launches"] - i10["launches"]) / 10
    assert per == {"pipelined": 4, "classical": 7, "pipelined+cgs2": 6, "classical+cgs2": 9, "pipelined+shift": 3}


def test_gmres_shift_form_rejections_and_loops():
    """PK_FLAG_GM_SHIFT is a form of pipelined GMRES with one Gram-Schmidt pass; the host loop
    and the graph give the same iterates; restart lengths 1 .. 64 match the oracle."""
    a = W.convdiff_3d(12)
    _, b, _ = W.manufactured(a, seed=3)
    A = pk.CSRMatrix.from_workload(a)
    for kw in (dict(variant="classical"), dict(flags=pk.FLAG_GM_SHIFT | pk.FLAG_CGS2)):
        kw.setdefault("flags", pk.FLAG_GM_SHIFT)
        with pytest.raises(RuntimeError, match="PK_FLAG_GM_SHIFT"):
            pk.gmres_solve(A, dev(b), dev(np.zeros(a.n)), **kw)
    for m in (1, 5, 30, 64):
        ref = O.gmres(a, b, tol=1e-9, maxit=5000, m=m, shift3=True)
        out = {}
        for loop in ("graph", "host"):
            info, x, tr = solve(a, b, A=A, tol=1e-9, maxit=5000, restart=m, loop=loop, check_every=1,
                                flags=pk.FLAG_GM_SHIFT | pk.FLAG_TRUE_RES)
            assert info["status"] == pk.PK_OK and abs(info["iters"] - ref["iters"]) <= 2, (m, loop, info["iters"])
            assert info["rel_res_true"] <= 1.5e-9
            out[loop] = (info["iters"], x)
        assert out["graph"][0] == out["host"][0] and np.array_equal(out["graph"][1], out["host"][1])


@pytest.mark.parametrize("make", [lambda: W.diag_scaled(W.laplace_2d(40), seed=3, spread=1e3),
                                  lambda: W.diag_scaled(W.fe_elasticity_3d(5), seed=6, spread=1e3)])
def test_gmres_cgs2_estimate_matches_true_residual(make):
    """After a full cycle of 30 pipelined steps the in-cycle estimate rho0 sqrt(1 - sum xi^2)
    equals ||b - A x|| to 1e-9 with CGS2 (the basis stays orthonormal), on the GPU as in the
    oracle."""
    a = make()
    _, b, _ = W.manufactured(a, seed=1)
    info, x, tr = solve(a, b, tol=0.0, maxit=30, restart=30, flags=pk.FLAG_CGS2 | pk.FLAG_TRUE_RES)
    assert info["iters"] == 30
    true = info["rel_res_true"] * np.linalg.norm(b)
    assert abs(tr[29, 3] - true) <= 1e-9 * true


def test_cgs2_flag_rejected_elsewhere():
    a = W.laplace_2d(20)
    _, b, _ = W.manufactured(a)
    A = pk.CSRMatrix.from_workload(a)
    for fn in (pk.cg_solve, pk.bicgstab_solve):
        with pytest.raises(RuntimeError, match="PK_FLAG_CGS2"):
            fn(A, dev(b), dev(np.zeros(a.n)), flags=pk.FLAG_CGS2)


def test_gmres_edge_cases():
    a = W.convdiff_3d(6)
    _, b, _ = W.manufactured(a)
    info, x, _ = solve(a, np.zeros(a.n), x0=np.ones(a.n))
    assert info["status"] == pk.PK_OK and info["iters"] == 0 and not x.any()
    info, _, _ = solve(a, b, maxit=0)
    assert info["status"] == pk.PK_NOT_CONVERGED and info["iters"] == 0
    ref = O.gmres(a, b, tol=0.0, maxit=13, m=5)
    info, x, _ = solve(a, b, tol=0.0, maxit=13, restart=5)
    assert info["status"] == pk.PK_NOT_CONVERGED and info["iters"] == 13 and info["cycles"] == 3
    assert rel(x, ref["x"]) <= 1e-10
    # full GMRES on a tiny system: lucky breakdown / precision floor end the cycle
    t = W.random_uniform(24, 5, seed=2)
    _, tb, _ = W.manufactured(t, seed=2)
    ref = O.gmres(t, tb, tol=1e-11, maxit=200, m=30)
    info, tx, _ = solve(t, tb, tol=1e-11, maxit=200, restart=30)
    assert info["status"] == pk.PK_OK and abs(info["iters"] - ref["iters"]) <= 2
    assert rel(tx, np.linalg.solve(t.to_dense(), tb)) < 1e-9


def test_gmres_large_convdiff():
    """128^3 convection-diffusion: the first 20 steps' full R column and xi (read back after a
    20-step solve) and the traced R_ii, xi against the oracle, x after 20 steps, then the full
    GMRES(30) solve checked by its true residual (its step count is compared with the stored
    oracle solve in test_gpu_fullsize.py)."""
    a = W.convdiff_3d(128)
    _, b, _ = W.manufactured(a)
    k = 20
    ref = O.gmres(a, b, tol=0.0, maxit=k, m=30)
    A = pk.CSRMatrix.from_workload(a)
    info, xk, tr = solve(a, b, A=A, tol=0.0, maxit=k, restart=30)
    scale = np.abs(ref["R"][:k, :k]).max()
    sR, sX = np.zeros(k), np.zeros(k)
    for smp in range(2):
        bp = b * (1 + 2.0 ** -52 * W.uniform_pm1(100 + smp, a.n))
        pert = O.gmres(a, bp, tol=0.0, maxit=k, m=30)
        sR = np.fmax(sR, np.abs(pert["R"][:k, :k] - ref["R"][:k, :k]).max(axis=0) / scale)
        sX = np.fmax(sX, np.abs(pert["xi"][:k] - ref["xi"][:k]))
    sR, sX = np.maximum.accumulate(sR), np.maximum.accumulate(sX)
    for i in range(1, k + 1):
        assert abs(tr[i - 1, 1] - ref["R"][i - 1, i - 1]) <= max(1e-12, 100 * sR[i - 1]) * scale
        assert abs(tr[i - 1, 2] - ref["xi"][i - 1]) <= max(1e-12, 100 * sX[i - 1])
    full_R_check(A, a, b, ref, sR, sX, k, "convdiff_128")
    assert rel(xk, ref["x"]) <= 1e-9
    info, _, _ = solve(a, b, A=A, tol=1e-8, maxit=20_000, restart=30, flags=pk.FLAG_TRUE_RES)
    assert info["status"] == pk.PK_OK and info["rel_res_true"] <= 1.5e-8


def test_gmres_persistent_selection_and_limits():
    """PK_LOOP_AUTO runs small pipelined GMRES on one cluster with the iterates of
    PK_LOOP_PERSISTENT; the persistent loop takes one Gram-Schmidt pass of the pipelined form
    only, n up to 16 x 4096 rows; the graph runs above PK_PERSISTENT_GMRES_AUTO_N."""
    a = W.convdiff_3d(20)
    _, b, _ = W.manufactured(a, seed=5)
    A = pk.CSRMatrix.from_workload(a)
    ia, xa, ta = solve(a, b, A=A, loop="auto", restart=30)
    ip, xp, tp = solve(a, b, A=A, loop="persistent", restart=30)
    assert ia["launches"] == ip["launches"] <= 4 and ia["iters"] == ip["iters"] and np.array_equal(xa, xp)
    assert np.array_equal(ta, tp, equal_nan=True)
    for kw in (dict(variant="classical"), dict(flags=pk.FLAG_CGS2), dict(flags=pk.FLAG_GM_SHIFT)):
        with pytest.raises(RuntimeError, match="PK_LOOP_PERSISTENT"):
            solve(a, b, A=A, loop="persistent", **kw)
    big = W.convdiff_3d(41)  # 68,921 rows
    _, bb, _ = W.manufactured(big, seed=1)
    with pytest.raises(RuntimeError, match="PK_LOOP_PERSISTENT"):
        solve(big, bb, loop="persistent")
    mid = W.convdiff_3d(36)  # 46,656 rows: fits one cluster, above the automatic threshold
    _, bm, _ = W.manufactured(mid, seed=1)
    ig, _, _ = solve(mid, bm, loop="auto", tol=0.0, maxit=3)
    ip, _, _ = solve(mid, bm, loop="persistent", tol=0.0, maxit=3)
    assert ig["launches"] > 4 and ip["launches"] <= 4
