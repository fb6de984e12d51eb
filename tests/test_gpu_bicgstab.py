"""GPU parity of BiCGStab (pipelined Alg. 4 with four fused kernels, classical Alg. 3) against
the CPU oracle: alpha, beta, omega within 1e-12 relative over the first iterations,
iterations to tol within +-2, x within 1e-9 of the oracle's at the same iteration count."""
import numpy as np
import pytest

import oracle as O
from _parity import count_gate, median, perturbed_b, record
from paper_1410_4054_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1410_4054_gb300 import pk  # noqa: E402

DEV = "cuda:0"


def dev(v):
    return torch.from_numpy(np.ascontiguousarray(v, dtype=np.float64)).to(DEV)


def solve(a, b, x0=None, A=None, trace_cap=64, **kw):
    A = A or pk.CSRMatrix.from_workload(a)
    x = dev(np.zeros(a.n) if x0 is None else x0)
    tr = torch.full((trace_cap, 4), float("nan"), dtype=torch.float64, device=DEV)
    info = pk.bicgstab_solve(A, dev(b), x, trace=tr, **kw)
    torch.cuda.synchronize()
    return info, x.cpu().numpy(), tr.cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


MATRICES = {
    "dense_rows_1e4": lambda: W.spd_dense_rows(),
    "fe2d_p1_961": lambda: W.fe_poisson_2d(5),
    "fe3d_elast_540": lambda: W.fe_elasticity_3d(5),
    "convdiff_16": lambda: W.convdiff_3d(16),
    "convdiff_23": lambda: W.convdiff_3d(23),   # ragged tiles
    "powerlaw_1e4": lambda: W.power_law(10_000, seed=1),
    "rand28": lambda: W.random_uniform(4000, 28, seed=2),
    "lap2d_ragged": lambda: W.laplace_2d(97, 41),
}


def oracle_sensitivity(a, b, variant, tol=1e-8, maxit=5000, nsamp=8, nsamp_x=3, precond="none"):
    """The oracle's own rounding sensitivity: rerun it with b perturbed by about one ulp
    (relative 2^-52, eight seeds) and record how far alpha, omega, beta (running maximum of
    the relative change per iteration) and the iteration count move (the counts of b and of
    the eight perturbed right-hand sides), and (first three seeds) x at a fixed count."""
    base = O.bicgstab(a, b, tol=tol, maxit=maxit, variant=variant, precond=precond)
    fixed = O.bicgstab(a, b, tol=0.0, maxit=max(base["iters"], 1), variant=variant, precond=precond)
    k = 20
    spread = np.zeros(k)
    counts, x_spread = [base["iters"]], 0.0
    for smp in range(nsamp):
        bp = perturbed_b(W, b, smp)
        r = O.bicgstab(a, bp, tol=tol, maxit=maxit, variant=variant, precond=precond)
        for key in ("alpha", "omega", "beta"):
            d = np.abs(r[key][:k] - base[key][:k]) / np.abs(base[key][:k])
            spread = np.fmax(spread, np.nan_to_num(d, nan=0.0))
        counts.append(r["iters"])
        if smp < nsamp_x:
            rf = O.bicgstab(a, bp, tol=0.0, maxit=max(base["iters"], 1), variant=variant, precond=precond)
            x_spread = max(x_spread, rel(rf["x"], fixed["x"]))
    return base, fixed, np.maximum.accumulate(spread), counts, x_spread


JACOBI_MATRICES = {
    "convdiff_16_scaled": lambda: W.diag_scaled(W.convdiff_3d(16), seed=1, spread=100.0),
    "powerlaw_1e4_scaled": lambda: W.diag_scaled(W.power_law(10_000, seed=1), seed=2, spread=100.0),
    "rand28_scaled": lambda: W.diag_scaled(W.random_uniform(4000, 28, seed=2), seed=3, spread=10.0),
    "lap2d_ragged_scaled": lambda: W.diag_scaled(W.laplace_2d(97, 41), seed=4, spread=10.0),
}


PARITY_CASES = [(n, v, lp) for n in sorted(MATRICES) + [f"jacobi:{k}" for k in sorted(JACOBI_MATRICES)]
                for v, lp in (("classical", "graph"), ("pipelined", "graph"), ("pipelined", "persistent"))]


@pytest.mark.parametrize("name,variant,loop", PARITY_CASES)
def test_bicgstab_parity(name, variant, loop):
    """Bars: alpha/omega/beta within max(1e-12, 100 x the oracle's own one-ulp spread) per
    iteration; the median iteration count over b and eight one-ulp perturbations of it within
    half the oracle's range + 2 of the oracle's median (count_gate); x at the oracle's
    iteration count within max(1e-9, 10 x the oracle's own spread); true residual <= tol.
    'jacobi:' cases: right preconditioning with M = diag(A) on both sides.  loop 'graph': the
    four fused kernels per iteration; 'persistent': the whole loop on one thread-block
    cluster."""
    precond = "jacobi" if name.startswith("jacobi:") else "none"
    a = JACOBI_MATRICES[name[7:]]() if precond == "jacobi" else MATRICES[name]()
    _, b, _ = W.manufactured(a, seed=0)
    ref, fixed, spread, orc_counts, x_spread = oracle_sensitivity(a, b, variant, precond=precond)
    assert ref["status"] == O.OK
    A = pk.CSRMatrix.from_workload(a)
    info, x, tr = solve(a, b, A=A, tol=1e-8, maxit=5000, variant=variant, flags=pk.FLAG_TRUE_RES,
                        precond=precond, loop=loop)
    assert info["status"] == pk.PK_OK, info
    if loop == "persistent":
        assert info["launches"] <= 4 + (2 if precond == "jacobi" else 0), info["launches"]  # (+1: true residual)
    case = f"{name} {variant} {loop}"
    # the iteration count: the GPU's counts on the same right-hand sides as the oracle's
    gpu_counts = [info["iters"]] + [solve(a, perturbed_b(W, b, k), A=A, tol=1e-8, maxit=5000, variant=variant,
                                          precond=precond, loop=loop)[0]["iters"] for k in range(len(orc_counts) - 1)]
    d_med = abs(median(gpu_counts) - median(orc_counts))
    record("bicgstab_parity", case, "iterations (one run)", abs(info["iters"] - ref["iters"]), 2,
           count_gate(orc_counts), oracle_counts=orc_counts, gpu_counts=gpu_counts)
    record("bicgstab_parity", case, "iterations (median of 9 right-hand sides)", d_med, 2, count_gate(orc_counts))
    assert d_med <= count_gate(orc_counts), (gpu_counts, orc_counts)
    k = min(20, ref["iters"] - 1)
    bar = np.maximum(1e-12, 100 * spread[:k])
    for col, key in ((0, "alpha"), (2, "omega"), (1, "beta")):
        dev_ = np.abs(tr[:k, col] - ref[key][:k]) / np.abs(ref[key][:k])
        record("bicgstab_parity", case, f"{key} (first {k})", float(np.nanmax(dev_)), 1e-12, float(bar.max()),
               oracle_spread=float(spread[:k].max()))
        assert np.all(dev_ <= bar), (key, dev_, bar)
    assert info["rel_res_true"] <= 1.5e-8
    info2, x2, _ = solve(a, b, tol=0.0, maxit=ref["iters"], variant=variant, precond=precond, loop=loop)
    assert info2["iters"] == ref["iters"]
    d_x = rel(x2, fixed["x"])
    record("bicgstab_parity", case, "x at the oracle's count", d_x, 1e-9, max(1e-9, 10 * x_spread),
           oracle_spread=x_spread)
    assert d_x <= max(1e-9, 10 * x_spread)


def test_bicgstab_jacobi_unit_diagonal_is_plain_and_handle_stays_clean():
    """diag(A) = I: the preconditioned solve is the plain one bitwise; plain solves on the same
    handle before and after a preconditioned one agree bitwise (values restored, separate
    cached graphs)."""
    a = W.convdiff_3d(12)
    u = W.CSR(a.n, a.row_ptr, a.col, a.val / 9.0, "convdiff_unit_diag")
    _, b, _ = W.manufactured(u, seed=1)
    for variant in ("pipelined", "classical"):
        A = pk.CSRMatrix.from_workload(u)
        i1, x1, t1 = solve(u, b, A=A, variant=variant)
        i2, x2, t2 = solve(u, b, A=A, variant=variant, precond="jacobi")
        assert i1["iters"] == i2["iters"] and np.array_equal(x1, x2)
        assert np.array_equal(t1, t2, equal_nan=True)
    s = W.diag_scaled(a, seed=5, spread=100.0)
    _, b, _ = W.manufactured(s, seed=2)
    A = pk.CSRMatrix.from_workload(s)
    i1, x1, _ = solve(s, b, A=A, tol=1e-8, maxit=5000)
    ij, xj, _ = solve(s, b, A=A, tol=1e-8, maxit=5000, precond="jacobi", flags=pk.FLAG_TRUE_RES)
    i3, x3, _ = solve(s, b, A=A, tol=1e-8, maxit=5000)
    assert i1["iters"] == i3["iters"] and np.array_equal(x1, x3)
    assert ij["status"] == pk.PK_OK and ij["rel_res_true"] <= 1.5e-8 and ij["iters"] < i1["iters"]


def test_bicgstab_jacobi_zero_diagonal_rejected():
    a = W.convdiff_3d(8)
    z = W.CSR(a.n, a.row_ptr, a.col, a.val.copy(), "zero_diag")
    rows = np.repeat(np.arange(a.n), np.diff(a.row_ptr))
    z.val[np.nonzero((rows == 100) & (a.col == 100))[0]] = 0.0
    _, b, _ = W.manufactured(a)
    with pytest.raises(RuntimeError, match="nonzero finite diagonal"):
        solve(z, b, precond="jacobi")


def test_bicgstab_launch_counts():
    """Sec. 3.2: four kernels per pipelined iteration; the classical form here takes eleven
    (two SpMV, nine BLAS-1 including the explicit residual norm)."""
    a = W.convdiff_3d(10)
    _, b, _ = W.manufactured(a)
    per = {}
    for variant in ("pipelined", "classical"):
        i5, _, _ = solve(a, b, tol=0.0, maxit=5, variant=variant, loop="host", check_every=1)
        i10, _, _ = solve(a, b, tol=0.0, maxit=10, variant=variant, loop="host", check_every=1)
        per[variant] = (i10["launches"] - i5["launches"]) / 5
    assert per == {"pipelined": 4, "classical": 11}


def test_bicgstab_edge_cases():
    a = W.convdiff_3d(6)
    _, b, _ = W.manufactured(a)
    for variant, loop in (("pipelined", "graph"), ("pipelined", "persistent"), ("classical", "graph")):
        info, x, _ = solve(a, np.zeros(a.n), x0=np.ones(a.n), variant=variant, loop=loop)
        assert info["status"] == pk.PK_OK and info["iters"] == 0 and not x.any()
        info, _, _ = solve(a, b, maxit=0, variant=variant, loop=loop)
        assert info["status"] == pk.PK_NOT_CONVERGED and info["iters"] == 0
        xs = np.linalg.solve(a.to_dense(), b)
        info, _, _ = solve(a, b, x0=xs, variant=variant, loop=loop)
        assert info["status"] == pk.PK_OK and info["iters"] == 0
        # early exit on a small s: b = A e_j for a diagonal-dominant row converges fast
        for loop in ("graph", "host") + (("persistent",) if variant == "pipelined" else ()):
            ref = O.bicgstab(a, b, tol=1e-3, maxit=100, variant=variant)
            info, x, _ = solve(a, b, tol=1e-3, maxit=100, variant=variant, loop=loop)
            assert info["status"] == pk.PK_OK and abs(info["iters"] - ref["iters"]) <= 1
            assert rel(x, ref["x"]) < 1e-6


def test_bicgstab_large_convdiff():
    """3D convection-diffusion 128^3: alpha, omega and beta of the first 20 iterations against
    the oracle (1e-12 where the oracle's own one-ulp spread allows it, else 100 x that spread,
    as in the smaller cases), x after 20 iterations, then a full solve to 1e-8 checked by its
    true residual (its iteration count is compared with the stored oracle solve in
    test_gpu_fullsize.py)."""
    a = W.convdiff_3d(128)
    _, b, _ = W.manufactured(a)
    k = 20
    ref = O.bicgstab(a, b, tol=0.0, maxit=k, variant="pipelined")
    spread = np.zeros(k)
    x_spread = 0.0
    for smp in range(2):
        bp = b * (1 + 2.0 ** -52 * W.uniform_pm1(100 + smp, a.n))
        r = O.bicgstab(a, bp, tol=0.0, maxit=k, variant="pipelined")
        for key in ("alpha", "omega", "beta"):
            spread = np.fmax(spread, np.abs(r[key][:k] - ref[key][:k]) / np.abs(ref[key][:k]))
        x_spread = max(x_spread, rel(r["x"], ref["x"]))
    spread = np.maximum.accumulate(spread)
    A = pk.CSRMatrix.from_workload(a)
    info, xk, tr = solve(a, b, A=A, tol=0.0, maxit=k)
    bar = np.maximum(1e-12, 100 * spread)
    for col, key in ((0, "alpha"), (2, "omega"), (1, "beta")):
        d = np.abs(tr[:k, col] - ref[key][:k]) / np.abs(ref[key][:k])
        record("bicgstab_large_convdiff", "convdiff_128", f"{key} (first {k})", float(d.max()), 1e-12,
               float(bar.max()), oracle_spread=float(spread.max()))
        assert np.all(d <= bar), (key, d, bar)
    np.testing.assert_allclose(tr[:6, 0], ref["alpha"][:6], rtol=1e-12)
    np.testing.assert_allclose(tr[:6, 1], ref["beta"][:6], rtol=1e-12)
    np.testing.assert_allclose(tr[:6, 2], ref["omega"][:6], rtol=1e-12)
    d_x = rel(xk, ref["x"])
    record("bicgstab_large_convdiff", "convdiff_128", f"x after {k}", d_x, 1e-9, max(1e-9, 10 * x_spread),
           oracle_spread=x_spread)
    assert d_x <= max(1e-9, 10 * x_spread)
    info, _, _ = solve(a, b, A=A, tol=1e-8, maxit=10_000, flags=pk.FLAG_TRUE_RES)
    assert info["status"] == pk.PK_OK and info["rel_res_true"] <= 1.5e-8


def test_bicgstab_persistent_loop_selection_and_limits():
    """PK_LOOP_AUTO runs small pipelined solves on one cluster (three launches: setup, x = 0
    test, the loop) with the same iterates as PK_LOOP_PERSISTENT, and the graph above
    PK_PERSISTENT_BICGSTAB_AUTO_N; the persistent loop takes the pipelined form only and n up to
    16 x 4096 rows; a breakdown (<Ap, r0*> = 0 exactly: a skew-symmetric matrix and an
    integer right-hand side) is reported;
    maxit stops it with PK_NOT_CONVERGED after exactly maxit iterations."""
    a = W.convdiff_3d(20)
    _, b, _ = W.manufactured(a, seed=4)
    A = pk.CSRMatrix.from_workload(a)
    ia, xa, ta = solve(a, b, A=A, loop="auto")
    ip, xp, tp = solve(a, b, A=A, loop="persistent")
    assert ia["launches"] == 3 and ia["iters"] == ip["iters"] and np.array_equal(xa, xp)
    assert np.array_equal(ta, tp, equal_nan=True)
    with pytest.raises(RuntimeError, match="PK_LOOP_PERSISTENT"):
        solve(a, b, A=A, loop="persistent", variant="classical")
    big = W.convdiff_3d(41)  # 68,921 rows
    _, bb, _ = W.manufactured(big, seed=1)
    with pytest.raises(RuntimeError, match="PK_LOOP_PERSISTENT"):
        solve(big, bb, loop="persistent")
    mid = W.convdiff_3d(36)  # 46,656 rows: fits one cluster, above the automatic threshold
    _, bm, _ = W.manufactured(mid, seed=1)
    ig, _, _ = solve(mid, bm, loop="auto", tol=0.0, maxit=3)
    ip, _, _ = solve(mid, bm, loop="persistent", tol=0.0, maxit=3)
    assert ig["launches"] > 3 and ip["launches"] == 3
    # skew-symmetric A: <Ap, r0*> = <A r0, r0> = 0 at the first step
    n = 64
    rp = np.arange(0, 2 * n + 1, 2, dtype=np.int32)
    ci = np.empty(2 * n, np.int32)
    va = np.empty(2 * n)
    for i in range(n):
        ci[2 * i], ci[2 * i + 1] = (i - 1) % n, (i + 1) % n
        va[2 * i], va[2 * i + 1] = -1.0, 1.0
    order = np.argsort(ci.reshape(n, 2), axis=1)
    ci = np.take_along_axis(ci.reshape(n, 2), order, 1).ravel()
    va = np.take_along_axis(va.reshape(n, 2), order, 1).ravel()
    sk = W.CSR(n, rp, ci, va, "skew_cycle")
    bs = np.round(3 * W.uniform_pm1(7, n))  # small integers: every product and sum is exact
    ref = O.bicgstab(sk, bs, tol=1e-10, maxit=50, variant="pipelined")
    info, _, _ = solve(sk, bs, tol=1e-10, maxit=50, loop="persistent")
    assert ref["status"] == O.BREAKDOWN and info["status"] == pk.PK_BREAKDOWN
    ref = O.bicgstab(a, b, tol=0.0, maxit=7, variant="pipelined")
    info, x, tr = solve(a, b, A=A, tol=0.0, maxit=7, loop="persistent")
    assert info["status"] == pk.PK_NOT_CONVERGED and info["iters"] == 7
    assert rel(x, ref["x"]) <= 1e-10
    np.testing.assert_allclose(tr[:7, 0], ref["alpha"][:7], rtol=1e-12)
