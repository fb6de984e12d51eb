"""GPU parity of CG (pipelined Alg. 2, split, classical Alg. 1) against the CPU oracle.

Bars: per-iteration alpha_i, beta_i within 1e-12 relative over the first 20 iterations;
iteration count to tol within +-2; x within 1e-9 relative of the oracle's x after the same
number of iterations; the true residual at exit within the tolerance.
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


def solve(a, b, x0=None, A=None, trace_cap=64, **kw):
    A = A or pk.CSRMatrix.from_workload(a)
    x = dev(np.zeros(a.n) if x0 is None else x0)
    tr = torch.full((trace_cap, 4), float("nan"), dtype=torch.float64, device=DEV)
    info = pk.cg_solve(A, dev(b), x, trace=tr, **kw)
    torch.cuda.synchronize()
    return info, x.cpu().numpy(), tr.cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


MATRICES = {
    "dense_rows_1e4": lambda: W.spd_dense_rows(),            # rows of 9,000 nonzeros: chunk tiles
    "dense_rows_62500": lambda: W.spd_dense_rows(k=250, dense=(0, 5, 31000, 62499), per_row=20000),
    "fe2d_p1_961": lambda: W.fe_poisson_2d(5),              # P1 triangles, ~7 per row
    "fe3d_elast_4752": lambda: W.fe_elasticity_3d(11),      # P1 elasticity, 3x3 blocks, <= 45 per row
    "lap2d_64": lambda: W.laplace_2d(64),                   # the 64 x 64 configuration
    "lap2d_ragged": lambda: W.laplace_2d(97, 41),           # several blocks, ragged tail
    "lap3d_16": lambda: W.laplace_3d(16),
    "lap3d_33": lambda: W.laplace_3d(33),
    "spd_rand": lambda: W.spd_random(300, seed=5, density=0.05),
    "shifted_rect": lambda: W.laplace_2d(130, 77, shift=0.3),
}


FORMS = [("pipelined", "graph"), ("pipelined", "persistent"), ("split", "graph"),
         ("classical", "graph")]


@pytest.mark.parametrize("variant,loop", FORMS)
@pytest.mark.parametrize("name", sorted(MATRICES))
def test_cg_parity(name, variant, loop):
    a = MATRICES[name]()
    _, b, _ = W.manufactured(a, seed=0)
    ovar = "classical" if variant == "classical" else "pipelined"
    ref = O.cg(a, b, tol=1e-8, maxit=5000, variant=ovar)
    info, x, tr = solve(a, b, tol=1e-8, maxit=5000, variant=variant, loop=loop,
                        flags=pk.FLAG_TRUE_RES)
    assert info["status"] == pk.PK_OK
    assert abs(info["iters"] - ref["iters"]) <= 2
    k = min(20, ref["iters"] - 1)
    np.testing.assert_allclose(tr[:k, 0], ref["alpha"][:k], rtol=1e-12, atol=0)
    np.testing.assert_allclose(tr[:k, 1], ref["beta"][:k], rtol=1e-12, atol=0)
    assert info["rel_res_true"] <= 1.5e-8
    # same iteration count: x within max(1e-9, 10 x the oracle's own one-ulp spread)
    fixed = ref["iters"]
    info2, x2, _ = solve(a, b, tol=0.0, maxit=fixed, variant=variant, loop=loop)
    assert info2["status"] == pk.PK_NOT_CONVERGED and info2["iters"] == fixed
    d_x = rel(x2, ref["x"])
    spread = oracle_x_spread(a, b, ovar, fixed, ref["x"])
    record("cg_parity", f"{name} {variant} {loop}", "x at the oracle's count", d_x, 1e-9, max(1e-9, 10 * spread),
           oracle_spread=spread)
    assert d_x <= max(1e-9, 10 * spread)


def oracle_x_spread(a, b, variant, iters, x_ref, nsamp=3):
    """How far the oracle's own x after `iters` iterations moves when b is perturbed by about
    one ulp (relative 2^-52, three seeds): 6e-16 on the Laplacians, 3.5e-9 on the irregular
    P1 triangulation with 961 unknowns after 104 iterations."""
    sp = 0.0
    for smp in range(nsamp):
        bp = b * (1 + 2.0 ** -52 * W.uniform_pm1(100 + smp, a.n))
        sp = max(sp, rel(O.cg(a, bp, tol=0.0, maxit=iters, variant=variant)["x"], x_ref))
    return sp


@pytest.mark.parametrize("loop", ["graph", "host"])
def test_cg_loop_modes_agree_bitwise(loop):
    a = W.laplace_2d(64)
    _, b, _ = W.manufactured(a)
    i1, x1, _ = solve(a, b, loop="graph")
    i2, x2, _ = solve(a, b, loop=loop, check_every=5)
    assert i1["iters"] == i2["iters"]
    assert np.array_equal(x1, x2)  # deterministic reductions: bitwise reproducible


def test_cg_persistent_is_repeatable_and_matches_graph():
    """One cooperative launch runs the whole solve: bitwise repeatable (fixed reduction order),
    same iterations as the graph loop, x equal up to the reduction order of the partial sums."""
    for a in (W.laplace_2d(64), W.laplace_3d(40)):
        _, b, _ = W.manufactured(a)
        i1, x1, t1 = solve(a, b, loop="persistent")
        i2, x2, t2 = solve(a, b, loop="persistent")
        i3, x3, t3 = solve(a, b, loop="graph")
        assert i1["status"] == i3["status"] == pk.PK_OK
        assert i1["iters"] == i2["iters"] == i3["iters"]
        assert np.array_equal(x1, x2) and np.array_equal(t1, t2, equal_nan=True)
        assert rel(x1, x3) <= 1e-12
        assert i1["launches"] == 3  # setup, zero-x guard, the persistent loop


def test_cg_persistent_largest_cluster_parity():
    """n = 32,768 fills a cluster's shared memory (2,048 or 4,096 rows per CTA, several rows
    per thread)."""
    a = W.laplace_3d(32)
    _, b, _ = W.manufactured(a, seed=2)
    ref = O.cg(a, b, tol=1e-8, maxit=5000, variant="pipelined")
    info, x, tr = solve(a, b, tol=1e-8, maxit=5000, loop="persistent", flags=pk.FLAG_TRUE_RES)
    assert info["status"] == pk.PK_OK and abs(info["iters"] - ref["iters"]) <= 2
    np.testing.assert_allclose(tr[:20, 0], ref["alpha"][:20], rtol=1e-12, atol=0)
    np.testing.assert_allclose(tr[:20, 1], ref["beta"][:20], rtol=1e-12, atol=0)
    assert info["rel_res_true"] <= 1.5e-8
    assert rel(x, ref["x"]) <= 1e-9


def test_cg_persistent_too_large_falls_back_under_auto():
    a = W.laplace_3d(64)  # 262,144 rows: more than one cluster's shared memory holds
    _, b, _ = W.manufactured(a)
    with pytest.raises(RuntimeError, match="persistent loop needs"):
        solve(a, b, loop="persistent")
    i_auto, x_auto, _ = solve(a, b, loop="auto")
    i_graph, x_graph, _ = solve(a, b, loop="graph")
    assert i_auto["iters"] == i_graph["iters"] and np.array_equal(x_auto, x_graph)


def test_cg_persistent_rejects_other_forms():
    """The persistent loop runs pipelined CG, BiCGStab and GMRES with one Gram-Schmidt pass
    (tested with those solvers)."""
    a = W.laplace_2d(16)
    _, b, _ = W.manufactured(a)
    A = pk.CSRMatrix.from_workload(a)
    for call, kw in ((pk.cg_solve, dict(variant="classical")), (pk.cg_solve, dict(precision="mixed")),
                     (pk.bicgstab_solve, dict(variant="classical")), (pk.gmres_solve, dict(flags=pk.FLAG_CGS2))):
        with pytest.raises(RuntimeError, match="PERSISTENT"):
            call(A, dev(b), dev(np.zeros(a.n)), loop="persistent", **kw)


def test_cg_launch_counts_match_the_paper():
    """Sec. 3.1: pipelined CG needs two kernels per iteration, classical six; split three."""
    a = W.laplace_2d(40)
    _, b, _ = W.manufactured(a)
    per_iter = {}
    for variant in ("pipelined", "split", "classical"):
        i10, _, _ = solve(a, b, tol=0.0, maxit=10, variant=variant, loop="host", check_every=1)
        i20, _, _ = solve(a, b, tol=0.0, maxit=20, variant=variant, loop="host", check_every=1)
        per_iter[variant] = (i20["launches"] - i10["launches"]) / 10
    assert per_iter == {"pipelined": 2, "split": 3, "classical": 6}


def test_cg_timing_mode_reports_kernels():
    a = W.laplace_2d(64)
    _, b, _ = W.manufactured(a)
    info, _, _ = solve(a, b, tol=0.0, maxit=30, flags=pk.FLAG_TIMING)
    assert info["kernel_count"]["spmv_dots"] == 31 and info["kernel_count"]["update"] == 30
    assert all(v > 0 for v in info["kernel_ms"].values())


@pytest.mark.parametrize("loop", ["graph", "persistent"])
def test_cg_edge_cases(loop):
    a = W.laplace_2d(8)
    _, b, _ = W.manufactured(a)

    def solve(*args, **kw):
        return globals()["solve"](*args, loop=loop, **kw)

    # b = 0 -> x = 0, no iterations
    info, x, _ = solve(a, np.zeros(a.n), x0=np.ones(a.n))
    assert info["status"] == pk.PK_OK and info["iters"] == 0 and not x.any()
    # exact initial guess -> 0 iterations
    xs = np.linalg.solve(a.to_dense(), b)
    info, x, _ = solve(a, b, x0=xs)
    assert info["status"] == pk.PK_OK and info["iters"] == 0
    # maxit = 0
    info, _, _ = solve(a, b, maxit=0)
    assert info["status"] == pk.PK_NOT_CONVERGED and info["iters"] == 0
    # not SPD
    neg = W.CSR(a.n, a.row_ptr, a.col, -a.val)
    info, _, _ = solve(neg, b)
    assert info["status"] == pk.PK_NOT_SPD
    # NaN in b
    nb = b.copy()
    nb[5] = np.nan
    info, _, _ = solve(a, nb)
    assert info["status"] == pk.PK_ERR_NAN
    # a 1 x 1 system and a 3 x 3 system (single partial block)
    one = W.CSR(1, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([4.0]))
    info, x, _ = solve(one, np.array([2.0]))
    assert info["status"] == pk.PK_OK and abs(x[0] - 0.5) < 1e-15 and info["iters"] == 1


def test_cg_host_pointers_match_device():
    a = W.laplace_3d(12)
    _, b, _ = W.manufactured(a)
    A = pk.CSRMatrix.from_workload(a)
    _, xd, _ = solve(a, b, A=A)
    xh = np.zeros(a.n)
    info = pk.cg_solve(A, np.ascontiguousarray(b), xh)
    assert info["status"] == pk.PK_OK
    assert np.array_equal(xh, xd)


def test_spmv_and_fused_dot_parity():
    for a in (W.power_law(20_000, seed=3), W.laplace_3d(20), W.random_uniform(5000, 28, seed=1)):
        A = pk.CSRMatrix.from_workload(a)
        xv = W.uniform_pm1(7, a.n)
        y = torch.zeros(a.n, dtype=torch.float64, device=DEV)
        pk.spmv(A, dev(xv), y)
        ref = O.spmv(a, xv)
        absrow = W.CSR(a.n, a.row_ptr, a.col, np.abs(a.val)).matvec(np.abs(xv))
        assert np.all(np.abs(y.cpu().numpy() - ref) <= 1e-14 * absrow + 1e-300)
        q1 = torch.zeros_like(y)
        q2 = torch.zeros_like(y)
        r1 = torch.zeros(1, dtype=torch.float64, device=DEV)
        r2 = torch.zeros(1, dtype=torch.float64, device=DEV)
        pk.spmv_dot(A, dev(xv), q1, r1, fused=True)
        pk.spmv_dot(A, dev(xv), q2, r2, fused=False)
        torch.cuda.synchronize()
        assert torch.equal(q1, q2) and torch.equal(q1, y)
        d_ref = O.dot(xv, ref)
        assert abs(r1.item() - d_ref) <= 1e-12 * np.dot(np.abs(xv), absrow)
        assert r1.item() == r2.item()  # same fixed reduction order in both forms


@pytest.mark.parametrize("k", [100, 160])
def test_cg_full_size_3d(k):
    """The large 3D sizes: first 20 alpha/beta against the oracle (20 oracle iterations),
    x after 20 iterations, and the full solve's true residual."""
    a = W.laplace_3d(k)
    _, b, _ = W.manufactured(a)
    ref = O.cg(a, b, tol=0.0, maxit=20, variant="pipelined")
    A = pk.CSRMatrix.from_workload(a)
    info, x20, tr = solve(a, b, A=A, tol=0.0, maxit=20)
    np.testing.assert_allclose(tr[:20, 0], ref["alpha"][:20], rtol=1e-12, atol=0)
    np.testing.assert_allclose(tr[:20, 1], ref["beta"][:20], rtol=1e-12, atol=0)
    assert rel(x20, ref["x"]) <= 1e-9
    info, x, _ = solve(a, b, A=A, tol=1e-8, maxit=50_000, flags=pk.FLAG_TRUE_RES)
    assert info["status"] == pk.PK_OK and info["rel_res_true"] <= 1.5e-8


@pytest.mark.parametrize("name", ["lap2d_64", "lap3d_33", "spd_rand", "lap2d_ragged"])
def test_cg_tile_engine_matches_row_kernels(name):
    """The warp-specialised bulk-copy kernels and the thread-per-row kernels agree to the
    parity bars (their reductions differ only in block partitioning)."""
    a = MATRICES[name]()
    _, b, _ = W.manufactured(a, seed=1)
    A = pk.CSRMatrix.from_workload(a)
    assert A.stats()["kernel"] == 2
    i1, x1, t1 = solve(a, b, A=A)
    i2, x2, t2 = solve(a, b, A=A, flags=pk.FLAG_NO_TMA)
    assert abs(i1["iters"] - i2["iters"]) <= 2
    k = min(20, i1["iters"] - 1)
    np.testing.assert_allclose(t1[:k, :2], t2[:k, :2], rtol=1e-12)
    assert rel(x1, x2) < 1e-7


def test_cg_unaligned_and_odd_length_x():
    """x that is not 16-byte aligned, and odd n, go through a padded library copy."""
    a = W.laplace_2d(33, 31)  # n = 1023, odd
    _, b, _ = W.manufactured(a)
    A = pk.CSRMatrix.from_workload(a)
    _, x_ref, _ = solve(a, b, A=A)
    buf = torch.zeros(a.n + 1, dtype=torch.float64, device=DEV)
    xv = buf[1:]  # 8-byte offset
    info = pk.cg_solve(A, dev(b), xv)
    torch.cuda.synchronize()
    assert info["status"] == pk.PK_OK
    assert np.array_equal(xv.cpu().numpy(), x_ref) and buf[0].item() == 0.0


def test_rows_longer_than_a_tile_use_chunk_tiles():
    """Rows of 20,000 nonzeros are cut into chunk tiles summed by a whole block: the tile
    engine stays in use (no thread-per-row fallback), and A p equals the oracle's row sums."""
    a = W.spd_dense_rows(k=250, dense=(0, 5, 31000, 62499), per_row=20000)
    A = pk.CSRMatrix.from_workload(a)
    st = A.stats()
    assert st["kernel"] == 2 and st["tiles_long"] >= 4 * 5
    lens = np.diff(a.row_ptr)
    edges = [0, 8, 16, 32, 64, 256, 4096, np.inf]
    assert st["row_hist"] == [int(((lens > lo) & (lens <= hi)).sum()) if lo else int((lens <= hi).sum())
                              for lo, hi in zip(edges[:-1], edges[1:])]
    assert st["row_hist"][6] == 4
    p = W.uniform_pm1(5, a.n)
    _, b, _ = W.manufactured(a, seed=1)
    # one K-CG-S through a fixed single CG iteration: alpha_0 = <r0,r0> / <r0, A r0>
    tr = torch.full((4, 4), float("nan"), dtype=torch.float64, device=DEV)
    x = dev(np.zeros(a.n))
    pk.cg_solve(A, dev(b), x, trace=tr, tol=0.0, maxit=1)
    ref = O.cg(a, b, tol=0.0, maxit=1, variant="pipelined")
    np.testing.assert_allclose(tr.cpu().numpy()[0, :2], [ref["alpha"][0], ref["beta"][0]], rtol=1e-12)
    assert rel(x.cpu().numpy(), ref["x"]) <= 1e-13
    del p


@pytest.mark.parametrize("solver", ["cg", "cg_jacobi", "cg_mixed", "bicgstab", "gmres"])
def test_bounded_waits_time_out_and_the_context_stays_usable(solver):
    """Failure detection without a GPU fault: with PK_FLAG_TEST_STALL the CSR tile engine's
    producer issues no copies, so every consumer's first wait (a barrier phase that nothing
    completes) runs out after the 1 ms bound; the kernel records it and returns, the solve
    ends with PK_TIMEOUT, and the next solve on the same handle, with the default bound and
    no flag, is exact."""
    a = W.laplace_3d(48)  # 110,592 rows: the graph loop with the tile engines
    _, b, _ = W.manufactured(a, seed=3)
    A = pk.CSRMatrix.from_workload(a)
    fn = pk.gmres_solve if solver == "gmres" else pk.bicgstab_solve if solver == "bicgstab" else pk.cg_solve
    kw = {"cg_jacobi": {"precond": "jacobi"}, "cg_mixed": {"precision": "mixed"}}.get(solver, {})
    x = dev(np.zeros(a.n))
    with pytest.raises(pk.PkError) as err:
        fn(A, dev(b), x, tol=1e-8, maxit=40, wait_ns=1_000_000, flags=pk.FLAG_TEST_STALL, **kw)
    assert err.value.status == pk.PK_TIMEOUT
    torch.cuda.synchronize()
    info = fn(A, dev(b), x.zero_(), tol=1e-8, maxit=5000, flags=pk.FLAG_TRUE_RES, **kw)
    assert info["status"] == pk.PK_OK and info["rel_res_true"] <= 1.5e-8
    with pytest.raises(RuntimeError, match="wait_ns"):
        fn(A, dev(b), x, wait_ns=-1)


@pytest.mark.parametrize("solver", ["bicgstab", "gmres", "cg_jacobi", "cg_mixed", "bicgstab_jacobi"])
def test_nan_in_b_is_reported(solver):
    """A NaN in b reaches <b, b> in the setup kernel's last block: PK_ERR_NAN, no iteration."""
    a = W.convdiff_3d(10) if solver.startswith(("bicgstab", "gmres")) else W.laplace_3d(10)
    _, b, _ = W.manufactured(a)
    b[17] = np.nan
    A = pk.CSRMatrix.from_workload(a)
    fn = pk.gmres_solve if solver == "gmres" else pk.bicgstab_solve if solver.startswith("bicgstab") else pk.cg_solve
    kw = {"cg_jacobi": {"precond": "jacobi"}, "bicgstab_jacobi": {"precond": "jacobi"},
          "cg_mixed": {"precision": "mixed"}}.get(solver, {})
    info = fn(A, dev(b), dev(np.zeros(a.n)), tol=1e-8, maxit=100, **kw)
    assert info["status"] == pk.PK_ERR_NAN and info["iters"] == 0


RESIDENT_MATRICES = {
    "lap3d_64": lambda: W.laplace_3d(64),                     # 262,144 rows, thread-per-row tiles
    "lap2d_513x400": lambda: W.laplace_2d(513, 400),          # 205,200 rows, ragged blocks, odd n
    "fe3d_elast_47": lambda: W.fe_elasticity_3d(47),          # 324,864 rows, G-lane tiles
    "spd_powerlaw_2e5": lambda: W.spd_power_law(200_000, seed=3),  # whole-warp rows, wide columns
    "dense_rows_3e5": lambda: W.spd_dense_rows(k=550, dense=(0, 7, 150_000, 302_499), per_row=20000),
}


@pytest.mark.parametrize("name", sorted(RESIDENT_MATRICES))
def test_cg_resident_parity(name):
    """The grid-resident loop (one cooperative launch, one block per SM): alpha/beta at 1e-12
    for 20 iterations, iterations +-2, x after the oracle's count at 1e-9 (or 10 x the
    oracle's own one-ulp spread), true residual; bitwise repeatable."""
    a = RESIDENT_MATRICES[name]()
    _, b, _ = W.manufactured(a, seed=0)
    ref = O.cg(a, b, tol=1e-8, maxit=20_000, variant="pipelined")
    A = pk.CSRMatrix.from_workload(a)
    info, x, tr = solve(a, b, A=A, tol=1e-8, maxit=20_000, loop="resident", flags=pk.FLAG_TRUE_RES)
    assert info["status"] == pk.PK_OK, info
    assert abs(info["iters"] - ref["iters"]) <= 2, (info["iters"], ref["iters"])
    assert info["launches"] <= 4  # setup, zero-x guard, the resident loop (+ true residual)
    k = min(20, ref["iters"] - 1)
    np.testing.assert_allclose(tr[:k, 0], ref["alpha"][:k], rtol=1e-12, atol=0)
    np.testing.assert_allclose(tr[:k, 1], ref["beta"][:k], rtol=1e-12, atol=0)
    np.testing.assert_allclose(tr[:k, 3], ref["res2"][:k], rtol=1e-11, atol=0)
    assert info["rel_res_true"] <= 1.5e-8
    fixed = ref["iters"]
    info2, x2, _ = solve(a, b, A=A, tol=0.0, maxit=fixed, loop="resident")
    assert info2["status"] == pk.PK_NOT_CONVERGED and info2["iters"] == fixed
    d_x = rel(x2, ref["x"])
    spread = oracle_x_spread(a, b, "pipelined", fixed, ref["x"]) if d_x > 1e-9 else 0.0
    record("cg_resident", name, "x at the oracle's count", d_x, 1e-9, max(1e-9, 10 * spread), oracle_spread=spread)
    assert d_x <= max(1e-9, 10 * spread)
    info3, x3, tr3 = solve(a, b, A=A, tol=1e-8, maxit=20_000, loop="resident")
    assert info3["iters"] == info["iters"] and np.array_equal(x3, x)
    assert np.array_equal(tr3, tr, equal_nan=True)


def test_cg_resident_edge_cases_and_rejections():
    a = W.laplace_3d(64)
    _, b, _ = W.manufactured(a, seed=1)
    A = pk.CSRMatrix.from_workload(a)
    # b = 0, exact x0, maxit = 0, maxit = 1, not SPD, NaN
    info, x, _ = solve(a, np.zeros(a.n), A=A, x0=np.ones(a.n), loop="resident")
    assert info["status"] == pk.PK_OK and info["iters"] == 0 and not x.any()
    info, _, _ = solve(a, b, A=A, maxit=0, loop="resident")
    assert info["status"] == pk.PK_NOT_CONVERGED and info["iters"] == 0
    ref = O.cg(a, b, tol=0.0, maxit=1, variant="pipelined")
    info, x, _ = solve(a, b, A=A, tol=0.0, maxit=1, loop="resident")
    assert info["status"] == pk.PK_NOT_CONVERGED and info["iters"] == 1 and rel(x, ref["x"]) <= 1e-13
    neg = W.CSR(a.n, a.row_ptr, a.col, -a.val)
    info, _, _ = solve(neg, b, loop="resident")
    assert info["status"] == pk.PK_NOT_SPD
    nb = b.copy()
    nb[77] = np.nan
    info, _, _ = solve(a, nb, A=A, loop="resident")
    assert info["status"] == pk.PK_ERR_NAN
    # the same handle afterwards: exact
    info, x, _ = solve(a, b, A=A, tol=1e-8, maxit=5000, loop="resident", flags=pk.FLAG_TRUE_RES)
    assert info["status"] == pk.PK_OK and info["rel_res_true"] <= 1.5e-8
    # too small for one block per SM taking two tile blocks; other forms rejected
    small = W.laplace_3d(20)
    _, sb, _ = W.manufactured(small)
    with pytest.raises(RuntimeError, match="resident loop needs"):
        solve(small, sb, loop="resident")
    for kw in (dict(variant="classical"), dict(flags=pk.FLAG_SELL), dict(flags=pk.FLAG_NO_TMA)):
        with pytest.raises(RuntimeError, match="PK_LOOP_RESIDENT"):
            solve(a, b, A=A, loop="resident", **kw)
    for call, kw in ((pk.cg_solve, dict(precision="mixed")), (pk.cg_solve, dict(precond="jacobi")),
                     (pk.bicgstab_solve, {}), (pk.gmres_solve, {})):
        with pytest.raises(RuntimeError, match="RESIDENT|graph or host loop"):
            call(A, dev(b), dev(np.zeros(a.n)), loop="resident", **kw)


def test_cg_resident_bounded_wait_times_out_and_context_stays_usable():
    """With PK_FLAG_TEST_STALL the CSR producer issues no copies: every consumer's first wait
    runs out after 1 ms, the blocks record PK_TIMEOUT and leave the loop, the launch ends, and
    the next solve on the handle is exact."""
    a = W.laplace_3d(64)
    _, b, _ = W.manufactured(a, seed=3)
    A = pk.CSRMatrix.from_workload(a)
    with pytest.raises(pk.PkError) as err:
        solve(a, b, A=A, tol=1e-8, maxit=40, loop="resident", wait_ns=1_000_000, flags=pk.FLAG_TEST_STALL)
    assert err.value.status == pk.PK_TIMEOUT
    info, _, _ = solve(a, b, A=A, tol=1e-8, maxit=5000, loop="resident", flags=pk.FLAG_TRUE_RES)
    assert info["status"] == pk.PK_OK and info["rel_res_true"] <= 1.5e-8
