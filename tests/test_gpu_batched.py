"""Batched persistent solves (one launch for many uneven SPD systems) against the oracle:
each system matches its own single-system oracle solve."""
import numpy as np
import pytest

import oracle as O
from paper_1410_4054_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1410_4054_gb300 import pk  # noqa: E402

DEV = "cuda:0"


def dev(v):
    return torch.from_numpy(np.ascontiguousarray(v, dtype=np.float64)).to(DEV)


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def make_batch(nsys=40, seed=0, lo=8, hi=64):
    mats = W.batched_rectangles(nsys, seed=seed, lo=lo, hi=hi)
    # edge members: a 1 x 1 system and a zero right-hand side
    mats.append(W.CSR(1, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([3.0])))
    mats.append(W.laplace_2d(5, 7, shift=0.5))
    rhs = []
    for k, a in enumerate(mats):
        _, b, _ = W.manufactured(a, seed=k)
        rhs.append(b)
    rhs[-1] = np.zeros(mats[-1].n)
    return mats, rhs


@pytest.mark.parametrize("autotune", [False, True])
def test_batched_fp64_matches_single_system_oracle(autotune):
    mats, rhs = make_batch()
    As = [pk.CSRMatrix.from_workload(a) for a in mats]
    bs = [dev(b) for b in rhs]
    # fixed iteration count: x after 25 iterations equals the oracle's
    xs = [torch.zeros(a.n, dtype=torch.float64, device=DEV) for a in mats]
    infos = pk.batched_solve(As, bs, xs, tol=0.0, maxit=25,
                             flags=pk.FLAG_AUTOTUNE if autotune else 0)
    torch.cuda.synchronize()
    for a, b, x, inf in zip(mats, rhs, xs, infos):
        ref = O.cg(a, b, tol=0.0, maxit=25, variant="pipelined")
        if ref["status"] == O.NOT_CONVERGED:  # (the 1 x 1 member can reach r = 0 exactly)
            assert inf["iters"] == ref["iters"], (a.name, inf, ref["iters"])
        assert rel(x.cpu().numpy(), ref["x"]) <= 1e-9, a.name
    if autotune:
        blk, per = pk.batched_last_config()
        assert (blk, per) == (288, 2) or (blk in (128, 256, 512, 1024) and per in (1, 2, 4, 8))
    # the tile engine (lanes = -1) on the same batch: the same oracle bars
    xs = [torch.zeros(a.n, dtype=torch.float64, device=DEV) for a in mats]
    infos = pk.batched_solve(As, bs, xs, tol=0.0, maxit=25, lanes=-1)
    torch.cuda.synchronize()
    assert pk.batched_last_lanes() == -1 and pk.batched_last_config() == (288, 2)
    for a, b, x, inf in zip(mats, rhs, xs, infos):
        ref = O.cg(a, b, tol=0.0, maxit=25, variant="pipelined")
        if ref["status"] == O.NOT_CONVERGED:
            assert inf["iters"] == ref["iters"], (a.name, inf, ref["iters"])
        assert rel(x.cpu().numpy(), ref["x"]) <= 1e-9, a.name
    # to tolerance: iterations within 2 of the oracle, true residual within tol
    xs = [torch.zeros(a.n, dtype=torch.float64, device=DEV) for a in mats]
    infos = pk.batched_solve(As, bs, xs, tol=1e-10, maxit=5000)
    torch.cuda.synchronize()
    for a, b, x, inf in zip(mats, rhs, xs, infos):
        ref = O.cg(a, b, tol=1e-10, maxit=5000, variant="pipelined")
        assert inf["status"] == pk.PK_OK
        assert abs(inf["iters"] - ref["iters"]) <= 2, (a.name, inf["iters"], ref["iters"])
        xh = x.cpu().numpy()
        if np.any(b):
            assert np.linalg.norm(b - a.matvec(xh)) <= 1.5e-10 * np.linalg.norm(b)
        else:
            assert not xh.any()


def test_batched_mixed_precision_reaches_fp64_accuracy():
    mats, rhs = make_batch(nsys=24, seed=3)
    As = [pk.CSRMatrix.from_workload(a) for a in mats]
    bs = [dev(b) for b in rhs]
    xs = [torch.zeros(a.n, dtype=torch.float64, device=DEV) for a in mats]
    infos = pk.batched_solve(As, bs, xs, tol=1e-10, maxit=20_000, precision="mixed")
    torch.cuda.synchronize()
    for a, b, x, inf in zip(mats, rhs, xs, infos):
        assert inf["status"] == pk.PK_OK, (a.name, inf)
        xh = x.cpu().numpy()
        if not np.any(b):
            assert not xh.any()
            continue
        assert np.linalg.norm(b - a.matvec(xh)) <= 1.5e-10 * np.linalg.norm(b)
        ref = O.cg(a, b, tol=1e-12, maxit=20_000, variant="pipelined")
        assert rel(xh, ref["x"]) <= 1e-8  # error vs the FP64 oracle's solution
        assert inf["cycles"] >= 1


def test_batched_not_spd_member_is_reported():
    mats, rhs = make_batch(nsys=6, seed=5)
    neg = W.CSR(mats[0].n, mats[0].row_ptr, mats[0].col, -mats[0].val)
    mats[0] = neg
    As = [pk.CSRMatrix.from_workload(a) for a in mats]
    bs = [dev(b) for b in rhs]
    xs = [torch.zeros(a.n, dtype=torch.float64, device=DEV) for a in mats]
    infos = pk.batched_solve(As, bs, xs, tol=1e-10, maxit=2000)
    assert infos[0]["status"] == pk.PK_NOT_SPD
    assert all(i["status"] == pk.PK_OK for i in infos[1:])


def test_batched_rejects_a_preconditioner():
    mats, rhs = make_batch(nsys=2, seed=1)
    As = [pk.CSRMatrix.from_workload(a) for a in mats]
    bs = [dev(b) for b in rhs]
    xs = [torch.zeros(a.n, dtype=torch.float64, device=DEV) for a in mats]
    with pytest.raises(RuntimeError, match="no preconditioner"):
        pk.batched_solve(As, bs, xs, tol=1e-10, maxit=2000, precond="jacobi")


def make_fe_batch(nsys=24, seed=0):
    """Uneven batch of P1 elasticity systems (3 x 3 blocks, up to 45 nonzeros per row)."""
    ks = 2 + (W.splitmix64(seed, nsys) % np.uint64(4)).astype(int)   # k = 2..5: 54 .. 540 rows
    mats = [W.fe_elasticity_3d(int(k), seed=i) for i, k in enumerate(ks)]
    rhs = [W.manufactured(a, seed=i)[1] for i, a in enumerate(mats)]
    return mats, rhs


def oracle_x_spread(a, b, iters, x_ref, nsamp=3):
    """The oracle's own one-ulp spread of x after `iters` pipelined-CG iterations: up to 1e-7 on
    the 54-unknown members, which reach the rounding floor before 20 iterations."""
    sp = 0.0
    for smp in range(nsamp):
        bp = b * (1 + 2.0 ** -52 * W.uniform_pm1(100 + smp, a.n))
        sp = max(sp, rel(O.cg(a, bp, tol=0.0, maxit=iters, variant="pipelined")["x"], x_ref))
    return sp


@pytest.mark.parametrize("lanes", [1, 2, 4, 8])
def test_batched_lanes_per_row_match_the_oracle(lanes):
    """Rows computed by 1, 2, 4 or 8 lanes: x after a fixed count matches each system's oracle
    solve within max(1e-9, 10 x the oracle's own one-ulp spread); to tolerance, every system
    converges with the oracle's iteration count (+-2)."""
    mats, rhs = make_fe_batch()
    As = [pk.CSRMatrix.from_workload(a) for a in mats]
    bs = [dev(b) for b in rhs]
    xs = [torch.zeros(a.n, dtype=torch.float64, device=DEV) for a in mats]
    pk.batched_solve(As, bs, xs, tol=0.0, maxit=20, lanes=lanes)
    torch.cuda.synchronize()
    assert pk.batched_last_lanes() == lanes
    for a, b, x in zip(mats, rhs, xs):
        ref = O.cg(a, b, tol=0.0, maxit=20, variant="pipelined")
        bar = max(1e-9, 10 * oracle_x_spread(a, b, 20, ref["x"]))
        assert rel(x.cpu().numpy(), ref["x"]) <= bar, a.name
    xs = [torch.zeros(a.n, dtype=torch.float64, device=DEV) for a in mats]
    infos = pk.batched_solve(As, bs, xs, tol=1e-10, maxit=5000, lanes=lanes)
    torch.cuda.synchronize()
    for a, b, x, inf in zip(mats, rhs, xs, infos):
        ref = O.cg(a, b, tol=1e-10, maxit=5000, variant="pipelined")
        assert inf["status"] == pk.PK_OK and abs(inf["iters"] - ref["iters"]) <= 2
        assert np.linalg.norm(b - a.matvec(x.cpu().numpy())) <= 1.5e-10 * np.linalg.norm(b)


def test_batched_autotuner_covers_lanes_per_row():
    mats, rhs = make_fe_batch(nsys=32, seed=4)
    As = [pk.CSRMatrix.from_workload(a) for a in mats]
    bs = [dev(b) for b in rhs]
    xs = [torch.zeros(a.n, dtype=torch.float64, device=DEV) for a in mats]
    for prec in ("fp64", "mixed"):
        infos = pk.batched_solve(As, bs, [x.zero_() for x in xs], tol=1e-10, maxit=5000, precision=prec,
                                 flags=pk.FLAG_AUTOTUNE)
        torch.cuda.synchronize()
        assert all(i["status"] == pk.PK_OK for i in infos)
        assert pk.batched_last_lanes() in ((-2, -1, 1, 2, 4, 8) if prec == "fp64" else (1, 2, 4, 8))  # -1 tiles, -2 clusters
        for a, b, x in zip(mats, rhs, xs):
            assert np.linalg.norm(b - a.matvec(x.cpu().numpy())) <= 1.5e-10 * np.linalg.norm(b)
    with pytest.raises(RuntimeError, match="lanes per row"):
        pk.batched_solve(As, bs, xs, tol=1e-10, maxit=10, lanes=3)
    with pytest.raises(RuntimeError, match="tile engine"):
        pk.batched_solve(As, bs, xs, tol=1e-10, maxit=10, lanes=-1, precision="mixed")


@pytest.mark.parametrize("precision,lanes", [("fp64", 0), ("fp64", -2), ("mixed", 0)])
def test_batched_config_512_rectangles(precision, lanes):
    """The benchmark's batch itself: 512 shifted 2D Laplacians on rectangles with sides drawn
    log-uniform from 32 to 256 (up to 65,536 rows each), one launch to 1e-10 (FP64: the row
    engine and the cluster engine).  Every system's true residual meets the tolerance; a
    sample of 16 systems (the largest, the smallest and 14 seeded picks) is checked against its
    own oracle solve: FP64 iterations within +-2 and x after 30 fixed iterations within 1e-9;
    mixed precision: the error against the FP64 oracle's solution."""
    mats = W.batched_rectangles(512, seed=0)
    rhs = [W.manufactured(a, seed=k)[1] for k, a in enumerate(mats)]
    As = [pk.CSRMatrix.from_workload(a) for a in mats]
    bs = [dev(b) for b in rhs]
    xs = [torch.zeros(a.n, dtype=torch.float64, device=DEV) for a in mats]
    ns = np.array([a.n for a in mats])
    pick = sorted({int(ns.argmax()), int(ns.argmin())}
                  | set(np.random.default_rng(5).choice(len(mats), 14, replace=False).tolist()))
    infos = pk.batched_solve(As, bs, xs, tol=1e-10, maxit=20_000, precision=precision, lanes=lanes)
    torch.cuda.synchronize()
    if lanes:
        assert pk.batched_last_lanes() == lanes
    for a, b, x, inf in zip(mats, rhs, xs, infos):
        assert inf["status"] == pk.PK_OK, (a.name, inf)
        assert np.linalg.norm(b - a.matvec(x.cpu().numpy())) <= 1.5e-10 * np.linalg.norm(b), a.name
    for k in pick:
        ref = O.cg(mats[k], rhs[k], tol=1e-10, maxit=20_000, variant="pipelined")
        if precision == "fp64":
            assert abs(infos[k]["iters"] - ref["iters"]) <= 2, (k, infos[k]["iters"], ref["iters"])
        else:
            assert rel(xs[k].cpu().numpy(), ref["x"]) <= 1e-8, k
    if precision == "fp64":
        pk.batched_solve(As, bs, [x.zero_() for x in xs], tol=0.0, maxit=30, lanes=lanes)
        torch.cuda.synchronize()
        for k in pick:
            ref = O.cg(mats[k], rhs[k], tol=0.0, maxit=30, variant="pipelined")
            assert rel(xs[k].cpu().numpy(), ref["x"]) <= 1e-9, k
    for A in As:
        A.close()


def test_batched_tile_engine_irregular_rows_and_unaligned_x():
    """The tile engine on P1 elasticity systems (G-lane tiles) and power-law SPD systems
    (whole-warp rows), with every other x 8 bytes off a 16-byte boundary (its update then
    runs without bulk copies of x): x after 20 fixed iterations matches each system's oracle
    solve within max(1e-9, 10 x the oracle's one-ulp spread), and to tolerance every system
    converges with the oracle's iteration count (+-2)."""
    mats, rhs = make_fe_batch(nsys=12, seed=2)
    mats += [W.spd_power_law(3000 + 1000 * k, seed=k) for k in range(4)]
    rhs += [W.manufactured(a, seed=40 + k)[1] for k, a in enumerate(mats[12:])]
    As = [pk.CSRMatrix.from_workload(a) for a in mats]
    bs = [dev(b) for b in rhs]
    bufs = [torch.zeros(a.n + 1, dtype=torch.float64, device=DEV) for a in mats]
    xs = [buf[k % 2:k % 2 + a.n] for k, (buf, a) in enumerate(zip(bufs, mats))]
    pk.batched_solve(As, bs, xs, tol=0.0, maxit=20, lanes=-1)
    torch.cuda.synchronize()
    assert pk.batched_last_lanes() == -1
    for a, b, x in zip(mats, rhs, xs):
        ref = O.cg(a, b, tol=0.0, maxit=20, variant="pipelined")
        bar = max(1e-9, 10 * oracle_x_spread(a, b, 20, ref["x"]))
        assert rel(x.cpu().numpy(), ref["x"]) <= bar, a.name
    for x in xs:
        x.zero_()
    infos = pk.batched_solve(As, bs, xs, tol=1e-10, maxit=5000, lanes=-1)
    torch.cuda.synchronize()
    for a, b, x, inf in zip(mats, rhs, xs, infos):
        ref = O.cg(a, b, tol=1e-10, maxit=5000, variant="pipelined")
        assert inf["status"] == pk.PK_OK and abs(inf["iters"] - ref["iters"]) <= 2, (a.name, inf["iters"], ref["iters"])
        assert np.linalg.norm(b - a.matvec(x.cpu().numpy())) <= 1.5e-10 * np.linalg.norm(b)
    for buf, k in zip(bufs, range(len(bufs))):
        assert buf[0 if k % 2 else -1].item() == 0.0  # nothing written outside x


def test_batched_tile_engine_bounded_wait_times_out():
    """PK_FLAG_TEST_STALL: the CSR producer issues no copies, every system's first wait runs
    out after 1 ms, the systems report PK_TIMEOUT, and the next batch on the same handles is
    exact."""
    mats, rhs = make_batch(nsys=6, seed=7)
    As = [pk.CSRMatrix.from_workload(a) for a in mats]
    bs = [dev(b) for b in rhs]
    xs = [torch.zeros(a.n, dtype=torch.float64, device=DEV) for a in mats]
    with pytest.raises(pk.PkError) as err:
        pk.batched_solve(As, bs, xs, tol=1e-10, maxit=100, wait_ns=1_000_000, flags=pk.FLAG_TEST_STALL, lanes=-1)
    assert err.value.status == pk.PK_TIMEOUT
    torch.cuda.synchronize()
    infos = pk.batched_solve(As, bs, [x.zero_() for x in xs], tol=1e-10, maxit=5000, lanes=-1)
    for a, b, x, inf in zip(mats, rhs, xs, infos):
        assert inf["status"] == pk.PK_OK
        if np.any(b):
            assert np.linalg.norm(b - a.matvec(x.cpu().numpy())) <= 1.5e-10 * np.linalg.norm(b)


def make_cluster_batch():
    """Members for every cluster size of the cluster engine (1 to 16 CTAs of up to 4096 rows):
    the small batch (with its 1 x 1 and zero right-hand-side members), P1 elasticity systems
    (rows of up to 45 nonzeros), power-law SPD systems and shifted Laplacians of 5,000 to
    65,536 rows (up to 4,096 rows on each of 16 CTAs)."""
    mats, rhs = make_batch(nsys=10, seed=11)
    fe, fe_rhs = make_fe_batch(nsys=4, seed=6)
    mats += fe
    rhs += fe_rhs
    extra = [W.spd_power_law(5000, seed=3), W.spd_power_law(9000, seed=4),
             W.laplace_2d(130, 130, shift=0.05), W.laplace_2d(181, 181, shift=0.02),
             W.laplace_2d(256, 256, shift=0.01)]
    mats += extra
    rhs += [W.manufactured(a, seed=60 + k)[1] for k, a in enumerate(extra)]
    return mats, rhs


def test_batched_cluster_engine_matches_the_oracle():
    """The cluster engine (lanes = -2): x after 25 fixed iterations matches each system's
    oracle solve within max(1e-9, 10 x the oracle's one-ulp spread); to tolerance every system
    converges with the oracle's iteration count (+-2) and meets the tolerance in its true
    residual; the zero right-hand side gives x = 0."""
    mats, rhs = make_cluster_batch()
    As = [pk.CSRMatrix.from_workload(a) for a in mats]
    bs = [dev(b) for b in rhs]
    xs = [torch.zeros(a.n, dtype=torch.float64, device=DEV) for a in mats]
    infos = pk.batched_solve(As, bs, xs, tol=0.0, maxit=25, lanes=-2)
    torch.cuda.synchronize()
    assert pk.batched_last_lanes() == -2 and pk.batched_last_config() == (256, 2)
    for a, b, x, inf in zip(mats, rhs, xs, infos):
        ref = O.cg(a, b, tol=0.0, maxit=25, variant="pipelined")
        if ref["status"] == O.NOT_CONVERGED:
            assert inf["iters"] == ref["iters"], (a.name, inf, ref["iters"])
        bar = max(1e-9, 10 * oracle_x_spread(a, b, 25, ref["x"])) if np.any(b) else 0.0
        assert rel(x.cpu().numpy(), ref["x"]) <= bar, a.name
    xs = [torch.zeros(a.n, dtype=torch.float64, device=DEV) for a in mats]
    infos = pk.batched_solve(As, bs, xs, tol=1e-10, maxit=5000, lanes=-2)
    torch.cuda.synchronize()
    for a, b, x, inf in zip(mats, rhs, xs, infos):
        ref = O.cg(a, b, tol=1e-10, maxit=5000, variant="pipelined")
        assert inf["status"] == pk.PK_OK, (a.name, inf)
        assert abs(inf["iters"] - ref["iters"]) <= 2, (a.name, inf["iters"], ref["iters"])
        xh = x.cpu().numpy()
        if np.any(b):
            assert np.linalg.norm(b - a.matvec(xh)) <= 1.5e-10 * np.linalg.norm(b)
        else:
            assert not xh.any()
    for A in As:
        A.close()


def test_batched_cluster_engine_reports_members_and_rejects():
    """A negated (negative definite) member reports PK_NOT_SPD while the others converge;
    mixed precision and a system of more than 65,536 rows are rejected; maxit = 0 leaves x."""
    mats, rhs = make_batch(nsys=6, seed=5)
    mats[0] = W.CSR(mats[0].n, mats[0].row_ptr, mats[0].col, -mats[0].val)
    As = [pk.CSRMatrix.from_workload(a) for a in mats]
    bs = [dev(b) for b in rhs]
    xs = [torch.zeros(a.n, dtype=torch.float64, device=DEV) for a in mats]
    infos = pk.batched_solve(As, bs, xs, tol=1e-10, maxit=2000, lanes=-2)
    assert infos[0]["status"] == pk.PK_NOT_SPD
    assert all(i["status"] == pk.PK_OK for i in infos[1:])
    with pytest.raises(RuntimeError, match="cluster engine"):
        pk.batched_solve(As, bs, xs, tol=1e-10, maxit=10, lanes=-2, precision="mixed")
    big = W.laplace_2d(257, 256, shift=0.1)
    Ab = pk.CSRMatrix.from_workload(big)
    bb = dev(W.manufactured(big, seed=1)[1])
    xb = torch.zeros(big.n, dtype=torch.float64, device=DEV)
    with pytest.raises(RuntimeError, match="65536 rows"):
        pk.batched_solve([Ab], [bb], [xb], tol=1e-10, maxit=10, lanes=-2)
    # maxit = 0: x stays as given, except x = 0 for the zero right-hand side (the last member)
    x0 = [torch.full((a.n,), 0.5, dtype=torch.float64, device=DEV) for a in mats[1:]]
    infos = pk.batched_solve(As[1:], bs[1:], x0, tol=1e-10, maxit=0, lanes=-2)
    assert all(bool((x == 0.5).all()) for x in x0[:-1]) and not x0[-1].any()
    assert infos[-1]["status"] == pk.PK_OK and all(i["status"] == pk.PK_NOT_CONVERGED for i in infos[:-1])
