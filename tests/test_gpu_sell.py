"""GPU checks of the SELL-C-sigma form of the fused SpMV + inner-product kernels (sliced
ELLPACK, the format family of the paper's finite-element runs, Sec. 4.1).

q = A p on the SELL copy must equal the CSR kernel's q bitwise (both sum every row left to
right with FMAs) and the oracle's row sums within rounding; <p, q> within rounding of the
CSR result; pipelined CG with its fused SpMV kernel on the SELL copy meets the CG parity bars
against the oracle."""
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


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def with_empty_rows(a, every=7):
    """a with every `every`-th row emptied (zero-length rows inside slices)."""
    lens = np.diff(a.row_ptr).copy()
    keep = np.ones(a.nnz, dtype=bool)
    rows = np.repeat(np.arange(a.n), lens)
    keep[rows % every == 3] = False
    lens[np.arange(a.n) % every == 3] = 0
    rp = np.zeros(a.n + 1, dtype=np.int32)
    np.cumsum(lens, out=rp[1:])
    return W.CSR(a.n, rp, a.col[keep], a.val[keep], a.name + "_holes")


SPMV_MATRICES = {
    "lap3d_20": lambda: W.laplace_3d(20),
    "lap2d_ragged": lambda: W.laplace_2d(97, 41),          # n = 3977, last slice partial
    "tiny_n5": lambda: W.laplace_2d(5, 1),                 # one partial slice
    "powerlaw_2e4": lambda: W.power_law(20_000, seed=3),   # rows 3..256, sorted windows
    "fe3d_elast_540": lambda: W.fe_elasticity_3d(5),
    "rand28": lambda: W.random_uniform(5000, 28, seed=1),
    "holes": lambda: with_empty_rows(W.convdiff_3d(12)),
}


@pytest.mark.parametrize("name", sorted(SPMV_MATRICES))
def test_sell_spmv_dot_matches_csr_bitwise_and_oracle(name):
    a = SPMV_MATRICES[name]()
    A = pk.CSRMatrix.from_workload(a)
    p = W.uniform_pm1(11, a.n)
    pd = dev(p)
    q1, q2 = torch.empty_like(pd), torch.empty_like(pd)
    r1 = torch.zeros(1, dtype=torch.float64, device=DEV)
    r2 = torch.zeros(1, dtype=torch.float64, device=DEV)
    pk.spmv_dot(A, pd, q1, r1, fused=True)
    pk.spmv_dot(A, pd, q2, r2, sell=True)
    pk.spmv_dot(A, pd, q2, r2, sell=True)      # second call reuses the cached copy
    torch.cuda.synchronize()
    y1, y2 = q1.cpu().numpy(), q2.cpu().numpy()
    assert np.array_equal(y1, y2)
    ref = O.spmv(a, p)
    absrow = np.abs(a.to_dense()) @ np.abs(p) if a.n <= 6000 else None
    if absrow is not None:
        assert np.all(np.abs(y2 - ref) <= 1e-14 * absrow + 1e-300)
    else:
        np.testing.assert_allclose(y2, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    d_ref = float(np.dot(p, ref))
    assert abs(float(r2.item()) - d_ref) <= 1e-12 * max(abs(d_ref), np.abs(p) @ np.abs(ref))


CG_MATRICES = {
    "lap3d_33": lambda: W.laplace_3d(33),
    "lap2d_ragged": lambda: W.laplace_2d(97, 41),
    "fe2d_p1_961": lambda: W.fe_poisson_2d(5),
    "spd_powerlaw": lambda: W.spd_power_law(20_000, seed=3),
}


@pytest.mark.parametrize("loop", ["graph", "host"])
@pytest.mark.parametrize("name", sorted(CG_MATRICES))
def test_cg_on_sell_parity(name, loop):
    a = CG_MATRICES[name]()
    _, b, _ = W.manufactured(a, seed=0)
    ref = O.cg(a, b, tol=1e-8, maxit=5000, variant="pipelined")
    A = pk.CSRMatrix.from_workload(a)
    x = dev(np.zeros(a.n))
    tr = torch.full((64, 4), float("nan"), dtype=torch.float64, device=DEV)
    info = pk.cg_solve(A, dev(b), x, trace=tr, tol=1e-8, maxit=5000, loop=loop,
                       flags=pk.FLAG_SELL | pk.FLAG_TRUE_RES)
    t = tr.cpu().numpy()
    assert info["status"] == pk.PK_OK and abs(info["iters"] - ref["iters"]) <= 2
    k = min(20, ref["iters"] - 1)
    np.testing.assert_allclose(t[:k, 0], ref["alpha"][:k], rtol=1e-12, atol=0)
    np.testing.assert_allclose(t[:k, 1], ref["beta"][:k], rtol=1e-12, atol=0)
    assert info["rel_res_true"] <= 1.5e-8
    # x after exactly the oracle's iteration count against the oracle's x
    fixed = ref["iters"]
    x2 = dev(np.zeros(a.n))
    info2 = pk.cg_solve(A, dev(b), x2, tol=0.0, maxit=fixed, loop=loop, flags=pk.FLAG_SELL)
    assert info2["iters"] == fixed
    xo = O.cg(a, b, tol=0.0, maxit=fixed, variant="pipelined")["x"]
    d_x = rel(x2.cpu().numpy(), xo)
    spread = 0.0
    if d_x > 1e-9:  # the oracle's own one-ulp spread (3.5e-9 on the irregular P1 mesh)
        for smp in range(3):
            bp = b * (1 + 2.0 ** -52 * W.uniform_pm1(100 + smp, a.n))
            spread = max(spread, rel(O.cg(a, bp, tol=0.0, maxit=fixed, variant="pipelined")["x"], xo))
    record("cg_sell", f"{name} {loop}", "x at the oracle's count", d_x, 1e-9, max(1e-9, 10 * spread),
           oracle_spread=spread)
    assert d_x <= max(1e-9, 10 * spread)


def test_sell_flag_is_rejected_elsewhere():
    a = W.laplace_2d(32)
    _, b, _ = W.manufactured(a)
    A = pk.CSRMatrix.from_workload(a)
    bd, x = dev(b), dev(np.zeros(a.n))
    for kw in (dict(variant="classical"), dict(precision="mixed"), dict(precond="jacobi"),
               dict(loop="persistent")):
        with pytest.raises(RuntimeError, match="PK_FLAG_SELL"):
            pk.cg_solve(A, bd, x, flags=pk.FLAG_SELL, **kw)
    for fn in (pk.bicgstab_solve, pk.gmres_solve):
        with pytest.raises(RuntimeError, match="PK_FLAG_SELL"):
            fn(A, bd, x, flags=pk.FLAG_SELL)
