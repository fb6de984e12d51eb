"""GPU parity of Jacobi-preconditioned pipelined CG against the CPU oracle.

The GPU form is the pipelined structure of Alg. 2 with M = diag(A) fused into its two kernels
(Sec. 5 names preconditioner fusion as the extension of the method).  Bars as for CG:
alpha_i, beta_i within 1e-12 relative over the first 20 iterations; iterations within +-2;
x within 1e-9 of the oracle's x after the same number of iterations; the true residual at
exit within the tolerance.
"""
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


def solve(a, b, x0=None, A=None, trace_cap=64, precond="jacobi", **kw):
    A = A or pk.CSRMatrix.from_workload(a)
    x = dev(np.zeros(a.n) if x0 is None else x0)
    tr = torch.full((trace_cap, 4), float("nan"), dtype=torch.float64, device=DEV)
    info = pk.cg_solve(A, dev(b), x, trace=tr, precond=precond, **kw)
    torch.cuda.synchronize()
    return info, x.cpu().numpy(), tr.cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


MATRICES = {
    "lap3d_16_scaled": lambda: W.diag_scaled(W.laplace_3d(16), seed=1, spread=30.0),
    "lap3d_33_scaled": lambda: W.diag_scaled(W.laplace_3d(33), seed=2, spread=100.0),
    "lap2d_ragged_scaled": lambda: W.diag_scaled(W.laplace_2d(97, 41), seed=3, spread=10.0),  # odd n
    "spd_rand_scaled": lambda: W.diag_scaled(W.spd_random(300, seed=5, density=0.05), seed=4),
    "spd_powerlaw_scaled": lambda: W.diag_scaled(W.spd_power_law(20_000, seed=3), seed=5),  # rows > 32
    "lap2d_64": lambda: W.laplace_2d(64),  # constant diagonal: Jacobi is a scalar multiple of I
    "fe3d_elast_4752": lambda: W.fe_elasticity_3d(11),       # grouped-lane tiles
    "dense_rows_1e4": lambda: W.spd_dense_rows(),             # rows longer than a tile: chunk tiles
}


@pytest.mark.parametrize("loop", ["graph", "host"])
@pytest.mark.parametrize("name", sorted(MATRICES))
def test_pcg_parity(name, loop):
    a = MATRICES[name]()
    _, b, _ = W.manufactured(a, seed=0)
    ref = O.pcg_jacobi(a, b, tol=1e-8, maxit=5000, variant="pipelined")
    assert ref["status"] == 0
    info, x, tr = solve(a, b, tol=1e-8, maxit=5000, loop=loop, flags=pk.FLAG_TRUE_RES)
    assert info["status"] == pk.PK_OK
    assert abs(info["iters"] - ref["iters"]) <= 2
    k = min(20, ref["iters"] - 1)
    np.testing.assert_allclose(tr[:k, 0], ref["alpha"][:k], rtol=1e-12, atol=0)
    np.testing.assert_allclose(tr[:k, 1], ref["beta"][:k], rtol=1e-12, atol=0)
    np.testing.assert_allclose(tr[:k, 3], ref["res2"][:k], rtol=1e-11, atol=0)
    assert info["rel_res_true"] <= 1.5e-8
    fixed = ref["iters"]
    info2, x2, _ = solve(a, b, tol=0.0, maxit=fixed, loop=loop)
    assert info2["status"] == pk.PK_NOT_CONVERGED and info2["iters"] == fixed
    assert rel(x2, ref["x"]) <= 1e-9


def test_pcg_graph_and_host_loops_agree_bitwise():
    a = W.diag_scaled(W.laplace_3d(24), seed=7)
    _, b, _ = W.manufactured(a)
    i1, x1, t1 = solve(a, b, loop="graph")
    i2, x2, t2 = solve(a, b, loop="host", check_every=3)
    assert i1["iters"] == i2["iters"] and np.array_equal(x1, x2)
    assert np.array_equal(t1, t2, equal_nan=True)


def test_pcg_unit_diagonal_is_cg():
    """diag(A) = I: M^-1 r = r, so PCG takes CG's scalars (up to the order of partial sums)."""
    a = W.laplace_3d(20)
    a = W.CSR(a.n, a.row_ptr, a.col, a.val / 6.0, "lap3d_unit_diag")
    _, b, _ = W.manufactured(a, seed=1)
    i1, x1, t1 = solve(a, b, precond="jacobi")
    i2, x2, t2 = solve(a, b, precond="none", loop="graph")
    assert i1["status"] == i2["status"] == pk.PK_OK and i1["iters"] == i2["iters"]
    k = i1["iters"] - 1
    np.testing.assert_allclose(t1[:min(k, 64), :2], t2[:min(k, 64), :2], rtol=1e-12)
    assert rel(x1, x2) <= 1e-12


def test_pcg_diagonal_matrix_one_iteration():
    n = 5000
    d = 1.0 + W.uniform_pm1(9, n) ** 2 * 1e3
    a = W.CSR(n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), d, "diag")
    b = W.uniform_pm1(10, n)
    info, x, _ = solve(a, b, tol=1e-14, maxit=10)
    assert info["status"] == pk.PK_OK and info["iters"] == 1
    np.testing.assert_allclose(x, b / d, rtol=1e-15)


def test_pcg_pays_on_a_badly_scaled_matrix():
    a = W.diag_scaled(W.laplace_3d(32), seed=11, spread=100.0)
    _, b, _ = W.manufactured(a, seed=2)
    ip, xp, _ = solve(a, b, tol=1e-8, maxit=20000, flags=pk.FLAG_TRUE_RES)
    ic, xc, _ = solve(a, b, tol=1e-8, maxit=20000, precond="none", loop="graph", flags=pk.FLAG_TRUE_RES)
    assert ip["status"] == ic["status"] == pk.PK_OK
    assert ip["iters"] < 0.5 * ic["iters"]
    assert ip["rel_res_true"] <= 1.5e-8 and ic["rel_res_true"] <= 1.5e-8


def test_pcg_nonpositive_diagonal_is_not_spd():
    a = W.laplace_2d(40)
    neg = W.CSR(a.n, a.row_ptr, a.col, a.val.copy(), "one_negative_diag")
    rows = np.repeat(np.arange(a.n), np.diff(a.row_ptr))
    neg.val[np.nonzero((rows == 777) & (a.col == 777))[0]] = -1.0
    _, b, _ = W.manufactured(a, seed=0)
    assert O.pcg_jacobi(neg, b)["status"] == 6
    info, _, _ = solve(neg, b)
    assert info["status"] == pk.PK_NOT_SPD and info["iters"] == 0


def test_pcg_zero_rhs_and_converged_start():
    a = W.diag_scaled(W.laplace_2d(50), seed=1)
    x_star, b, _ = W.manufactured(a, seed=3)
    info, x, _ = solve(a, np.zeros(a.n), x0=np.ones(a.n))
    assert info["status"] == pk.PK_OK and info["iters"] == 0 and not x.any()
    info, x, _ = solve(a, b, x0=x_star, tol=1e-6)
    assert info["status"] == pk.PK_OK and info["iters"] == 0
    assert np.array_equal(x, x_star)


def test_pcg_rejects_other_forms():
    a = W.laplace_2d(32)
    _, b, _ = W.manufactured(a)
    for kw in (dict(variant="classical"), dict(variant="split"), dict(precision="mixed"),
               dict(loop="persistent")):
        with pytest.raises(RuntimeError, match="PK_PRECOND_JACOBI"):
            solve(a, b, **kw)
    with pytest.raises(RuntimeError, match="tile engine"):
        solve(a, b, flags=pk.FLAG_NO_TMA)
