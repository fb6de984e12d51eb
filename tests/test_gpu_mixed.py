"""Mixed precision (FP32 pipelined CG inside FP64 iterative refinement) for one system:
the FP64 true residual reaches the tolerance, and the solution's error against the FP64
oracle's is within the conditioning of the system."""
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


@pytest.mark.parametrize("make", [lambda: W.laplace_2d(64), lambda: W.laplace_3d(32),
                                  lambda: W.laplace_2d(130, 77, shift=0.3),
                                  lambda: W.spd_random(500, seed=2, density=0.02),
                                  lambda: W.spd_dense_rows(),   # rows longer than a tile
                                  lambda: W.fe_elasticity_3d(8)])  # grouped-lane tiles (FP32 path)
@pytest.mark.parametrize("loop", ["graph", "host"])
def test_mixed_reaches_fp64_tolerance(make, loop):
    a = make()
    _, b, _ = W.manufactured(a, seed=0)
    A = pk.CSRMatrix.from_workload(a)
    x = torch.zeros(a.n, dtype=torch.float64, device=DEV)
    info = pk.cg_solve(A, dev(b), x, tol=1e-10, maxit=50_000, precision="mixed", loop=loop,
                       flags=pk.FLAG_TRUE_RES)
    torch.cuda.synchronize()
    assert info["status"] == pk.PK_OK, info
    xh = x.cpu().numpy()
    assert np.linalg.norm(b - a.matvec(xh)) <= 1.5e-10 * np.linalg.norm(b)
    assert info["rel_res_true"] <= 1.5e-10
    ref = O.cg(a, b, tol=1e-12, maxit=50_000, variant="pipelined")
    assert rel(xh, ref["x"]) <= 1e-8
    assert 1 <= info["cycles"] <= 20


def test_mixed_graph_and_host_loops_agree_bitwise():
    a = W.laplace_3d(20)
    _, b, _ = W.manufactured(a)
    A = pk.CSRMatrix.from_workload(a)
    xs = []
    for loop in ("graph", "host"):
        x = torch.zeros(a.n, dtype=torch.float64, device=DEV)
        pk.cg_solve(A, dev(b), x, tol=1e-10, maxit=50_000, precision="mixed", loop=loop, check_every=3)
        xs.append(x.cpu().numpy())
    assert np.array_equal(xs[0], xs[1])


def test_mixed_large_3d_against_fp64_solve():
    a = W.laplace_3d(160)
    _, b, _ = W.manufactured(a)
    A = pk.CSRMatrix.from_workload(a)
    bd = dev(b)
    x64 = torch.zeros(a.n, dtype=torch.float64, device=DEV)
    i64 = pk.cg_solve(A, bd, x64, tol=1e-10, maxit=50_000)
    xm = torch.zeros(a.n, dtype=torch.float64, device=DEV)
    im = pk.cg_solve(A, bd, xm, tol=1e-10, maxit=50_000, precision="mixed", flags=pk.FLAG_TRUE_RES)
    torch.cuda.synchronize()
    assert i64["status"] == pk.PK_OK and im["status"] == pk.PK_OK
    assert im["rel_res_true"] <= 1.5e-10
    assert rel(xm.cpu().numpy(), x64.cpu().numpy()) <= 1e-7
