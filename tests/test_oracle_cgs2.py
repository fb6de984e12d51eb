"""Pins for the oracle's GMRES with classical Gram-Schmidt applied twice per step (CGS2).

In exact arithmetic CGS2 is GMRES: x_k minimises ||b - A x|| over x0 + K_k(A, r0) (brute
force by QR + least squares), R and xi equal the one-pass values (checked on a
well-conditioned matrix, where rounding keeps them close), and a restarted solve reaches the
dense LU solution.  In floating point the second pass keeps the basis orthonormal, so the
in-cycle estimate rho0 sqrt(1 - sum xi^2) of the pipelined form keeps matching the true
residual after a full cycle on badly scaled matrices, where one pass loses it."""
import numpy as np
import pytest

import oracle as O
from paper_1410_4054_gb300 import workloads as W


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("variant", ["classical", "pipelined"])
@pytest.mark.parametrize("k", [1, 4, 9])
def test_cgs2_minimises_over_the_krylov_space(variant, k):
    a = W.convdiff_3d(5)
    _, b, _ = W.manufactured(a, seed=3)
    x0 = W.uniform_pm1(4, a.n)
    A = a.to_dense()
    r0 = b - A @ x0
    K = [r0]
    for _ in range(k - 1):
        K.append(A @ K[-1])
    Q, _ = np.linalg.qr(np.stack(K, axis=1))
    c, *_ = np.linalg.lstsq(A @ Q, r0, rcond=None)
    best = np.linalg.norm(r0 - A @ Q @ c)
    got = O.gmres(a, b, x0=x0, tol=0.0, maxit=k, m=30, variant=variant, cgs2=True)
    assert got["iters"] == k
    assert abs(np.linalg.norm(b - A @ got["x"]) - best) <= 1e-10 * np.linalg.norm(r0)
    np.testing.assert_allclose(got["x"], x0 + Q @ c, rtol=1e-8, atol=1e-10)


@pytest.mark.parametrize("variant", ["classical", "pipelined"])
def test_cgs2_equals_one_pass_on_a_well_conditioned_matrix(variant):
    a = W.convdiff_3d(8)
    _, b, _ = W.manufactured(a, seed=1)
    one = O.gmres(a, b, tol=0.0, maxit=12, m=30, variant=variant)
    two = O.gmres(a, b, tol=0.0, maxit=12, m=30, variant=variant, cgs2=True)
    scale = np.abs(one["R"]).max()
    np.testing.assert_allclose(two["R"], one["R"], rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(two["xi"], one["xi"], rtol=0, atol=1e-12)
    assert rel(two["x"], one["x"]) < 1e-11


@pytest.mark.parametrize("variant", ["classical", "pipelined"])
def test_cgs2_restarted_matches_dense_lu(variant):
    a = W.power_law(400, seed=2, lmax=40, mean=8)
    _, b, _ = W.manufactured(a, seed=6)
    ref = np.linalg.solve(a.to_dense(), b)
    r = O.gmres(a, b, tol=1e-11, maxit=5000, m=10, variant=variant, cgs2=True)
    assert r["status"] == O.OK
    assert rel(r["x"], ref) < 1e-8


@pytest.mark.parametrize("make", [lambda: W.diag_scaled(W.laplace_2d(20), seed=3, spread=1e3),
                                  lambda: W.diag_scaled(W.fe_elasticity_3d(3), seed=6, spread=1e3)])
def test_cgs2_keeps_the_pipelined_estimate_exact(make):
    """After a full cycle of 30 steps the pipelined estimate matches ||b - A x|| to 1e-9
    with two passes; with one pass it drifts by 1e-8 .. 6e-7 on these matrices."""
    a = make()
    _, b, _ = W.manufactured(a, seed=1)
    dev = {}
    for c2 in (False, True):
        r = O.gmres(a, b, tol=0.0, maxit=30, m=30, variant="pipelined", cgs2=c2)
        true = np.linalg.norm(b - a.matvec(r["x"]))
        dev[c2] = abs(r["est"][29] - true) / true
    assert dev[True] <= 1e-9
    assert dev[False] >= 100 * dev[True]


@pytest.mark.parametrize("variant", ["classical", "pipelined"])
@pytest.mark.parametrize("make", [lambda: W.diag_scaled(W.fe_elasticity_3d(3), seed=6, spread=1e6),
                                  lambda: W.convdiff_3d(6)])
def test_cgs2_arnoldi_relation_and_orthonormal_basis(variant, make):
    """The first cycle's basis and R satisfy A v_{i-1} = sum_{j<=i} R_{j,i} v_j (j >= 1) to
    rounding, and v_1 .. v_k are orthonormal to rounding, even where one pass of
    Gram-Schmidt is far from orthogonal."""
    a = make()
    _, b, _ = W.manufactured(a, seed=1)
    r = O.gmres(a, b, tol=0.0, maxit=30, m=30, variant=variant, cgs2=True)
    V, R = r["V"], r["R"]
    k = int(np.count_nonzero(np.diag(R)))           # first cycle's length
    assert k >= 15
    A = a.to_dense()
    AV = A @ V[:k].T                               # columns A v_0 .. A v_{k-1}
    WR = V[1:k + 1].T @ np.triu(R[:k, :k])         # sum_j R_{j,i} v_j
    scale = np.abs(A).sum(axis=1).max()
    assert np.abs(AV - WR).max() <= 1e-13 * scale
    G = V[1:k + 1] @ V[1:k + 1].T
    assert np.abs(G - np.eye(k)).max() <= 1e-14 * k
