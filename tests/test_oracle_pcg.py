"""Pins for the oracle's Jacobi-preconditioned CG (CPU only).

Preconditioned CG with M = diag(A) is CG on the symmetrically scaled system
D^-1/2 A D^-1/2 y = D^-1/2 b, x = D^-1/2 y (same alpha_i, beta_i in exact arithmetic), so the
oracle's already pinned CG fixes every scalar of both PCG forms; plus the special cases a
diagonal matrix (one iteration, exact) and a unit diagonal (PCG is CG)."""
import numpy as np
import pytest

import oracle as O
from paper_1410_4054_gb300 import workloads as W


def scaled(a, d):
    """The CSR matrix diag(d) A diag(d)."""
    rows = np.repeat(np.arange(a.n), np.diff(a.row_ptr))
    return W.CSR(a.n, a.row_ptr.copy(), a.col.copy(), a.val * d[rows] * d[a.col], a.name + "_scaled")


def badly_scaled(k=10, seed=3):
    a = W.laplace_3d(k)
    d = np.exp(np.random.default_rng(seed).uniform(0, np.log(30.0), a.n))
    return scaled(a, d)


def diag_of(a):
    rows = np.repeat(np.arange(a.n), np.diff(a.row_ptr))
    d = np.zeros(a.n)
    np.add.at(d, rows[a.col == rows], a.val[a.col == rows])
    return d


@pytest.mark.parametrize("variant", ["classical", "pipelined"])
def test_pcg_equals_cg_on_the_scaled_system(variant):
    a = badly_scaled()
    _, b, _ = W.manufactured(a, seed=1)
    s = 1.0 / np.sqrt(diag_of(a))
    ah = scaled(a, s)                      # D^-1/2 A D^-1/2 (unit diagonal)
    ref = O.cg(ah, b * s, tol=0.0, maxit=20, variant=variant)
    got = O.pcg_jacobi(a, b, tol=0.0, maxit=20, variant=variant)
    assert got["iters"] == ref["iters"] == 20
    k = 19 if variant == "classical" else 20  # classical records beta after the update
    np.testing.assert_allclose(got["alpha"][:20], ref["alpha"][:20], rtol=1e-10)
    np.testing.assert_allclose(got["beta"][:k], ref["beta"][:k], rtol=1e-9, atol=1e-14)
    np.testing.assert_allclose(got["x"], ref["x"] * s, rtol=1e-9, atol=1e-12)


def test_diagonal_matrix_converges_in_one_iteration():
    n = 50
    d = 1.0 + np.random.default_rng(4).random(n)
    a = W.CSR(n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), d, "diag")
    b = np.random.default_rng(5).standard_normal(n)
    for variant in ("classical", "pipelined"):
        got = O.pcg_jacobi(a, b, tol=1e-14, maxit=10, variant=variant)
        assert got["status"] == 0 and got["iters"] == 1
        np.testing.assert_allclose(got["x"], b / d, rtol=1e-15)


@pytest.mark.parametrize("variant", ["classical", "pipelined"])
def test_unit_diagonal_reduces_to_cg(variant):
    a = W.laplace_2d(20)
    a = W.CSR(a.n, a.row_ptr, a.col, a.val / 4.0, "lap_unit_diag")
    _, b, _ = W.manufactured(a, seed=2)
    ref = O.cg(a, b, tol=1e-10, maxit=500, variant=variant)
    got = O.pcg_jacobi(a, b, tol=1e-10, maxit=500, variant=variant)
    assert got["iters"] == ref["iters"]
    np.testing.assert_allclose(got["alpha"][: ref["iters"]], ref["alpha"][: ref["iters"]], rtol=1e-14)
    np.testing.assert_allclose(got["x"], ref["x"], rtol=1e-13, atol=1e-15)


def test_pipelined_and_classical_pcg_agree_and_jacobi_pays():
    a = badly_scaled(k=14, seed=7)
    x_star, b, _ = W.manufactured(a, seed=3)
    cls = O.pcg_jacobi(a, b, tol=1e-10, maxit=2000, variant="classical")
    pip = O.pcg_jacobi(a, b, tol=1e-10, maxit=2000, variant="pipelined")
    plain = O.cg(a, b, tol=1e-10, maxit=5000, variant="pipelined")
    assert cls["status"] == pip["status"] == 0
    assert abs(cls["iters"] - pip["iters"]) <= 1
    np.testing.assert_allclose(pip["alpha"][:20], cls["alpha"][:20], rtol=1e-10)
    assert pip["iters"] < 0.6 * plain["iters"]          # the diagonal scaling is what Jacobi undoes
    res = np.linalg.norm(b - a.matvec(pip["x"])) / np.linalg.norm(b)
    assert res <= 1e-10
    assert np.linalg.norm(pip["x"] - x_star) / np.linalg.norm(x_star) <= 1e-6


def test_nonpositive_diagonal_is_not_spd():
    a = W.laplace_2d(6)
    neg = W.CSR(a.n, a.row_ptr, a.col, -a.val, "neg")
    _, b, _ = W.manufactured(a, seed=0)
    assert O.pcg_jacobi(neg, b)["status"] == 6
