"""Pins for the oracle's right Jacobi preconditioning of BiCGStab and GMRES (CPU only).

The oracle runs the pinned Alg. 3/4/5/6 oracles on A M^-1 y = b with M = diag(A) and returns
x = M^-1 y.  Pinned here against facts that do not go through that construction: van der
Vorst's right-preconditioned BiCGStab written with M^-1 applied to vectors (p^ = M^-1 p,
s^ = M^-1 s; the textbook form, a different formulation), the dense LU solution, GMRES's
minimal-residual property over x0 + M^-1 K_k(A M^-1, r0) by brute force, a diagonal matrix
(one step), a unit diagonal (the unpreconditioned solver, bitwise) and the zero-diagonal
rejection."""
import numpy as np
import pytest

import oracle as O
from paper_1410_4054_gb300 import workloads as W


def diag_of(a):
    rows = np.repeat(np.arange(a.n), np.diff(a.row_ptr))
    d = np.zeros(a.n)
    np.add.at(d, rows[a.col == rows], a.val[a.col == rows])
    return d


def nonsym_scaled(k=6, seed=1, spread=50.0):
    return W.diag_scaled(W.convdiff_3d(k), seed=seed, spread=spread)


def textbook_bicgstab(A, b, dinv, iters):
    """Right-preconditioned BiCGStab (van der Vorst 1992) with M^-1 applied to vectors;
    alpha_i, omega_i and the beta_i that forms p_{i+1}."""
    x = np.zeros_like(b)
    r = b - A @ x
    rs = r.copy()
    p = r.copy()
    rho = rs @ r
    out = {"alpha": [], "omega": [], "beta": []}
    for _ in range(iters):
        ph = dinv * p
        v = A @ ph
        alpha = rho / (rs @ v)
        s = r - alpha * v
        sh = dinv * s
        t = A @ sh
        omega = (t @ s) / (t @ t)
        x = x + alpha * ph + omega * sh
        r = s - omega * t
        rho_new = rs @ r
        beta = (rho_new / rho) * (alpha / omega)
        p = r + beta * (p - omega * v)
        rho = rho_new
        out["alpha"].append(alpha)
        out["omega"].append(omega)
        out["beta"].append(beta)
    return {k: np.array(v) for k, v in out.items()}, x


@pytest.mark.parametrize("variant", ["classical", "pipelined"])
def test_bicgstab_jacobi_equals_textbook_preconditioned_form(variant):
    a = nonsym_scaled()
    _, b, _ = W.manufactured(a, seed=2)
    A = a.to_dense()
    ref, xt = textbook_bicgstab(A, b, 1.0 / diag_of(a), 8)
    got = O.bicgstab(a, b, tol=0.0, maxit=8, variant=variant, precond="jacobi")
    assert got["iters"] == 8
    for key in ("alpha", "omega", "beta"):
        np.testing.assert_allclose(got[key][:8], ref[key], rtol=1e-9, err_msg=key)
    np.testing.assert_allclose(got["x"], xt, rtol=1e-8, atol=1e-12 * np.abs(xt).max())


@pytest.mark.parametrize("variant", ["classical", "pipelined"])
def test_bicgstab_jacobi_solves_and_pays(variant):
    a = nonsym_scaled(k=10, seed=3, spread=100.0)
    x_star, b, _ = W.manufactured(a, seed=4)
    pre = O.bicgstab(a, b, tol=1e-10, maxit=5000, variant=variant, precond="jacobi")
    plain = O.bicgstab(a, b, tol=1e-10, maxit=5000, variant=variant)
    assert pre["status"] == O.OK
    xs = np.linalg.solve(a.to_dense(), b)
    assert np.linalg.norm(pre["x"] - xs) / np.linalg.norm(xs) <= 1e-7
    assert np.linalg.norm(b - a.matvec(pre["x"])) / np.linalg.norm(b) <= 1e-10
    assert pre["iters"] < 0.5 * plain["iters"]


@pytest.mark.parametrize("variant", ["classical", "pipelined"])
@pytest.mark.parametrize("k", [1, 4, 9])
def test_gmres_jacobi_minimises_over_the_preconditioned_space(variant, k):
    """After k Arnoldi steps of the first cycle, x minimises ||b - A x|| over
    x0 + M^-1 K_k(A M^-1, r0) (brute force: QR of the basis, least squares)."""
    a = nonsym_scaled(k=5, seed=5)
    _, b, _ = W.manufactured(a, seed=6)
    x0 = W.uniform_pm1(7, a.n)
    A = a.to_dense()
    dinv = 1.0 / diag_of(a)
    Ah = A * dinv[None, :]
    r0 = b - A @ x0
    K = [r0]
    for _ in range(k - 1):
        K.append(Ah @ K[-1])
    Q, _ = np.linalg.qr(np.stack(K, axis=1))
    Z = dinv[:, None] * Q                       # M^-1 K_k
    c, *_ = np.linalg.lstsq(A @ Z, r0, rcond=None)
    best = np.linalg.norm(r0 - A @ Z @ c)
    got = O.gmres(a, b, x0=x0, tol=0.0, maxit=k, m=30, variant=variant, precond="jacobi")
    res = np.linalg.norm(b - A @ got["x"])
    assert got["iters"] == k
    assert abs(res - best) <= 1e-9 * np.linalg.norm(r0)
    np.testing.assert_allclose(got["x"], x0 + Z @ c, rtol=1e-7, atol=1e-9)


def test_gmres_jacobi_restarted_solves():
    a = nonsym_scaled(k=8, seed=8, spread=100.0)
    _, b, _ = W.manufactured(a, seed=9)
    xs = np.linalg.solve(a.to_dense(), b)
    for variant in ("classical", "pipelined"):
        pre = O.gmres(a, b, tol=1e-10, maxit=5000, m=20, variant=variant, precond="jacobi")
        plain = O.gmres(a, b, tol=1e-10, maxit=5000, m=20, variant=variant)
        assert pre["status"] == O.OK
        assert np.linalg.norm(pre["x"] - xs) / np.linalg.norm(xs) <= 1e-7
        assert pre["iters"] < plain["iters"]


def test_unit_diagonal_is_the_plain_solver_bitwise():
    a = W.convdiff_3d(6)
    a = W.CSR(a.n, a.row_ptr, a.col, a.val / 9.0, "convdiff_unit_diag")
    _, b, _ = W.manufactured(a, seed=1)
    for variant in ("classical", "pipelined"):
        p = O.bicgstab(a, b, tol=1e-10, maxit=500, variant=variant, precond="jacobi")
        q = O.bicgstab(a, b, tol=1e-10, maxit=500, variant=variant)
        assert p["iters"] == q["iters"] and np.array_equal(p["x"], q["x"])
        assert np.array_equal(p["alpha"], q["alpha"], equal_nan=True)
        g = O.gmres(a, b, tol=1e-10, maxit=500, m=10, variant=variant, precond="jacobi")
        h = O.gmres(a, b, tol=1e-10, maxit=500, m=10, variant=variant)
        assert g["iters"] == h["iters"] and np.array_equal(g["x"], h["x"])


def test_diagonal_matrix_one_step():
    n = 40
    d = 1.0 + np.arange(n) * 0.37 * (-1.0) ** np.arange(n)   # mixed signs are allowed
    a = W.CSR(n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), d, "diag")
    b = W.uniform_pm1(3, n)
    for variant in ("classical", "pipelined"):
        got = O.bicgstab(a, b, tol=1e-14, maxit=10, variant=variant, precond="jacobi")
        assert got["status"] == O.OK and got["iters"] == 1
        np.testing.assert_allclose(got["x"], b / d, rtol=1e-15)
        got = O.gmres(a, b, tol=1e-14, maxit=10, m=5, variant=variant, precond="jacobi")
        assert got["status"] == O.OK and got["iters"] == 1
        np.testing.assert_allclose(got["x"], b / d, rtol=1e-14)


def test_zero_diagonal_is_rejected():
    a = W.convdiff_3d(4)
    z = W.CSR(a.n, a.row_ptr, a.col, a.val.copy(), "zero_diag")
    rows = np.repeat(np.arange(a.n), np.diff(a.row_ptr))
    z.val[np.nonzero((rows == 5) & (a.col == 5))[0]] = 0.0
    _, b, _ = W.manufactured(a)
    with pytest.raises(ValueError, match="nonzero finite diagonal"):
        O.bicgstab(z, b, precond="jacobi")
    with pytest.raises(ValueError, match="nonzero finite diagonal"):
        O.gmres(z, b, precond="jacobi")
