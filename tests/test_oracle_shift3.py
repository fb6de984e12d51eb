"""Pins for the oracle's shift-invariant three-kernel GMRES (Sec. 3.3: the normalisation's
inner product avoided through the shift invariance of the Krylov space).

Shifting the operator does not change the Krylov space, and the oracle maps the shifted
coefficients back to those of A, so in exact arithmetic the method is GMRES: x_k minimises
||b - A x|| over x0 + K_k(A, r0) (brute force by QR + least squares), restarted solves reach
the dense LU solution, and an invariant subspace ends the cycle with the exact solution.  The
shift rule itself (sigma_1 = 0, sigma_{i+1} = <v_{i-1}, A v_{i-1}>) is checked on the first two
shifts, whose basis vectors are known in closed form."""
import numpy as np
import pytest

import oracle as O
from paper_1410_4054_gb300 import workloads as W


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("k", [1, 2, 4, 9])
def test_shift3_minimises_over_the_krylov_space(k):
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
    got = O.gmres(a, b, x0=x0, tol=0.0, maxit=k, m=30, shift3=True)
    assert got["iters"] == k
    assert abs(np.linalg.norm(b - A @ got["x"]) - best) <= 1e-10 * np.linalg.norm(r0)
    np.testing.assert_allclose(got["x"], x0 + Q @ c, rtol=1e-8, atol=1e-10)
    # the basis is shifted from the second step on
    if k >= 2:
        assert got["sigma"][0] == 0.0 and got["sigma"][1] != 0.0


def test_shift3_first_two_shifts_are_rayleigh_quotients():
    """sigma_2 = <v_0, A v_0> with v_0 = r0 / ||r0||; step 1 orthogonalises nothing, so
    v_1 = A v_0 / ||A v_0|| and sigma_3 = <v_1, A v_1>."""
    a = W.convdiff_3d(6)
    _, b, _ = W.manufactured(a, seed=8)
    A = a.to_dense()
    v0 = b / np.linalg.norm(b)
    w = A @ v0
    v1 = w / np.linalg.norm(w)
    got = O.gmres(a, b, tol=0.0, maxit=3, m=30, shift3=True)
    np.testing.assert_allclose(got["sigma"][:3], [0.0, v0 @ A @ v0, v1 @ A @ v1], rtol=1e-12, atol=0)


def test_shift3_gives_the_four_kernel_R_and_xi():
    """On a well-conditioned matrix the unshifted R (R_{i-1,i} = R'_{i-1,i} + sigma_i), xi and
    x agree with Algorithm 6's within rounding of the norm identity."""
    a = W.convdiff_3d(8)
    _, b, _ = W.manufactured(a, seed=1)
    four = O.gmres(a, b, tol=0.0, maxit=12, m=30)
    three = O.gmres(a, b, tol=0.0, maxit=12, m=30, shift3=True)
    scale = np.abs(four["R"]).max()
    np.testing.assert_allclose(three["R"], four["R"], rtol=0, atol=1e-9 * scale)
    np.testing.assert_allclose(three["xi"], four["xi"], rtol=0, atol=1e-9)
    assert rel(three["x"], four["x"]) < 1e-10


@pytest.mark.parametrize("m", [5, 30])
def test_shift3_restarted_matches_dense_lu(m):
    a = W.power_law(400, seed=2, lmax=40, mean=8)
    _, b, _ = W.manufactured(a, seed=6)
    ref = np.linalg.solve(a.to_dense(), b)
    r = O.gmres(a, b, tol=1e-11, maxit=5000, m=m, shift3=True)
    assert r["status"] == O.OK and r["cycles"] >= 2
    assert rel(r["x"], ref) < 1e-8


def test_shift3_invariant_subspace_ends_the_cycle_exactly():
    """b in the span of two eigenvectors of a diagonal matrix: the Krylov space stops growing
    after two steps, R_{3,3}^2 = nu - sum R'^2 falls to rounding, the cycle ends with k = 2
    and x is exact."""
    n = 12
    d = np.arange(1.0, n + 1.0)
    a = W.CSR(n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), d)
    b = np.zeros(n)
    b[2], b[7] = 1.5, -0.5
    r = O.gmres(a, b, tol=1e-14, maxit=50, m=10, shift3=True)
    assert r["status"] == O.OK
    assert r["iters"] == 2
    np.testing.assert_allclose(r["x"], b / d, rtol=1e-13, atol=1e-15)
