"""Pins for the CPU oracle: each check ties it to something other than itself.

- dense LU solves (numpy.linalg.solve) on small systems;
- closed forms: the 2D Dirichlet Laplacian's eigenpairs (CG converges in one step on an
  eigenvector with alpha_0 = 1/lambda, and in exactly d steps on a sum of d eigenvectors);
- optimality characterisations evaluated by brute force on tiny systems: the k-th CG
  iterate minimises the A-norm error over x0 + K_k(A, r0); the k-th GMRES iterate
  minimises the 2-norm residual there; the first BiCGStab iterate is the Galerkin step
  followed by a 1-D residual minimisation;
- invariants of the paper: pipelined and classical CG produce the same alpha_i, beta_i
  up to rounding (Eq. (3)); the BiCGStab residual-norm expansion of Sec. 3.2 equals the
  direct norm; classical and pipelined GMRES give the same R and xi (Sec. 3.3);
- finite termination of CG (n <= 32, well conditioned) and of full GMRES (m >= n).
"""
import numpy as np
import pytest

import oracle as O
from paper_1410_4054_gb300 import workloads as W


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def krylov_basis(a_dense, r0, k):
    """Orthonormal basis of K_k(A, r0) by numpy QR of [r0, A r0, ..., A^{k-1} r0]."""
    cols = [r0 / np.linalg.norm(r0)]
    for _ in range(k - 1):
        w = a_dense @ cols[-1]
        cols.append(w / np.linalg.norm(w))
    q, _ = np.linalg.qr(np.stack(cols, axis=1))
    return q


# ------------------------------------------------------------------------------- CG

@pytest.mark.parametrize("variant", ["classical", "pipelined"])
@pytest.mark.parametrize("make", [lambda: W.laplace_2d(6, 5), lambda: W.spd_random(20, seed=3),
                                  lambda: W.laplace_3d(4)])
def test_cg_matches_dense_lu(variant, make):
    a = make()
    d = a.to_dense()
    xs, b, _ = W.manufactured(a, seed=1)
    ref = np.linalg.solve(d, b)
    r = O.cg(a, b, tol=1e-13, maxit=500, variant=variant)
    assert r["status"] == O.OK
    assert rel(r["x"], ref) < 1e-10
    assert rel(r["x"], xs) < 1e-9


@pytest.mark.parametrize("variant", ["classical", "pipelined"])
def test_cg_finite_termination(variant):
    for seed in range(4):
        a = W.spd_random(24, seed=seed, density=0.4, cond_shift=5.0)
        d = a.to_dense()
        ev = np.linalg.eigvalsh(d)
        assert ev.max() / ev.min() < 100
        _, b, _ = W.manufactured(a, seed=seed)
        r = O.cg(a, b, tol=1e-10, maxit=1000, variant=variant)
        assert r["status"] == O.OK and r["iters"] <= a.n


@pytest.mark.parametrize("variant", ["classical", "pipelined"])
@pytest.mark.parametrize("k", [5, 8])
def test_cg_iterates_minimise_energy_norm(variant, k):
    """x_k = argmin ||x - x*||_A over x0 + K_k(A, r0) (brute force, dense)."""
    a = W.spd_random(18, seed=7, density=0.5, cond_shift=2.0)
    d = a.to_dense()
    xs, b, _ = W.manufactured(a, seed=2)
    x0 = W.uniform_pm1(99, a.n)
    r0 = b - d @ x0
    q = krylov_basis(d, r0, k)
    y = np.linalg.solve(q.T @ d @ q, q.T @ r0)
    xk = x0 + q @ y
    r = O.cg(a, b, x0=x0, tol=0.0, maxit=k, variant=variant)
    assert r["status"] == O.NOT_CONVERGED and r["iters"] == k
    assert rel(r["x"], xk) < 1e-10


def laplace_2d_eig(k, p, q):
    """Eigenvector (p,q) of the k x k Dirichlet 5-point Laplacian and its eigenvalue."""
    t = np.pi / (k + 1)
    xs = np.sin(np.arange(1, k + 1) * p * t)
    ys = np.sin(np.arange(1, k + 1) * q * t)
    u = np.outer(ys, xs).ravel()  # row index = y * k + x
    lam = (2 - 2 * np.cos(p * t)) + (2 - 2 * np.cos(q * t))
    return u, lam


@pytest.mark.parametrize("variant", ["classical", "pipelined"])
def test_cg_eigenvector_one_step(variant):
    k = 64
    a = W.laplace_2d(k)
    u, lam = laplace_2d_eig(k, 3, 5)
    r = O.cg(a, u, tol=1e-10, maxit=50, variant=variant)
    assert r["status"] == O.OK and r["iters"] == 1
    assert abs(r["alpha"][0] * lam - 1) < 1e-13
    assert rel(r["x"], u / lam) < 1e-13
    if variant == "pipelined":
        assert abs(r["beta"][0]) < 1e-12  # r_1 = 0, so beta_0 = <r1,r1>/<r0,r0> = 0


@pytest.mark.parametrize("variant", ["classical", "pipelined"])
def test_cg_sum_of_d_eigenvectors_takes_d_steps(variant):
    k = 32
    a = W.laplace_2d(k)
    # high modes: every factor |1 - lambda/lambda_j| of the residual polynomial stays <= 1
    # on the spectrum, so rounding in b is not amplified
    pairs = [(32, 32), (31, 32), (31, 31), (30, 32), (30, 30)]
    b = sum(laplace_2d_eig(k, p, q)[0] for p, q in pairs)
    r = O.cg(a, b, tol=1e-10, maxit=50, variant=variant)
    assert r["status"] == O.OK and r["iters"] == len(pairs)


def test_cg_pipelined_equals_classical_scalars():
    """Eq. (3): the pipelined beta equals the classical beta, so both alpha/beta traces agree."""
    a = W.laplace_2d(64)
    _, b, _ = W.manufactured(a, seed=0)
    c = O.cg(a, b, tol=1e-8, maxit=1000, variant="classical")
    p = O.cg(a, b, tol=1e-8, maxit=1000, variant="pipelined")
    assert abs(c["iters"] - p["iters"]) <= 1
    for key in ("alpha", "beta"):
        np.testing.assert_allclose(p[key][:20], c[key][:20], rtol=1e-12, atol=0)
    assert rel(p["x"], c["x"]) < 1e-9


def test_cg_not_spd_and_edge_cases():
    a = W.laplace_2d(8)
    neg = W.CSR(a.n, a.row_ptr, a.col, -a.val)
    _, b, _ = W.manufactured(a)
    for v in ("classical", "pipelined"):
        assert O.cg(neg, b, variant=v)["status"] == O.NOT_SPD
        r = O.cg(a, np.zeros(a.n), x0=np.ones(a.n), variant=v)  # b = 0 -> x = 0
        assert r["status"] == O.OK and r["iters"] == 0 and not r["x"].any()
        xs = np.linalg.solve(a.to_dense(), b)
        r = O.cg(a, b, x0=xs, tol=1e-8, variant=v)       # exact start -> 0 iterations
        assert r["status"] == O.OK and r["iters"] == 0
        r = O.cg(a, b, tol=0.0, maxit=7, variant=v)        # fixed iteration count
        assert r["status"] == O.NOT_CONVERGED and r["iters"] == 7
        nan_b = b.copy(); nan_b[3] = np.nan
        assert O.cg(a, nan_b, variant=v)["status"] == O.NAN


def test_cg_table2_bound_classical_vs_pipelined():
    """Table 2 / Sec. 4.3: after 30 iterations the relative difference of the classical and
    pipelined CG residual norms stays below 1e-10 on SPD systems."""
    paper = np.loadtxt("tests/golden/table2_residual_diffs.txt", usecols=(1,), comments="#")
    assert paper.max() < 1e-10
    for a in (W.laplace_2d(64), W.laplace_3d(16), W.laplace_2d(50, 30, shift=0.05)):
        _, b, _ = W.manufactured(a)
        c = O.cg(a, b, tol=0.0, maxit=30, variant="classical")
        p = O.cg(a, b, tol=0.0, maxit=30, variant="pipelined")
        rc = np.linalg.norm(b - O.spmv(a, c["x"]))
        rp = np.linalg.norm(b - O.spmv(a, p["x"]))
        assert abs(rc - rp) / rc < 1e-10


def test_nonsymmetric_table2_bounds_classical_vs_pipelined():
    """Table 2 / Sec. 4.3, nonsymmetric rows: after 30 iterations the relative difference of
    the classical and pipelined residual norms.  The table's GMRES column reaches 5.3e-8
    (rma10), although the text puts CG and GMRES below 1e-10; the pin takes the table's own
    maximum.  BiCGStab differs by up to 0.41 there, and the text bounds it by 1.  On synthetic
    nonsymmetric matrices of the same shapes (upwind convection-diffusion, power-law rows,
    P1 triangles, a badly scaled copy) the oracle's two forms stay within those bounds.  The
    measure compares unconverged residuals: every case is still above 1e-6 relative after 30
    steps (a solve that reaches the rounding floor compares noise)."""
    paper = np.loadtxt("tests/golden/table2_residual_diffs_nonsym.txt", usecols=(1, 2), comments="#")
    assert paper.shape == (7, 2)
    bicg_max, gmres_max = paper[:, 0].max(), paper[:, 1].max()
    assert bicg_max == 0.41 and gmres_max == 5.3e-8
    for a in (W.convdiff_3d(20), W.power_law(5000, seed=3), W.fe_poisson_2d(6),
              W.diag_scaled(W.convdiff_3d(12), seed=1, spread=100.0)):
        _, b, _ = W.manufactured(a, seed=1)

        def res(x):
            return np.linalg.norm(b - O.spmv(a, x))

        g = [res(O.gmres(a, b, tol=0.0, maxit=30, m=30, variant=v)["x"]) for v in ("classical", "pipelined")]
        assert g[0] > 1e-6 * np.linalg.norm(b), a.name
        assert abs(g[0] - g[1]) / g[0] < gmres_max, a.name
        s = [res(O.bicgstab(a, b, tol=0.0, maxit=30, variant=v)["x"]) for v in ("classical", "pipelined")]
        assert s[0] > 1e-6 * np.linalg.norm(b), a.name
        assert np.isfinite(s).all() and abs(s[0] - s[1]) / s[0] < 1.0, a.name


# ------------------------------------------------------------------------------- BiCGStab

NONSYM = [lambda: W.convdiff_3d(4), lambda: W.power_law(60, seed=2, lmax=12, mean=6),
          lambda: W.random_uniform(50, 6, seed=4)]


@pytest.mark.parametrize("variant", ["classical", "pipelined"])
@pytest.mark.parametrize("make", NONSYM)
def test_bicgstab_matches_dense_lu(variant, make):
    a = make()
    xs, b, _ = W.manufactured(a, seed=5)
    ref = np.linalg.solve(a.to_dense(), b)
    r = O.bicgstab(a, b, tol=1e-13, maxit=2000, variant=variant)
    assert r["status"] == O.OK
    assert rel(r["x"], ref) < 1e-9


@pytest.mark.parametrize("variant", ["classical", "pipelined"])
def test_bicgstab_first_iterate_by_characterisation(variant):
    """s_0 = r_0 - alpha A r_0 with <s_0, r0*> = 0 (r0* = r0); omega minimises
    ||s_0 - omega A s_0||_2; x_1 = x_0 + alpha r_0 + omega s_0."""
    a = W.random_uniform(40, 5, seed=9)
    d = a.to_dense()
    _, b, _ = W.manufactured(a, seed=1)
    x0 = W.uniform_pm1(3, a.n)
    r0 = b - d @ x0
    ar0 = d @ r0
    # Galerkin condition <r0 - alpha A r0, r0> = 0, solved as a 1x1 linear system
    alpha = np.linalg.solve(np.array([[ar0 @ r0]]), np.array([r0 @ r0]))[0]
    s0 = r0 - alpha * ar0
    as0 = d @ s0
    omega = np.linalg.lstsq(as0[:, None], s0, rcond=None)[0][0]
    x1 = x0 + alpha * r0 + omega * s0
    r = O.bicgstab(a, b, x0=x0, tol=0.0, maxit=1, variant=variant)
    assert r["iters"] == 1
    assert abs(r["alpha"][0] - alpha) < 1e-12 * abs(alpha)
    assert abs(r["omega"][0] - omega) < 1e-12 * abs(omega)
    assert rel(r["x"], x1) < 1e-12


def _poly_apply(d, coef, v):
    """sum_m coef[m] A^m v."""
    out = np.zeros_like(v)
    w = v.copy()
    for c in coef:
        out += c * w
        w = d @ w
    return out


@pytest.mark.parametrize("variant", ["classical", "pipelined"])
def test_bicgstab_residual_polynomials(variant):
    """Van der Vorst's characterisation, built by brute force from dense linear algebra:
    r_k = Q_k(A) phi_k(A) r_0 where phi_k is the BiCG residual polynomial (phi_k(0) = 1,
    <phi_k(A) r_0, (A^T)^i r0*> = 0 for i < k, r0* = r_0), Q_k(t) = prod_{j<k} (1 - omega_j t)
    and omega_j minimises ||(I - omega A) s_j||_2 with s_j = Q_j(A) phi_{j+1}(A) r_0."""
    a = W.random_uniform(14, 4, seed=21)
    d = a.to_dense() / 8.0
    a = W.CSR(a.n, a.row_ptr, a.col, a.val / 8.0)
    _, b, _ = W.manufactured(a, seed=4)
    x0 = W.uniform_pm1(8, a.n)
    r0 = b - d @ x0
    kmax = 4
    # moments mu_j = <A^j r0, r0*> with r0* = r0
    mu = [r0 @ r0]
    w = r0.copy()
    for _ in range(2 * kmax):
        w = d @ w
        mu.append(w @ r0)

    def phi(k):
        if k == 0:
            return np.array([1.0])
        h = np.array([[mu[m + i] for m in range(1, k + 1)] for i in range(k)])
        c = np.linalg.solve(h, -np.array([mu[i] for i in range(k)]))
        return np.concatenate([[1.0], c])

    q = np.array([1.0])  # coefficients of Q_j
    omegas = []
    for j in range(kmax):
        s_j = _poly_apply(d, q, _poly_apply(d, phi(j + 1), r0))
        as_j = d @ s_j
        om = np.linalg.lstsq(as_j[:, None], s_j, rcond=None)[0][0]
        omegas.append(om)
        q = np.convolve(q, [1.0, -om])
        r_pred = s_j - om * as_j
        r = O.bicgstab(a, b, x0=x0, tol=0.0, maxit=j + 1, variant=variant)
        assert r["iters"] == j + 1
        r_true = b - d @ r["x"]
        assert rel(r_true, r_pred) < 1e-7, (j, rel(r_true, r_pred))
        assert abs(r["omega"][j] - om) < 1e-7 * abs(om)


def test_bicgstab_alpha0_equals_cg_alpha0_on_spd():
    a = W.laplace_2d(16)
    _, b, _ = W.manufactured(a)
    c = O.cg(a, b, maxit=3)
    for v in ("classical", "pipelined"):
        r = O.bicgstab(a, b, maxit=3, variant=v)
        assert abs(r["alpha"][0] - c["alpha"][0]) < 1e-13 * c["alpha"][0]


def test_bicgstab_pipelined_equals_classical_early_scalars():
    """In exact arithmetic the pipelined beta (Sec. 3.2, using <s_i, r0*> = 0) equals the
    classical one; the traces agree to rounding over the first iterations."""
    a = W.convdiff_3d(8)
    _, b, _ = W.manufactured(a)
    c = O.bicgstab(a, b, tol=0.0, maxit=10, variant="classical")
    p = O.bicgstab(a, b, tol=0.0, maxit=10, variant="pipelined")
    for key in ("alpha", "omega", "beta"):
        np.testing.assert_allclose(p[key][:8], c[key][:8], rtol=1e-9)


def test_bicgstab_residual_expansion_matches_direct_norm():
    """Sec. 3.2: <r_{i+1}, r_{i+1}> = <s,s> - 2 omega <s,As> + omega^2 <As,As>."""
    a = W.convdiff_3d(8)
    _, b, _ = W.manufactured(a)
    p = O.bicgstab(a, b, tol=1e-10, maxit=200, variant="pipelined")
    k = p["iters"] - 1
    est, direct = p["res2_est"][:k], p["res2"][:k]
    scale = np.dot(b, b)
    assert np.all(np.abs(est - direct) <= 1e-10 * np.maximum(direct, 1e-6 * scale))


def test_bicgstab_edge_cases():
    a = W.convdiff_3d(4)
    _, b, _ = W.manufactured(a)
    for v in ("classical", "pipelined"):
        r = O.bicgstab(a, np.zeros(a.n), x0=np.ones(a.n), variant=v)
        assert r["status"] == O.OK and r["iters"] == 0 and not r["x"].any()
        r = O.bicgstab(a, b, tol=0.0, maxit=5, variant=v)
        assert r["status"] == O.NOT_CONVERGED and r["iters"] == 5


# ------------------------------------------------------------------------------- GMRES

@pytest.mark.parametrize("variant", ["classical", "pipelined"])
@pytest.mark.parametrize("k", [1, 4, 9])
def test_gmres_iterate_minimises_residual(variant, k):
    """One cycle of k steps gives argmin ||b - A x||_2 over x0 + K_k(A, r0)."""
    a = W.random_uniform(30, 6, seed=11)
    d = a.to_dense()
    _, b, _ = W.manufactured(a, seed=3)
    x0 = W.uniform_pm1(5, a.n)
    r0 = b - d @ x0
    q = krylov_basis(d, r0, k)
    y = np.linalg.lstsq(d @ q, r0, rcond=None)[0]
    xk = x0 + q @ y
    r = O.gmres(a, b, x0=x0, tol=0.0, maxit=k, m=10, variant=variant)
    assert r["iters"] == k and r["cycles"] == 1
    assert rel(r["x"], xk) < 1e-10
    # the in-cycle estimate equals the true minimal residual norm
    assert abs(r["est"][k - 1] - np.linalg.norm(b - d @ xk)) < 1e-9 * np.linalg.norm(r0)


@pytest.mark.parametrize("variant", ["classical", "pipelined"])
def test_full_gmres_terminates(variant):
    a = W.random_uniform(24, 5, seed=2)
    _, b, _ = W.manufactured(a, seed=2)
    ref = np.linalg.solve(a.to_dense(), b)
    r = O.gmres(a, b, tol=1e-6, maxit=200, m=30, variant=variant)
    assert r["status"] == O.OK and r["iters"] <= a.n and r["cycles"] == 1
    # below the 1e-12 floor on the squared in-cycle estimate a restart finishes the job
    r = O.gmres(a, b, tol=1e-11, maxit=200, m=30, variant=variant)
    assert r["status"] == O.OK and r["cycles"] == 2
    assert rel(r["x"], ref) < 1e-10


@pytest.mark.parametrize("variant", ["classical", "pipelined"])
@pytest.mark.parametrize("make", NONSYM)
def test_gmres_restarted_matches_dense_lu(variant, make):
    a = make()
    _, b, _ = W.manufactured(a, seed=6)
    ref = np.linalg.solve(a.to_dense(), b)
    r = O.gmres(a, b, tol=1e-12, maxit=3000, m=8, variant=variant)
    assert r["status"] == O.OK and r["cycles"] >= 1
    assert rel(r["x"], ref) < 1e-9


def test_gmres_classical_and_pipelined_share_R_and_xi():
    """Sec. 3.3: dropping the residual update leaves R and xi unchanged (exact arithmetic)."""
    a = W.convdiff_3d(8)
    _, b, _ = W.manufactured(a)
    c = O.gmres(a, b, tol=0.0, maxit=20, m=20, variant="classical")
    p = O.gmres(a, b, tol=0.0, maxit=20, m=20, variant="pipelined")
    np.testing.assert_allclose(p["R"], c["R"], rtol=0, atol=1e-12 * np.abs(c["R"]).max())
    np.testing.assert_allclose(p["xi"], c["xi"], rtol=0, atol=1e-10)
    R = p["R"]
    assert np.all(np.diag(R) > 0) and np.allclose(np.tril(R, -1), 0)
    assert np.sum(p["xi"] ** 2) <= 1 + 1e-12


def test_gmres_edge_cases():
    a = W.convdiff_3d(4)
    _, b, _ = W.manufactured(a)
    for v in ("classical", "pipelined"):
        r = O.gmres(a, np.zeros(a.n), x0=np.ones(a.n), variant=v)
        assert r["status"] == O.OK and r["iters"] == 0 and not r["x"].any()
        r = O.gmres(a, b, tol=0.0, maxit=13, m=5, variant=v)
        assert r["status"] == O.NOT_CONVERGED and r["iters"] == 13 and r["cycles"] == 3


def test_dot_is_compensated():
    """orc_dot agrees with math.fsum (correctly rounded sum of the rounded products)."""
    import math
    for n in (10, 1000, 300_000):
        x = W.uniform_pm1(11, n)
        y = W.uniform_pm1(12, n)
        for a_, b_ in ((x, y), (np.abs(x), np.abs(y))):
            exact = math.fsum((a_ * b_).tolist())
            bound = 2.3e-16 * abs(exact) + 1e-30 * float(np.sum(np.abs(a_ * b_)))
            assert abs(O.dot(a_, b_) - exact) <= max(bound, 4.5e-16 * abs(exact))


def test_spmv_and_dot_against_dense():
    a = W.power_law(300, seed=1)
    x = W.uniform_pm1(1, a.n)
    np.testing.assert_allclose(O.spmv(a, x), a.to_dense() @ x, rtol=1e-13, atol=1e-12)
    assert abs(O.dot(x, x) - float(np.sum(x * x))) < 1e-12 * float(np.sum(x * x))
