"""The seeded input recipes (CPU only): generator test vectors, closed forms of the stencil
matrices, and the stated properties of the random and transient workloads.

The same generators feed the oracle and the CUDA path, so a mistake here would not show up
as a parity failure; these tests tie them to their published definitions instead."""
import numpy as np
import pytest

from paper_1410_4054_gb300 import workloads as W


def dense(a):
    return a.to_dense()


def test_splitmix64_published_test_vectors():
    """Outputs of the reference splitmix64 (Steele, Lea, Flood 2014; Vigna's C version)."""
    assert [int(v) for v in W.splitmix64(1234567, 5)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423,
        4593380528125082431, 16408922859458223821]
    assert [int(v) for v in W.splitmix64(0, 3)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniform_pm1_mapping_and_range():
    u = W.uniform_pm1(0, 100_000)
    assert u[0] == (0xE220A8397B1DCDAF >> 11) * 2.0 ** -53 * 2.0 - 1.0
    assert u.min() >= -1.0 and u.max() < 1.0
    assert abs(u.mean()) < 0.01 and abs(u.var() - 1.0 / 3.0) < 0.01


@pytest.mark.parametrize("k", [5, 8])
def test_laplacians_match_their_closed_forms(k):
    for a, dim in ((W.laplace_2d(k), 2), (W.laplace_3d(k), 3)):
        assert a.n == k ** dim
        assert a.nnz == (5 * k * k - 4 * k if dim == 2 else 7 * k ** 3 - 6 * k * k)
        d = dense(a)
        assert np.array_equal(d, d.T)
        assert set(np.unique(np.diag(d))) == {2.0 * dim}
        off = d - np.diag(np.diag(d))
        assert set(np.unique(off)) <= {0.0, -1.0}
        ev = np.linalg.eigvalsh(d)
        lam = lambda j: dim * (2.0 - 2.0 * np.cos(j * np.pi / (k + 1)))  # noqa: E731
        np.testing.assert_allclose([ev[0], ev[-1]], [lam(1), lam(k)], rtol=1e-12)


def test_rectangle_laplacian_with_shift():
    a = W.laplace_2d(7, 4, shift=0.25)
    assert a.n == 28 and a.nnz == 5 * 28 - 2 * 7 - 2 * 4
    assert np.allclose(np.diag(dense(a)), 4.25)


def test_convdiff_upwind_coefficients():
    """Pe = 0.5 per axis: diagonal 9, the upstream (index - 1) neighbour -2, downstream -1."""
    k = 6
    a = W.convdiff_3d(k)
    d = dense(a)
    assert a.nnz == 7 * k ** 3 - 6 * k * k
    assert np.all(np.diag(d) == 9.0)
    i = (2 * k + 3) * k + 2  # interior cell (z, y, x) = (2, 3, 2)
    for step in (1, k, k * k):
        assert d[i, i - step] == -2.0 and d[i, i + step] == -1.0
    assert d[i].sum() == 0.0
    assert not np.array_equal(d, d.T)


def test_power_law_rows():
    n = 20_000
    a = W.power_law(n, seed=3)
    lens = np.diff(a.row_ptr)
    assert lens.min() >= 3 and lens.max() <= 256
    assert abs(lens.mean() - 12.0) < 0.3
    rows = np.repeat(np.arange(n), lens)
    assert np.unique(rows * n + a.col.astype(np.int64)).size == a.nnz  # distinct columns per row
    is_diag = a.col == rows
    assert np.array_equal(np.bincount(rows[is_diag], minlength=n), np.ones(n, dtype=np.int64))
    absum = np.bincount(rows[~is_diag], weights=np.abs(a.val[~is_diag]), minlength=n)
    np.testing.assert_allclose(a.val[is_diag], 1.1 * absum, rtol=1e-14)
    # the length distribution falls off as a power law: short rows dominate, long rows exist
    assert (lens <= 8).mean() > 0.6 and (lens > 64).sum() > 0


def test_power_law_pmf_mean_is_exact():
    p = W._power_law_pmf(3, 256, 12.0)
    L = np.arange(3, 257)
    assert p.sum() == pytest.approx(1.0, abs=1e-14)
    assert (p * L).sum() == pytest.approx(12.0, rel=1e-10)
    assert np.all(np.diff(p) < 0)


def test_batched_rectangles_recipe():
    mats = W.batched_rectangles(512, seed=0)
    assert len(mats) == 512
    sides, shifts = [], []
    for m in mats:
        d0 = float(m.val[m.col == 0][0])  # row 0's diagonal = 4 + sigma
        shifts.append(d0 - 4.0)
        sides.append(m.n)
    shifts = np.array(shifts)
    assert shifts.min() >= 0.01 and shifts.max() <= 1.0
    n = np.array(sides)
    assert n.min() >= 32 * 32 and n.max() <= 256 * 256
    # log-uniform sides on [32, 256]: the median side is near sqrt(32 * 256) ~ 90.5
    assert 0.8 * 90.5 ** 2 < np.median(n) < 1.25 * 90.5 ** 2


def test_transient_operator():
    tr = W.transient_heat(k=10, steps=20, seed=1)
    M = dense(tr.M)
    assert np.allclose(M, M.T, rtol=0, atol=1e-15)
    L = (M - np.eye(tr.M.n)) / tr.dt
    diagL = np.diag(L)
    assert tr.dt == pytest.approx(2.0 / diagL.max(), rel=1e-12)
    off = np.abs(L - np.diag(diagL)).sum(axis=1)
    slack = diagL - off  # boundary-face conductivities; zero on interior rows
    assert slack.min() > -1e-12
    interior = np.zeros((10, 10, 10), dtype=bool)
    interior[1:-1, 1:-1, 1:-1] = True
    assert np.abs(slack[interior.ravel()]).max() < 1e-12
    ratio = np.diag(M) / (np.abs(M - np.diag(np.diag(M))).sum(axis=1))
    assert ratio.min() >= 1.5 * (1 - 1e-12)
    # right-hand side b_t = x_{t-1} + dt f_t with a Gaussian source of peak 1
    f = tr.source(0)
    assert f.max() <= 1.0 and f.max() > 0.9
    x = W.uniform_pm1(2, tr.M.n)
    np.testing.assert_allclose(tr.rhs(x, 0), x + tr.dt * f, rtol=0, atol=0)


def test_manufactured_right_hand_side():
    a = W.laplace_2d(9, 5)
    xs, b, x0 = W.manufactured(a, seed=4)
    np.testing.assert_array_equal(xs, W.uniform_pm1(4, a.n))
    np.testing.assert_allclose(b, dense(a) @ xs, rtol=1e-15, atol=1e-15)
    assert not x0.any()
