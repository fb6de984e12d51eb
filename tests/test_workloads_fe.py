"""Checks of the finite-element input generators (CPU only): sizes of the paper's 2D Poisson
hierarchy and the 3D elasticity shape, symmetry, definiteness, and the kernels of the
unconstrained operators (constants for the Laplacian, rigid-body motions for elasticity) on
rows whose neighbours are all unknowns."""
import numpy as np
import pytest

from paper_1410_4054_gb300 import workloads as W


def rows_of(a):
    return np.repeat(np.arange(a.n), np.diff(a.row_ptr))


@pytest.mark.parametrize("level,n", [(4, 225), (5, 961), (6, 3969)])
def test_fe_poisson_2d_sizes_symmetry_definiteness(level, n):
    a = W.fe_poisson_2d(level, seed=level)
    assert a.n == n
    d = a.to_dense()
    assert np.array_equal(d, d.T)
    if n <= 961:
        assert np.linalg.eigvalsh(d).min() > 0
    assert 6.0 < a.nnz / a.n < 7.0 and np.diff(a.row_ptr).max() <= 9


def test_fe_poisson_2d_rows_annihilate_constants():
    """grad of a constant is zero: every row whose neighbours are all unknowns sums to 0; the
    diagonal is positive and off-diagonals of interior rows sum to minus the diagonal."""
    a = W.fe_poisson_2d(5, seed=3)
    N = 32
    rs = np.bincount(rows_of(a), weights=a.val, minlength=a.n)
    ij = np.stack(np.unravel_index(np.arange(a.n), (N - 1, N - 1)), 1)
    deep = ((ij >= 1) & (ij <= N - 3)).all(1)       # no neighbour on the boundary
    assert np.abs(rs[deep]).max() < 1e-12
    assert (rs[~deep] > 0).all()                     # the Dirichlet rows lose negative entries


def test_fe_elasticity_3d_shape_and_definiteness():
    a = W.fe_elasticity_3d(3, seed=1)
    assert a.n == 3 * 3 * 16
    d = a.to_dense()
    assert np.abs(d - d.T).max() <= 1e-15 * np.abs(d).max()
    assert np.linalg.eigvalsh(0.5 * (d + d.T)).min() > 0
    b = W.fe_elasticity_3d(5, seed=0)
    assert b.n == 540 and np.diff(b.row_ptr).max() == 45


def test_fe_elasticity_3d_rigid_body_motions():
    """Rows of nodes whose element neighbours are all free annihilate the six rigid-body
    motions (three translations, three infinitesimal rotations)."""
    k, seed, jitter = 4, 2, 0.2
    a = W.fe_elasticity_3d(k, seed=seed, jitter=jitter)
    n1 = k + 1
    g = np.arange(n1) / k
    X = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    idx = np.arange(n1 ** 3).reshape(n1, n1, n1)
    move = np.zeros(n1 ** 3, dtype=bool)
    move[idx[1:-1, 1:-1, 1:-1].ravel()] = True
    X = X + np.where(move[:, None], jitter / k * W.uniform_pm1(seed, 3 * n1 ** 3).reshape(-1, 3), 0.0)
    free = np.arange(n1 ** 3).reshape(n1, n1, n1)[1:].ravel()   # x index >= 1
    P = X[free]
    modes = []
    for t in np.eye(3):
        modes.append(np.tile(t, len(free)))
    for axis in np.eye(3):
        modes.append(np.cross(axis, P).ravel())
    node_i = np.arange(n1 ** 3).reshape(n1, n1, n1)
    deep_nodes = set(node_i[2:, :, :].ravel())                     # no neighbour on x = 0
    deep = np.array([free[i // 3] in deep_nodes for i in range(a.n)])
    for m in modes:
        y = a.matvec(m)
        assert np.abs(y[deep]).max() < 1e-12 * np.abs(a.val).max() * np.abs(m).max()
