"""Seeded synthetic inputs shared by the CUDA path, its tests and the oracle.

This module only *builds inputs*: sparse matrices in CSR form (int32 row pointers
and column indices, float64 values), exact solutions x* and right-hand sides
b = A x*.  It contains none of the solvers' arithmetic.  Both the CUDA path and
the CPU oracle receive the very same arrays from here, so neither draws random
numbers of its own.

Shapes follow the paper's workloads (Section 4): 2D/3D Poisson-type stencils
(the finite-element Poisson benchmark of Sec. 4.1 and the 3D elasticity
benchmark of Sec. 4.2 have about 7 nonzeros per row), nonsymmetric
convection-diffusion operators, and power-law random matrices standing in for the
nonsymmetric SuiteSparse matrices of Table 1 (3.8 to 98 nonzeros per row), plus
uniform random matrices with 4 and 28 nonzeros per row for the fused
SpMV + inner product experiment of Sec. 2.2.

x* uses splitmix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) evaluated at counter i, mapped to uniform[-1, 1).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int) -> np.ndarray:
    """Outputs 0..count-1 of splitmix64 started at ``seed`` (uint64 array)."""
    with np.errstate(over="ignore"):
        i = np.arange(1, count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_pm1(seed: int, count: int) -> np.ndarray:
    """uniform[-1, 1) doubles: (u >> 11) * 2^-53 * 2 - 1 with u = splitmix64 output."""
    u = splitmix64(seed, count) >> np.uint64(11)
    return u.astype(np.float64) * (2.0 ** -53) * 2.0 - 1.0


@dataclass
class CSR:
    """A square sparse matrix in CSR form (row_ptr int32[n+1], col int32[nnz], val f64[nnz])."""

    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def matvec(self, x: np.ndarray) -> np.ndarray:
        """y = A x through scipy's CSR kernel (used only to manufacture right-hand sides)."""
        import scipy.sparse as sp

        a = sp.csr_matrix((self.val, self.col, self.row_ptr), shape=(self.n, self.n))
        return a @ x

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.n, self.n))
        for i in range(self.n):
            for j in range(self.row_ptr[i], self.row_ptr[i + 1]):
                d[i, self.col[j]] += self.val[j]
        return d


def _from_coo(n: int, rows: np.ndarray, cols: np.ndarray, vals: np.ndarray, name: str) -> CSR:
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    counts = np.bincount(rows, minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    assert row_ptr[-1] < 2**31
    return CSR(n, row_ptr.astype(np.int32), cols.astype(np.int32), vals.astype(np.float64), name)


def _stencil(shape: tuple, diag: float, lower: float, upper: float, name: str, shift=None) -> CSR:
    """Grid stencil on a lexicographically ordered grid (last axis fastest).

    Each row couples to its 2*d axis neighbours inside the grid (Dirichlet: neighbours
    outside are dropped); ``lower`` is the coefficient of the neighbour at index-1 along
    an axis, ``upper`` that at index+1.  ``shift`` (scalar) is added to the diagonal.
    """
    shape = tuple(int(s) for s in shape)
    n = int(np.prod(shape))
    idx = np.arange(n, dtype=np.int64).reshape(shape)
    rows = [idx.ravel()]
    cols = [idx.ravel()]
    d = diag + (0.0 if shift is None else shift)
    vals = [np.full(n, d)]
    for ax in range(len(shape)):
        lo = [slice(None)] * len(shape)
        hi = [slice(None)] * len(shape)
        lo[ax] = slice(1, None)
        hi[ax] = slice(0, -1)
        r = idx[tuple(lo)].ravel()
        c = idx[tuple(hi)].ravel()
        rows += [r, c]
        cols += [c, r]
        vals += [np.full(r.size, lower), np.full(r.size, upper)]
    return _from_coo(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals), name)


def laplace_2d(k: int, ky: int | None = None, shift: float = 0.0) -> CSR:
    """5-point Laplacian (diag 4 [+shift], neighbours -1) on a ky x k grid, Dirichlet."""
    ky = k if ky is None else ky
    return _stencil((ky, k), 4.0, -1.0, -1.0, f"lap2d_{ky}x{k}", shift)


def laplace_3d(k: int) -> CSR:
    """7-point Laplacian (diag 6, neighbours -1) on a k^3 grid, Dirichlet."""
    return _stencil((k, k, k), 6.0, -1.0, -1.0, f"lap3d_{k}")


def convdiff_3d(k: int, peclet: float = 0.5) -> CSR:
    """First-order upwind convection-diffusion, velocity (1,1,1), cell Peclet ``peclet``.

    Scaled by h^2/D: diffusion gives 6 / -1; upwind convection adds 2*Pe per axis to the
    diagonal and -2*Pe to the upstream (index-1) neighbour.  Pe = 0.5: diag 9, upstream -2,
    downstream -1.
    """
    c = 2.0 * peclet
    return _stencil((k, k, k), 6.0 + 3.0 * c, -1.0 - c, -1.0, f"convdiff3d_{k}")


def _power_law_pmf(lmin: int, lmax: int, mean: float) -> np.ndarray:
    lengths = np.arange(lmin, lmax + 1, dtype=np.float64)

    def mean_for(a):
        w = lengths ** (-a)
        return float((w * lengths).sum() / w.sum())

    lo, hi = 0.0, 10.0  # mean_for is decreasing in a
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if mean_for(mid) > mean:
            lo = mid
        else:
            hi = mid
    w = lengths ** (-0.5 * (lo + hi))
    return w / w.sum()


def power_law(n: int, seed: int = 0, lmin: int = 3, lmax: int = 256, mean: float = 12.0) -> CSR:
    """Random nonsymmetric matrix with power-law row lengths.

    Row length L (diagonal included) ~ P(L) proportional to L^-a on [lmin, lmax], with a set
    by bisection so that E[L] = mean.  The L-1 off-diagonal columns are distinct and uniform
    over the other columns; off-diagonal values are N(0,1); the diagonal is 1.1 times the
    row's absolute off-diagonal sum (strict diagonal dominance).
    """
    rng = np.random.default_rng(seed)
    pmf = _power_law_pmf(lmin, lmax, mean)
    lengths = rng.choice(np.arange(lmin, lmax + 1), size=n, p=pmf).astype(np.int64)
    lengths = np.minimum(lengths, n)
    noff = lengths - 1
    total = int(noff.sum())
    rows = np.repeat(np.arange(n, dtype=np.int64), noff)
    # draw columns from the n-1 "other" columns, then redraw duplicates within a row
    cols = rng.integers(0, n - 1, size=total, dtype=np.int64)
    for _ in range(64):
        key = rows * n + cols
        order = np.argsort(key, kind="stable")
        dup = np.zeros(total, dtype=bool)
        sk = key[order]
        dup[order[1:]] = sk[1:] == sk[:-1]
        if not dup.any():
            break
        cols[dup] = rng.integers(0, n - 1, size=int(dup.sum()), dtype=np.int64)
    cols = np.where(cols >= rows, cols + 1, cols)  # skip the diagonal
    vals = rng.standard_normal(total)
    absum = np.bincount(rows, weights=np.abs(vals), minlength=n)
    diag_rows = np.arange(n, dtype=np.int64)
    return _from_coo(
        n,
        np.concatenate([rows, diag_rows]),
        np.concatenate([cols, diag_rows]),
        np.concatenate([vals, 1.1 * absum]),
        f"powerlaw_{n}",
    )


def spd_power_law(n: int, seed: int = 0, lmin: int = 3, lmax: int = 256, mean: float = 12.0) -> CSR:
    """Symmetric positive definite matrix with power-law row lengths.

    The off-diagonal part of ``power_law(n, seed, ...)`` plus its transpose (coincident
    entries summed); the diagonal is 1.1 times the row's absolute off-diagonal sum plus 1
    (strict diagonal dominance, so SPD).  Rows average about 2 * (mean - 1) + 1 entries and the
    longest reach past ``lmax``.
    """
    p = power_law(n, seed, lmin, lmax, mean)
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(p.row_ptr))
    cols = p.col.astype(np.int64)
    off = cols != rows
    r, c, v = rows[off], cols[off], p.val[off]
    key, inv = np.unique(np.concatenate([r * n + c, c * n + r]), return_inverse=True)
    vals = np.bincount(inv, weights=np.concatenate([v, v]))
    ur, uc = key // n, key % n
    absum = np.bincount(ur, weights=np.abs(vals), minlength=n)
    d = np.arange(n, dtype=np.int64)
    return _from_coo(n, np.concatenate([ur, d]), np.concatenate([uc, d]),
                     np.concatenate([vals, 1.1 * absum + 1.0]), f"spdpowerlaw_{n}")


def spd_dense_rows(k: int = 100, dense=(0, 17, 5000), per_row: int = 9000, seed: int = 0) -> CSR:
    """SPD matrix with a few rows longer than any tile: the 2D 5-point Laplacian on a k x k
    grid plus, for each row r in ``dense``, ``per_row`` couplings to distinct random columns
    (values N(0,1)/per_row, mirrored into the columns), the diagonal raised to 1.1 times the
    absolute row sum plus 1 (strict diagonal dominance).  Stands in for the dense rows of
    arrow-shaped systems (a global constraint or a hub node coupled to many unknowns).
    """
    lap = laplace_2d(k)
    n = lap.n
    rng = np.random.default_rng(seed)
    rows = [np.repeat(np.arange(n, dtype=np.int64), np.diff(lap.row_ptr))]
    cols = [lap.col.astype(np.int64)]
    vals = [lap.val.copy()]
    rows[0], cols[0], vals[0] = rows[0][rows[0] != cols[0]], cols[0][rows[0] != cols[0]], vals[0][rows[0] != cols[0]]
    for r in dense:
        c = rng.choice(np.setdiff1d(np.arange(n), [r]), size=min(per_row, n - 1), replace=False).astype(np.int64)
        v = rng.standard_normal(c.size) / per_row
        rows += [np.full(c.size, r, dtype=np.int64), c]
        cols += [c, np.full(c.size, r, dtype=np.int64)]
        vals += [v, v]
    r_all, c_all, v_all = np.concatenate(rows), np.concatenate(cols), np.concatenate(vals)
    key, inv = np.unique(r_all * n + c_all, return_inverse=True)
    v_sum = np.bincount(inv, weights=v_all)
    ur, uc = key // n, key % n
    absum = np.bincount(ur, weights=np.abs(v_sum), minlength=n)
    d = np.arange(n, dtype=np.int64)
    return _from_coo(n, np.concatenate([ur, d]), np.concatenate([uc, d]),
                     np.concatenate([v_sum, 1.1 * absum + 1.0]), f"spd_dense_rows_{n}")


def diag_scaled(a: CSR, seed: int = 0, spread: float = 100.0) -> CSR:
    """D A D with D = diag(d), ln d uniform on [0, ln spread) from splitmix64(seed).

    Keeps A's sparsity and definiteness while its diagonal spans a factor spread^2: the
    badly scaled systems (cell coefficients that vary over orders of magnitude) on which the
    Jacobi preconditioner diag(A) pays.
    """
    d = np.exp(0.5 * (uniform_pm1(seed, a.n) + 1.0) * np.log(spread))
    rows = np.repeat(np.arange(a.n, dtype=np.int64), np.diff(a.row_ptr))
    return CSR(a.n, a.row_ptr.copy(), a.col.copy(), a.val * d[rows] * d[a.col],
               f"{a.name}_scaled{spread:g}")


def random_uniform(n: int, per_row: int, seed: int = 0) -> CSR:
    """``per_row`` distinct uniformly random columns per row, diagonal included, values N(0,1)
    and a dominant diagonal (the random matrices of the fused SpMV + dot experiment)."""
    rng = np.random.default_rng(seed)
    per_row = min(per_row, n)
    rows = np.repeat(np.arange(n, dtype=np.int64), per_row - 1)
    cols = rng.integers(0, n - 1, size=rows.size, dtype=np.int64)
    for _ in range(64):
        key = rows * n + cols
        order = np.argsort(key, kind="stable")
        sk = key[order]
        dup = np.zeros(rows.size, dtype=bool)
        dup[order[1:]] = sk[1:] == sk[:-1]
        if not dup.any():
            break
        cols[dup] = rng.integers(0, n - 1, size=int(dup.sum()), dtype=np.int64)
    cols = np.where(cols >= rows, cols + 1, cols)
    vals = rng.standard_normal(rows.size)
    absum = np.bincount(rows, weights=np.abs(vals), minlength=n)
    d = np.arange(n, dtype=np.int64)
    return _from_coo(n, np.concatenate([rows, d]), np.concatenate([cols, d]),
                     np.concatenate([vals, 1.1 * absum + 1.0]), f"rand{per_row}_{n}")


def spd_random(n: int, seed: int = 0, density: float = 0.3, cond_shift: float = 1.0) -> CSR:
    """Small dense-ish SPD matrix: B^T B + shift I sparsified symmetrically (tiny tests only)."""
    rng = np.random.default_rng(seed)
    b = rng.standard_normal((n, n))
    mask = rng.random((n, n)) < density
    mask = mask | mask.T | np.eye(n, dtype=bool)
    s = (b + b.T) * mask
    s = s + np.diag(np.abs(s).sum(axis=1) + cond_shift)
    r, c = np.nonzero(s)
    return _from_coo(n, r, c, s[r, c], f"spd_{n}")


def csr_product(a: CSR, x: np.ndarray) -> np.ndarray:
    """y = A x with every product rounded on its own and each row's products added left to
    right, as separate numpy multiply and add operations: the same bits on every host (a
    compiled CSR loop may fuse the multiply-add on one architecture and not on another)."""
    x = np.asarray(x, dtype=np.float64)
    prod = a.val * x[a.col]
    lens = np.diff(a.row_ptr).astype(np.int64)
    order = np.argsort(-lens, kind="stable")  # longest rows first: pass k touches a prefix
    starts = a.row_ptr[:-1].astype(np.int64)[order]
    ys = np.zeros(a.n)
    active = np.searchsorted(-lens[order], 0, side="left")  # rows with at least one entry
    for k in range(int(lens.max()) if a.n else 0):
        while active > 0 and lens[order[active - 1]] <= k:
            active -= 1
        ys[:active] += prod[starts[:active] + k]
    y = np.empty(a.n)
    y[order] = ys
    return y


def manufactured(a: CSR, seed: int = 0):
    """x* uniform[-1,1) from splitmix64(seed), b = A x* (csr_product), x0 = 0."""
    xs = uniform_pm1(seed, a.n)
    b = csr_product(a, xs)
    return xs, b, np.zeros(a.n)


def batched_rectangles(nsys: int = 512, seed: int = 0, lo: int = 32, hi: int = 256):
    """Uneven batch of shifted 2D Laplacians on a x b rectangles.

    Sides a, b = round(exp(U[ln lo, ln hi])); diagonal shift sigma ~ U[0.01, 1].
    Returns a list of CSR matrices.
    """
    rng = np.random.default_rng(seed)
    sides = np.rint(np.exp(rng.uniform(np.log(lo), np.log(hi), size=(nsys, 2)))).astype(int)
    shifts = rng.uniform(0.01, 1.0, size=nsys)
    return [laplace_2d(int(s[0]), int(s[1]), float(sh)) for s, sh in zip(sides, shifts)]


# Named configurations (sizes of the paper-shaped workloads)
LAPLACE_3D_SWEEP = (16, 32, 64, 100, 160)
LAPLACE_2D_SWEEP = (256, 1024, 2048)
CONVDIFF_SWEEP = (32, 64, 128)
POWER_LAW_SWEEP = (10_000, 100_000, 1_000_000)


# ------------------------------------------------------------------ transient heat equation

def _csr_from_coo_summed(n: int, rows: np.ndarray, cols: np.ndarray, vals: np.ndarray, name: str) -> CSR:
    """CSR with coincident (row, col) entries summed (finite-element assembly)."""
    import scipy.sparse as sp

    m = sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr()
    m.sum_duplicates()
    m.sort_indices()
    assert m.nnz < 2**31
    return CSR(n, m.indptr.astype(np.int32), m.indices.astype(np.int32), m.data.astype(np.float64), name)


def fe_poisson_2d(level: int, seed: int = 0, jitter: float = 0.25) -> CSR:
    """Linear (P1) finite elements for -Laplace u = f on the unit square, Dirichlet boundary.

    The mesh: 2^level x 2^level squares, each cut along a diagonal whose direction is drawn
    per square, interior nodes moved by up to ``jitter`` cells in x and y (splitmix64(seed)),
    so that the triangles are irregular and the node valence varies (4..8, mean 6): about 7
    nonzeros per row, (2^level - 1)^2 unknowns (225, 961, 3969, 16129, 65025, 261121 for
    level 4..9), the sizes of the hierarchy of refined triangular meshes of the 2D Poisson
    benchmark.  Element matrices (grad phi_i . grad phi_j) |T|, assembled and summed.
    """
    N = 1 << level
    h = 1.0 / N
    g = np.arange(N + 1)
    X, Y = np.meshgrid(g * h, g * h, indexing="ij")
    inner = np.zeros((N + 1, N + 1), dtype=bool)
    inner[1:-1, 1:-1] = True
    u = uniform_pm1(seed, 2 * (N + 1) ** 2).reshape(2, N + 1, N + 1)
    X = X + np.where(inner, jitter * h * u[0], 0.0)
    Y = Y + np.where(inner, jitter * h * u[1], 0.0)
    node = np.arange((N + 1) ** 2).reshape(N + 1, N + 1)
    a, b_, c, d = node[:-1, :-1].ravel(), node[1:, :-1].ravel(), node[1:, 1:].ravel(), node[:-1, 1:].ravel()
    flip = (splitmix64(seed + 1, N * N) >> np.uint64(63)).astype(bool)
    t1 = np.where(flip[:, None], np.stack([a, b_, d], 1), np.stack([a, b_, c], 1))
    t2 = np.where(flip[:, None], np.stack([b_, c, d], 1), np.stack([a, c, d], 1))
    tri = np.concatenate([t1, t2])
    px, py = X.ravel()[tri], Y.ravel()[tri]
    # gradients of the barycentric coordinates: (y_j - y_k, x_k - x_j) / (2|T|)
    bx = np.stack([py[:, 1] - py[:, 2], py[:, 2] - py[:, 0], py[:, 0] - py[:, 1]], 1)
    by = np.stack([px[:, 2] - px[:, 1], px[:, 0] - px[:, 2], px[:, 1] - px[:, 0]], 1)
    area2 = px[:, 0] * bx[:, 0] + px[:, 1] * bx[:, 1] + px[:, 2] * bx[:, 2]
    assert (area2 > 0).all()
    ke = (bx[:, :, None] * bx[:, None, :] + by[:, :, None] * by[:, None, :]) / (2.0 * area2)[:, None, None]
    dof = np.full((N + 1) ** 2, -1, dtype=np.int64)
    dof[node[inner]] = np.arange((N - 1) ** 2)
    td = dof[tri]
    r = np.broadcast_to(td[:, :, None], ke.shape).ravel()
    c_ = np.broadcast_to(td[:, None, :], ke.shape).ravel()
    keep = (r >= 0) & (c_ >= 0)
    return _csr_from_coo_summed((N - 1) ** 2, r[keep], c_[keep], ke.ravel()[keep], f"fe2d_p1_{N - 1}sq")


def fe_elasticity_3d(k: int, seed: int = 0, jitter: float = 0.2, E: float = 1.0, nu: float = 0.3) -> CSR:
    """Linear (P1) finite elements for isotropic linear elasticity on the unit cube, three
    displacement unknowns per node (3 x 3 blocks), clamped on the face x = 0, free elsewhere.

    The mesh: k^3 cubes, each cut into the six tetrahedra of the Kuhn subdivision, nodes off
    the clamped face moved by up to ``jitter`` cells (splitmix64(seed)).  3 k (k+1)^2
    unknowns (540, 4752, 39744, 324864 for k = 5, 11, 23, 47, near the 693 ... 319,725 of the
    3D elasticity benchmark) and up to 45 nonzeros per row (15 nodes x 3), against the
    benchmark's about 60 from unstructured meshes.  Element matrices |T| B^T D B with B the
    6 x 12 strain-displacement matrix and D the isotropic stiffness (Young's modulus E,
    Poisson ratio nu), assembled and summed: symmetric positive definite.
    """
    n1 = k + 1
    g = np.arange(n1) / k
    X = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    free = X[:, 0] > 0.0
    u = uniform_pm1(seed, 3 * n1 ** 3).reshape(-1, 3)
    move = np.zeros(n1 ** 3, dtype=bool)
    idx = np.arange(n1 ** 3).reshape(n1, n1, n1)
    move[idx[1:-1, 1:-1, 1:-1].ravel()] = True
    X = X + np.where(move[:, None], jitter / k * u, 0.0)
    corner = idx[:-1, :-1, :-1].ravel()
    step = np.array([n1 * n1, n1, 1])
    tets = []
    for perm in ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)):
        v0 = corner
        v1 = v0 + step[perm[0]]
        v2 = v1 + step[perm[1]]
        v3 = v2 + step[perm[2]]
        tets.append(np.stack([v0, v1, v2, v3], 1))
    tet = np.concatenate(tets)
    P = X[tet]                                           # ne x 4 x 3
    M = np.concatenate([np.ones((tet.shape[0], 4, 1)), P], 2)
    vol6 = np.linalg.det(M)
    flipped = vol6 < 0
    tet[flipped] = tet[flipped][:, [0, 2, 1, 3]]
    P = X[tet]
    M = np.concatenate([np.ones((tet.shape[0], 4, 1)), P], 2)
    vol = np.linalg.det(M) / 6.0
    assert (vol > 0).all()
    G = np.linalg.inv(M)[:, 1:, :]                       # ne x 3 x 4: d phi_a / d x_i
    ne = tet.shape[0]
    B = np.zeros((ne, 6, 12))
    for a in range(4):
        gx, gy, gz = G[:, 0, a], G[:, 1, a], G[:, 2, a]
        B[:, 0, 3 * a] = gx
        B[:, 1, 3 * a + 1] = gy
        B[:, 2, 3 * a + 2] = gz
        B[:, 3, 3 * a] = gy
        B[:, 3, 3 * a + 1] = gx
        B[:, 4, 3 * a + 1] = gz
        B[:, 4, 3 * a + 2] = gy
        B[:, 5, 3 * a] = gz
        B[:, 5, 3 * a + 2] = gx
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[np.arange(3), np.arange(3)] += 2 * mu
    D[np.arange(3, 6), np.arange(3, 6)] = mu
    ke = np.einsum("eki,kl,elj->eij", B, D, B) * vol[:, None, None]
    ke = 0.5 * (ke + ke.transpose(0, 2, 1))             # exactly symmetric
    nd = np.full(n1 ** 3, -1, dtype=np.int64)
    nd[free] = np.arange(int(free.sum()))
    td = np.repeat(nd[tet], 3, axis=1) * 3 + np.tile(np.arange(3), 4)
    td = np.where(np.repeat(nd[tet], 3, axis=1) >= 0, td, -1)
    r = np.broadcast_to(td[:, :, None], ke.shape).ravel()
    c = np.broadcast_to(td[:, None, :], ke.shape).ravel()
    keep = (r >= 0) & (c >= 0)
    n = 3 * int(free.sum())
    return _csr_from_coo_summed(n, r[keep], c[keep], ke.ravel()[keep], f"fe3d_elast_{k}")


@dataclass
class Transient:
    """Implicit-Euler heat equation on a k^3 grid: M x_t = x_{t-1} + dt f_t with M = I + dt L."""

    M: CSR
    dt: float
    k: int
    steps: int
    sigma: float
    seed: int

    def source(self, t: int) -> np.ndarray:
        """Gaussian of width sigma cells moving on a circle of radius k/4 around the centre."""
        k = self.k
        th = 2.0 * np.pi * t / self.steps
        c = np.array([k / 2, k / 2 + (k / 4) * np.sin(th), k / 2 + (k / 4) * np.cos(th)])
        z, y, x = np.meshgrid(np.arange(k), np.arange(k), np.arange(k), indexing="ij")
        d2 = (z - c[0]) ** 2 + (y - c[1]) ** 2 + (x - c[2]) ** 2
        return np.exp(-d2 / (2.0 * self.sigma ** 2)).ravel()

    def rhs(self, x_prev: np.ndarray, t: int) -> np.ndarray:
        return x_prev + self.dt * self.source(t)


def _box_filter_3d(a: np.ndarray, w: int) -> np.ndarray:
    """Mean over the w^3 box of in-domain cells around every cell."""
    h = w // 2
    k = a.shape[0]
    s = np.zeros((k + 1,) * 3)
    s[1:, 1:, 1:] = a.cumsum(0).cumsum(1).cumsum(2)
    one = np.zeros((k + 1,) * 3)
    one[1:, 1:, 1:] = np.ones_like(a).cumsum(0).cumsum(1).cumsum(2)
    lo = np.clip(np.arange(k) - h, 0, k)
    hi = np.clip(np.arange(k) + h + 1, 0, k)

    def box(c):
        z0, y0, x0 = np.ix_(lo, lo, lo)
        z1, y1, x1 = np.ix_(hi, hi, hi)
        return (c[z1, y1, x1] - c[z0, y1, x1] - c[z1, y0, x1] - c[z1, y1, x0]
                + c[z0, y0, x1] + c[z0, y1, x0] + c[z1, y0, x0] - c[z0, y0, x0])

    return box(s) / box(one)


def transient_heat(k: int = 64, steps: int = 300, seed: int = 0, sigma: float = 4.0) -> Transient:
    """Variable-coefficient 7-point operator M = I + dt L on a k^3 grid.

    Conductivity: lognormal (mu 0, sigma 1) per cell, smoothed by a 5^3 box filter over the
    in-domain cells; face conductivity = harmonic mean of the two cells; Dirichlet boundary
    faces use the cell's own conductivity.  L_ii = sum of the 6 face conductivities,
    L_ij = -face conductivity.  dt = 2 / max_i L_ii, so the least diagonally dominant row
    has |M_ii| / sum_j |M_ij| = 1.5.
    """
    rng = np.random.default_rng(seed)
    kap = _box_filter_3d(np.exp(rng.standard_normal((k, k, k))), 5)
    n = k ** 3
    idx = np.arange(n, dtype=np.int64).reshape(k, k, k)
    diag = np.zeros((k, k, k))
    rows, cols, vals = [], [], []
    for ax in range(3):
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[ax] = slice(0, -1)
        hi[ax] = slice(1, None)
        ka, kb = kap[tuple(lo)], kap[tuple(hi)]
        kf = 2.0 * ka * kb / (ka + kb)
        diag[tuple(lo)] += kf
        diag[tuple(hi)] += kf
        ia, ib = idx[tuple(lo)].ravel(), idx[tuple(hi)].ravel()
        rows += [ia, ib]
        cols += [ib, ia]
        vals += [-kf.ravel(), -kf.ravel()]
        # boundary faces (one per side) use the cell's conductivity
        first = [slice(None)] * 3
        last = [slice(None)] * 3
        first[ax] = slice(0, 1)
        last[ax] = slice(k - 1, k)
        diag[tuple(first)] += kap[tuple(first)]
        diag[tuple(last)] += kap[tuple(last)]
    dt = 2.0 / diag.max()
    rows.append(idx.ravel())
    cols.append(idx.ravel())
    vals.append(np.zeros(n))
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    v = np.concatenate(vals) * dt
    d = 1.0 + dt * diag.ravel()
    v[-n:] = d
    M = _from_coo(n, r, c, v, f"transient_{k}")
    return Transient(M=M, dt=dt, k=k, steps=steps, sigma=sigma, seed=seed)
