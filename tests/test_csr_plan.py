"""The CSR analysis and tile schedule (pk_csr_plan: the host part of pk_csr_create, no GPU):
row statistics, the row-length histogram, and which row schedule the tiles take for each
matrix shape -- one thread per row for stencils, lane groups for rows of similar length,
whole warps for power-law rows, chunk tiles (block per row) for rows longer than a tile."""
import numpy as np
import pytest

from paper_1410_4054_gb300 import pk
from paper_1410_4054_gb300 import workloads as W

EDGES = [8, 16, 32, 64, 256, 4096]


def hist(a):
    lens = np.diff(a.row_ptr)
    b = np.searchsorted(EDGES, lens, side="left")   # bin k: EDGES[k-1] < len <= EDGES[k]
    return np.bincount(b, minlength=7).tolist()


@pytest.mark.parametrize("make,expect", [
    (lambda: W.laplace_3d(24), "thread"),
    (lambda: W.fe_poisson_2d(7), "thread"),
    (lambda: W.fe_elasticity_3d(8), "group"),
    (lambda: W.random_uniform(20_000, 28, seed=1), "group"),
    (lambda: W.power_law(20_000, seed=3), "long"),
    (lambda: W.spd_dense_rows(), "chunk"),
])
def test_schedule_by_matrix_shape(make, expect):
    a = make()
    st = pk.csr_plan(a.row_ptr)
    lens = np.diff(a.row_ptr)
    assert st["n"] == a.n and st["nnz"] == a.nnz
    assert st["row_min"] == lens.min() and st["row_max"] == lens.max()
    assert st["row_mean"] == pytest.approx(a.nnz / a.n)
    assert st["row_hist"] == hist(a) and sum(st["row_hist"]) == a.n
    assert st["kernel"] == 2 and st["values_fp32_exact"] == -1
    tiles = st["tiles_thread"] + st["tiles_group"] + st["tiles_long"]
    assert tiles >= max(a.n // 512, a.nnz // 4096)
    if expect == "thread":
        assert st["tiles_group"] == 0 and st["tiles_long"] == 0
    elif expect == "group":
        assert st["tiles_group"] > 0.9 * tiles
    elif expect == "long":
        assert st["tiles_long"] > 0.5 * tiles
    else:
        long_rows = lens[lens > 4096]
        chunks = int(sum(-(-int(L) // 4096) for L in long_rows))
        assert st["row_hist"][6] == len(long_rows) and st["tiles_long"] >= chunks


def test_plan_matches_rows_longer_than_a_tile_exactly():
    """Every row of more than 4096 nonzeros becomes ceil(len / 4096) chunk tiles: a matrix of
    only such rows (and short ones) has exactly that many long tiles."""
    n = 2000
    lens = np.full(n, 3)
    lens[[0, 999, 1999]] = [4097, 8192, 12289]
    rp = np.zeros(n + 1, dtype=np.int32)
    np.cumsum(lens, out=rp[1:])
    st = pk.csr_plan(rp)
    assert st["tiles_long"] == 2 + 2 + 4
    assert st["row_hist"] == [n - 3, 0, 0, 0, 0, 0, 3]


def test_grid_follows_the_device_size():
    a = W.laplace_3d(40)
    g152 = pk.csr_plan(a.row_ptr, sms=152)["grid"]
    g20 = pk.csr_plan(a.row_ptr, sms=20)["grid"]
    assert g20 < g152


@pytest.mark.parametrize("rp", [np.array([1, 2, 3], np.int32), np.array([0, 3, 2], np.int32)])
def test_invalid_row_pointers_are_rejected(rp):
    with pytest.raises(RuntimeError, match="row_ptr"):
        pk.csr_plan(rp)


def test_empty_matrix():
    st = pk.csr_plan(np.zeros(1, np.int32))
    assert st["n"] == 0 and st["row_hist"] == [0] * 7
