"""The allocation-free fused SpMV + inner product (pk_spmv_dot_noalloc).

It is for callers that cannot allocate device memory where they need the product (a memory
budget fixed in advance, no access to the process's caching allocator): it takes the caller's
device CSR arrays and keeps its scratch in a fixed device array.  Checked through the C ABI
against the existing entry point (pk_spmv_dot on a pk_csr handle) and against the oracle's
product and inner product, on two calls in a row.  This file sorts last so that a run
stopping at the first failure has run everything else first.
"""
import ctypes as C

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


def _dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).to(DEV)


@pytest.mark.parametrize("make", [lambda: W.power_law(20_000, seed=3), lambda: W.laplace_3d(24),
                                  lambda: W.random_uniform(3001, 28, seed=1),
                                  lambda: W.laplace_2d(7, 3)])
def test_noalloc_matches_existing_entry_point(make):
    a = make()
    A = pk.CSRMatrix.from_workload(a)
    rp, ci, va = _dev(a.row_ptr, np.int32), _dev(a.col, np.int32), _dev(a.val, np.float64)
    ref_q = torch.zeros(a.n, dtype=torch.float64, device=DEV)
    ref_r = torch.zeros(1, dtype=torch.float64, device=DEV)
    for call in range(2):  # two calls in a row, different inputs
        p = _dev(W.uniform_pm1(10 + call, a.n), np.float64)
        pk.spmv_dot(A, p, ref_q, ref_r, fused=True)
        q = torch.full((a.n,), float("nan"), dtype=torch.float64, device=DEV)
        r = torch.full((1,), float("nan"), dtype=torch.float64, device=DEV)
        pk.spmv_dot_noalloc(a.n, rp, ci, va, p, q, r)
        torch.cuda.synchronize()
        assert torch.equal(q, ref_q)  # same row products, same order
        scale = float(torch.dot(p.abs(), ref_q.abs()))
        assert abs(r.item() - ref_r.item()) <= 1e-12 * scale
        # and the oracle's A p (rows summed left to right) and <p, A p>
        ph = p.cpu().numpy()
        qo = O.spmv(a, ph)
        absrow = W.CSR(a.n, a.row_ptr, a.col, np.abs(a.val)).matvec(np.abs(ph))
        assert np.all(np.abs(q.cpu().numpy() - qo) <= 1e-14 * absrow + 1e-300)
        assert abs(r.item() - O.dot(ph, qo)) <= 1e-12 * float(np.dot(np.abs(ph), absrow))
    A.close()


def test_noalloc_rejects_sizes_beyond_the_limit():
    r = torch.zeros(1, dtype=torch.float64, device=DEV)
    st = pk.lib().pk_spmv_dot_noalloc(pk.NOALLOC_MAX_N + 1, None, None, None, None, None,
                                      C.c_void_p(r.data_ptr()), None)
    assert st == pk.PK_ERR_ARG
    assert "PK_NOALLOC_MAX_N" in pk.lib().pk_last_error().decode()
    # q must not be p (rows read p at other rows' columns while q is written)
    p = torch.zeros(8, dtype=torch.float64, device=DEV)
    rp = _dev(np.arange(9), np.int32)
    st = pk.lib().pk_spmv_dot_noalloc(8, C.c_void_p(rp.data_ptr()), C.c_void_p(rp.data_ptr()),
                                      C.c_void_p(p.data_ptr()), C.c_void_p(p.data_ptr()),
                                      C.c_void_p(p.data_ptr()), C.c_void_p(r.data_ptr()), None)
    assert st == pk.PK_ERR_ARG and "q must not be p" in pk.lib().pk_last_error().decode()
    # n = 0: result 0, nothing else touched
    r.fill_(5.0)
    pk.spmv_dot_noalloc(0, None, None, None, None, None, r)
    torch.cuda.synchronize()
    assert r.item() == 0.0
