"""The C-ABI library builds, loads and exports every entry point include/*.h declares;
host-side argument validation (no GPU needed)."""
import ctypes as C
import re
from pathlib import Path

import numpy as np
import pytest

ROOT = Path(__file__).resolve().parents[1]


def declared_symbols():
    names = set()
    for h in (ROOT / "include").glob("*.h"):
        text = re.sub(r"/\*.*?\*/", "", h.read_text(), flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(pk_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("pk_csr_create", "pk_csr_destroy", "pk_cg_solve", "pk_bicgstab_solve",
                     "pk_gmres_solve", "pk_batched_solve", "pk_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_1410_4054_gb300 import pk
    L = pk.lib()
    missing = [n for n in declared_symbols() if not hasattr(L, n)]
    assert not missing, f"declared but not exported: {missing}"


def test_status_strings_and_version():
    from paper_1410_4054_gb300 import pk
    assert pk.status_string(pk.PK_NOT_SPD) == "PK_NOT_SPD"
    assert pk.status_string(99) == "PK_UNKNOWN"
    assert pk.version() >= 100


def _create(n, nnz, rp, ci, va):
    from paper_1410_4054_gb300 import pk
    h = C.c_void_p()
    st = pk.lib().pk_csr_create(n, nnz, rp.ctypes.data_as(C.c_void_p), ci.ctypes.data_as(C.c_void_p),
                                va.ctypes.data_as(C.c_void_p), 0, None, C.byref(h))
    return st, h


@pytest.mark.parametrize("case", ["row_ptr0", "row_ptr_end", "decreasing", "col_range", "neg_col"])
def test_csr_validation_rejects_bad_input(case):
    from paper_1410_4054_gb300 import pk
    rp = np.array([0, 2, 3, 5], dtype=np.int32)
    ci = np.array([0, 1, 1, 0, 2], dtype=np.int32)
    va = np.ones(5)
    if case == "row_ptr0":
        rp[0] = 1
    elif case == "row_ptr_end":
        rp[-1] = 4
    elif case == "decreasing":
        rp[1] = 4
        rp[2] = 3
    elif case == "col_range":
        ci[3] = 3
    elif case == "neg_col":
        ci[3] = -1
    st, h = _create(3, 5, rp, ci, va)
    assert st == pk.PK_ERR_ARG
    assert pk.lib().pk_last_error().decode()


def test_csr_create_rejects_null_and_sizes():
    from paper_1410_4054_gb300 import pk
    h = C.c_void_p()
    assert pk.lib().pk_csr_create(-1, 0, None, None, None, 0, None, C.byref(h)) == pk.PK_ERR_ARG
    assert pk.lib().pk_csr_create(3, 5, None, None, None, 0, None, C.byref(h)) == pk.PK_ERR_ARG
    assert pk.lib().pk_csr_create(1 << 31, 5, None, None, None, 0, None, C.byref(h)) == pk.PK_ERR_ARG
    assert pk.lib().pk_csr_create(3, 5, None, None, None, 0, None, None) == pk.PK_ERR_ARG


def test_solver_rejects_null_handle():
    from paper_1410_4054_gb300 import pk
    o = pk.make_opts()
    info = pk.Info()
    assert pk.lib().pk_cg_solve(None, None, None, C.byref(o), C.byref(info), None) == pk.PK_ERR_ARG
