"""The ctypes binding agrees with include/pk.h (CPU only): a small C program compiled against
the header prints the size and every field offset of pk_opts, pk_info and pk_csr_stats and the
values of the enums and defines the binding mirrors; each must equal the binding's."""
import ctypes as C
import shutil
import subprocess
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]

CONSTANTS = {
    "PK_OK": "PK_OK", "PK_ERR_ARG": "PK_ERR_ARG", "PK_ERR_CUDA": "PK_ERR_CUDA", "PK_ERR_OOM": "PK_ERR_OOM",
    "PK_NOT_CONVERGED": "PK_NOT_CONVERGED", "PK_BREAKDOWN": "PK_BREAKDOWN", "PK_NOT_SPD": "PK_NOT_SPD",
    "PK_ERR_NAN": "PK_ERR_NAN", "PK_TIMEOUT": "PK_TIMEOUT",
    "FLAG_TIMING": "PK_FLAG_TIMING", "FLAG_TRUE_RES": "PK_FLAG_TRUE_RES", "FLAG_NO_TMA": "PK_FLAG_NO_TMA",
    "FLAG_AUTOTUNE": "PK_FLAG_AUTOTUNE", "FLAG_SELL": "PK_FLAG_SELL", "FLAG_CGS2": "PK_FLAG_CGS2",
    "FLAG_TEST_STALL": "PK_FLAG_TEST_STALL", "FLAG_GM_SHIFT": "PK_FLAG_GM_SHIFT",
    "PERSISTENT_AUTO_N": "PK_PERSISTENT_AUTO_N", "PERSISTENT_AUTO_NNZ": "PK_PERSISTENT_AUTO_NNZ",
    "PERSISTENT_BICGSTAB_AUTO_N": "PK_PERSISTENT_BICGSTAB_AUTO_N",
    "PERSISTENT_BICGSTAB_AUTO_NNZ": "PK_PERSISTENT_BICGSTAB_AUTO_NNZ",
    "PERSISTENT_GMRES_AUTO_N": "PK_PERSISTENT_GMRES_AUTO_N", "PERSISTENT_GMRES_AUTO_NNZ": "PK_PERSISTENT_GMRES_AUTO_NNZ",
    "MAX_SLOTS": "PK_MAX_KERNEL_SLOTS",
}
TABLES = {
    "VARIANTS": {"pipelined": "PK_VARIANT_PIPELINED", "classical": "PK_VARIANT_CLASSICAL",
                 "split": "PK_VARIANT_SPLIT"},
    "PRECISIONS": {"fp64": "PK_PREC_FP64", "mixed": "PK_PREC_MIXED"},
    "LOOPS": {"graph": "PK_LOOP_GRAPH", "host": "PK_LOOP_HOST", "persistent": "PK_LOOP_PERSISTENT",
              "auto": "PK_LOOP_AUTO", "resident": "PK_LOOP_RESIDENT"},
    "PRECONDS": {"none": "PK_PRECOND_NONE", "jacobi": "PK_PRECOND_JACOBI"},
}
SLOTS = ["PK_SLOT_SPMV_DOTS", "PK_SLOT_UPDATE", "PK_SLOT_MULTIDOT", "PK_SLOT_ORTHO", "PK_SLOT_SPMV",
         "PK_SLOT_BLAS1", "PK_SLOT_OTHER", "PK_SLOT_RESIDENT"]


@pytest.fixture(scope="module")
def header_values(tmp_path_factory):
    if shutil.which("gcc") is None:  # pragma: no cover
        pytest.skip("gcc not available")
    from paper_1410_4054_gb300 import pk

    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pk.h"', "int main(void) {"]
    for cname, st in (("pk_opts", pk.Opts), ("pk_info", pk.Info), ("pk_csr_stats", pk.Stats)):
        lines.append(f'  printf("size {cname} %zu\\n", sizeof({cname}));')
        for f, _ in st._fields_:
            lines.append(f'  printf("off {cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    names = set(CONSTANTS.values()) | {c for t in TABLES.values() for c in t.values()} | set(SLOTS)
    for c in sorted(names):
        lines.append(f'  printf("const {c} %lld\\n", (long long)({c}));')
    lines += ["  return 0;", "}"]
    d = tmp_path_factory.mktemp("abi")
    src, exe = d / "layout.c", d / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run(["gcc", "-std=c11", "-I", str(ROOT / "include"), "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    vals = {}
    for ln in out.splitlines():
        kind, key, v = ln.split()
        vals[(kind, key)] = int(v)
    return vals


def test_struct_layouts_match(header_values):
    from paper_1410_4054_gb300 import pk

    for cname, st in (("pk_opts", pk.Opts), ("pk_info", pk.Info), ("pk_csr_stats", pk.Stats)):
        assert header_values[("size", cname)] == C.sizeof(st), cname
        for f, _ in st._fields_:
            assert header_values[("off", f"{cname}.{f}")] == getattr(st, f).offset, (cname, f)


def test_constants_match(header_values):
    from paper_1410_4054_gb300 import pk

    for py, c in CONSTANTS.items():
        assert getattr(pk, py) == header_values[("const", c)], py
    for table, entries in TABLES.items():
        t = getattr(pk, table)
        for k, c in entries.items():
            assert t[k] == header_values[("const", c)], (table, k)
    assert [header_values[("const", c)] for c in SLOTS] == list(range(len(pk.SLOTS)))
