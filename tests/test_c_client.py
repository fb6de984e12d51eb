"""The boundary is a plain C ABI (CPU only): a C program compiled against include/pk.h and
linked to libpk.so (no Python, no torch) calls the entry points that need no GPU and gets
the same results as the Python binding."""
import shutil
import subprocess
from pathlib import Path

import numpy as np
import pytest

from paper_1410_4054_gb300 import pk
from paper_1410_4054_gb300 import workloads as W

ROOT = Path(__file__).resolve().parents[1]

PROGRAM = r"""
#include <stdio.h>
#include <stdlib.h>
#include "pk.h"

int main(void) {
  /* row pointers of the 5-point Laplacian on a k x k grid */
  const int k = 40, n = k * k;
  int32_t* rp = (int32_t*)malloc(sizeof(int32_t) * (n + 1));
  rp[0] = 0;
  for (int i = 0; i < n; ++i) {
    const int x = i % k, y = i / k;
    rp[i + 1] = rp[i] + 1 + (x > 0) + (x < k - 1) + (y > 0) + (y < k - 1);
  }
  pk_csr_stats st;
  pk_status s = pk_csr_plan(n, rp[n], rp, 152, &st);
  printf("plan %d %lld %lld %d %d %d %d %d %d\n", (int)s, (long long)st.n, (long long)st.nnz,
         st.row_min, st.row_max, st.grid, st.tiles_thread, st.tiles_group, st.tiles_long);
  rp[n / 2] = -1; /* not nondecreasing */
  s = pk_csr_plan(n, rp[n], rp, 152, &st);
  printf("bad %d %s | %s\n", (int)s, pk_status_string(s), pk_last_error());
  pk_csr* h = (pk_csr*)1;
  s = pk_csr_create(-1, 0, NULL, NULL, NULL, 0, NULL, &h);
  printf("create %d %d\n", (int)s, h == NULL);
  printf("version %d\n", (int)pk_version());
  free(rp);
  return 0;
}
"""


def test_plain_c_program_uses_the_library(tmp_path):
    if shutil.which("gcc") is None:  # pragma: no cover
        pytest.skip("gcc not available")
    pk.lib()  # builds libpk.so if needed
    lib = Path(pk.lib_path())
    src, exe = tmp_path / "client.c", tmp_path / "client"
    src.write_text(PROGRAM)
    subprocess.run(["gcc", "-std=c11", "-I", str(ROOT / "include"), "-o", str(exe), str(src),
                    str(lib), f"-Wl,-rpath,{lib.parent}"], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True, timeout=60).stdout
    lines = dict(ln.split(" ", 1) for ln in out.strip().splitlines())

    ref = pk.csr_plan(W.laplace_2d(40).row_ptr, sms=152)
    got = [int(v) for v in lines["plan"].split()]
    assert got == [pk.PK_OK, ref["n"], ref["nnz"], ref["row_min"], ref["row_max"], ref["grid"],
                   ref["tiles_thread"], ref["tiles_group"], ref["tiles_long"]]
    code, rest = lines["bad"].split(" ", 1)
    assert int(code) == pk.PK_ERR_ARG and rest.startswith("PK_ERR_ARG | row_ptr")
    assert lines["create"].split() == [str(pk.PK_ERR_ARG), "1"]
    assert int(lines["version"]) == pk.lib().pk_version()
    assert np.array_equal(W.laplace_2d(40).row_ptr[:3], [0, 3, 7])
