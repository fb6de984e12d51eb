"""The stored full-size oracle solves (tests/golden/oracle_fullsize.json, written by
tests/golden/make_oracle_fullsize.py from oracle/ alone) still describe the current oracle and
inputs (CPU only): the stencil matrices and right-hand sides hash as stored, and the cheapest
case, BiCGStab on the power-law matrix with 10^5 rows, reruns to the stored iteration count
and sampled entries of x."""
import hashlib
import json
from pathlib import Path

import numpy as np

import oracle as O
from paper_1410_4054_gb300 import workloads as W

FIX = json.loads((Path(__file__).resolve().parent / "golden" / "oracle_fullsize.json").read_text())["cases"]


def sha(*arrays):
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()[:24]


def test_fixture_covers_the_benchmark_configs():
    assert set(FIX) == {"cg:lap3d_160", "cg:lap2d_2048", "bicgstab:convdiff_128", "gmres:convdiff_128",
                        "bicgstab:powerlaw_1e5", "gmres:powerlaw_1e5", "bicgstab:powerlaw_1e6",
                        "gmres:powerlaw_1e6"}
    for key, rec in FIX.items():
        assert rec["status"] == O.OK and rec["iters"] > 0, key
        assert len(rec["x_idx"]) == len(rec["x_vals"]) == 64
        assert len(rec["iters_perturbed"]) == (8 if key.startswith("bicgstab") else 2)
        assert rec["x_fixed_spread"] >= 0 and rec["tol"] == 1e-8


def test_stencil_inputs_hash_as_stored():
    for key, make in (("cg:lap3d_160", lambda: W.laplace_3d(160)), ("cg:lap2d_2048", lambda: W.laplace_2d(2048)),
                      ("gmres:convdiff_128", lambda: W.convdiff_3d(128))):
        a = make()
        _, b, _ = W.manufactured(a, seed=0)
        assert sha(a.row_ptr, a.col, a.val) == FIX[key]["matrix_sha"], key
        assert sha(b) == FIX[key]["b_sha"], key


def test_cheapest_case_reruns_to_the_stored_result():
    rec = FIX["bicgstab:powerlaw_1e5"]
    a = W.power_law(100_000, seed=0)
    _, b, _ = W.manufactured(a, seed=0)
    assert sha(a.row_ptr, a.col, a.val) == rec["matrix_sha"] and sha(b) == rec["b_sha"]
    r = O.bicgstab(a, b, tol=1e-8, maxit=50_000, variant="pipelined", cap=1)
    assert r["iters"] == rec["iters"] and r["status"] == rec["status"]
    assert np.array_equal(r["x"][rec["x_idx"]], np.array(rec["x_vals"]))
