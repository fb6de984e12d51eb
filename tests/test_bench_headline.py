"""bench.py's result line (CPU only): it is the last stdout line, parses as JSON, stays under
2 KB with every key the benchmark contract names, and the CPU baseline reports the faster of
the one-core oracle and its OpenMP copy on every host core."""
import json
import os
import subprocess
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]
sys.path.insert(0, str(ROOT))
import bench  # noqa: E402

from paper_1410_4054_gb300 import workloads as W  # noqa: E402

KEYS = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
        "scaling", "vs_baseline", "dtype", "data", "config", "e2e", "roofline", "cpu_baseline",
        "clocks", "gpu_launches"}


def _cpu_small():
    a = W.laplace_3d(16)
    _, b, _ = W.manufactured(a, seed=0)
    return bench.cpu_legs(a, b, 16, it1=4, itp=4)


def test_cpu_legs_report_the_faster_one_on_host_cores():
    cpu = _cpu_small()
    import oracle as O
    assert cpu["kind"] == "oracle" and cpu["unit"] == bench.UNIT and cpu["value"] > 0
    if O.omp_lib() is not None:
        assert set(cpu["legs"]) == {"one_core", "all_cores"}
        assert cpu["value"] == pytest.approx(max(cpu["legs"].values()), rel=1e-3)
        best = max(cpu["legs"], key=cpu["legs"].get)
        assert cpu["cores"] == (len(os.sched_getaffinity(0)) if best == "all_cores" else 1)
    else:
        assert cpu["cores"] == 1


def test_openmp_copy_follows_the_sequential_oracle():
    import oracle as O
    if O.omp_lib() is None:
        pytest.skip("gcc without OpenMP")
    a = W.laplace_3d(12)
    _, b, _ = W.manufactured(a, seed=1)
    seq = O.cg(a, b, tol=1e-10, maxit=500)
    for t in (1, 3):
        par = O.cg_omp(a, b, tol=1e-10, maxit=500, threads=t)
        assert par["status"] == seq["status"] == O.OK
        assert abs(par["iters"] - seq["iters"]) <= 1
        assert abs(par["x"] - seq["x"]).max() <= 1e-12 * abs(seq["x"]).max()


def test_headline_is_short_and_complete():
    a = W.laplace_3d(160)
    args = bench.argparse.Namespace(steps=20, warmup=5)
    roof = {"bound": "hbm", "achieved": 4685.123456789, "peak": 6790.7, "unit": "GB/s",
            "frac": 0.6899999999, "traffic": 402_123_456, "kernel": "k_cg_spmv_dots_tma (K-CG-S)",
            "peak_source": "of measured (MEASURED_PEAKS.json hbm_gbs)",
            "algorithmic_bytes_per_launch": bench.spmv_dots_bytes(a.n, a.nnz), "launch_ms": 0.0905123}
    e2e = {"value": 5073.2222222, "unit": "GB/s", "h2d_bytes_per_step": 16 * a.n,
           "d2h_bytes_per_step": 8 * a.n, "ms_per_step": 48.999999}
    clk = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 480}
    s = bench.headline(value=5121.987654321, ws=1, args=args, ms=48.3333333, cfg=bench.config(160, a),
                       it=378, launches=15160, e2e=e2e, roofline=roof, cpu=_cpu_small(), clk=clk)
    assert "\n" not in s and len(s) < bench.HEADLINE_MAX
    line = json.loads(s)
    assert KEYS <= set(line)
    assert line["e2e"]["h2d_bytes_per_step"] > 0 and line["e2e"]["d2h_bytes_per_step"] > 0
    assert set(line["roofline"]) >= {"bound", "achieved", "peak", "unit", "frac", "traffic"}
    assert line["config"]["workload"].startswith("pipelined CG")


def test_detail_lines_are_separate_json(capsys):
    bench.emit_detail("sweep", {"matrix": "lap3d_16", "n": 4096})
    bench.emit_detail("form:batched", {"systems": 512})
    out = capsys.readouterr().out.splitlines()
    assert [json.loads(x)["detail"] for x in out] == ["sweep", "form:batched"]


def test_reference_arm_last_line_parses():
    r = subprocess.run([sys.executable, str(ROOT / "bench.py"), "--impl", "reference", "--k", "20",
                        "--steps", "2", "--warmup", "1"], capture_output=True, text=True, timeout=300,
                       cwd=str(ROOT))
    assert r.returncode == 0, r.stderr
    last = r.stdout.strip().splitlines()[-1]
    assert len(last) < bench.HEADLINE_MAX
    line = json.loads(last)
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["cores"] in (1, len(os.sched_getaffinity(0)))
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
