"""bench.py host logic (CPU only).

The algorithmic byte counts behind its rooflines are rebuilt here from the arrays each kernel
reads and writes: CSR values (8 B) and column indices (4 B) per nonzero, row pointers (4 B per
row + 1), and 8 B per FP64 vector element.  Also the working-set label and the summary of the
clock samples taken during the timed region."""
import sys
from pathlib import Path

import pytest

sys.path.insert(0, str(Path(__file__).resolve().parents[1]))
import bench  # noqa: E402

from paper_1410_4054_gb300 import workloads as W  # noqa: E402


def csr(n, nnz):
    return 8 * nnz + 4 * nnz + 4 * (n + 1)


@pytest.mark.parametrize("n,nnz", [(4_096_000, 28_518_400), (2_097_152, 14_581_760), (1, 1)])
def test_cg_kernel_bytes(n, nnz):
    vec = 8 * n
    # K-CG-S: the matrix, p gathered once, Ap written
    assert bench.spmv_dots_bytes(n, nnz) == csr(n, nnz) + vec + vec
    # K-CG-U: read x, r, p, Ap; write x, r, p
    assert bench.update_bytes(n) == 4 * vec + 3 * vec
    # one iteration = one K-CG-U + one K-CG-S = 12 nnz + 76 n + 4
    per_it = bench.bytes_per_solve(n, nnz, 11) - bench.bytes_per_solve(n, nnz, 10)
    assert per_it == bench.spmv_dots_bytes(n, nnz) + bench.update_bytes(n) == 12 * nnz + 76 * n + 4
    # setup: r0 = b - A x0 (matrix, read b, x; write r, p) and the first K-CG-S
    assert bench.bytes_per_solve(n, nnz, 0) == csr(n, nnz) + 4 * vec


def test_headline_workload_bytes():
    a = W.laplace_3d(160)
    assert (a.n, a.nnz) == (4_096_000, 28_518_400)
    assert bench.spmv_dots_bytes(a.n, a.nnz) == 424_140_804
    assert bench.bytes_per_solve(a.n, a.nnz, 1) - bench.bytes_per_solve(a.n, a.nnz, 0) == 653_516_804


def test_job_value_sums_replicas():
    assert bench.job_value(1, 5e9, 1.0) == pytest.approx(5.0)
    assert bench.job_value(4, 5e9, 2.0) == pytest.approx(10.0)


def test_working_set_and_l2_label():
    a = W.laplace_3d(160)
    assert bench.working_set_bytes(a.n, a.nnz) == 12 * a.nnz + 4 * (a.n + 1) + 5 * 8 * a.n
    assert bench.config(160, a)["l2"].startswith("inputs larger than L2 (working set ~522 MB")
    small = W.laplace_3d(64)
    assert bench.working_set_bytes(small.n, small.nnz) <= bench.L2_BYTES
    assert bench.config(64, small)["l2"].startswith("working set ~33 MB <= 129 MB L2")


class _DoneProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_samples_are_summarised(tmp_path):
    """The nvidia-smi sampler's CSV (sm, max sm, active mask, four throttle reasons) becomes
    the median SM clock, the max clock and the set of throttle reasons seen."""
    csv = tmp_path / "clocks.csv"
    csv.write_text("2070, 2070, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                   "1980, 2070, 0x4, Not Active, Not Active, Not Active, Active\n"
                   "2070, 2070, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                   "[N/A], 2070, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                   "truncated line\n")
    c = bench.Clocks(0)
    c.proc, c.path = _DoneProc(), str(csv)
    out = c.stop()
    assert out == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert not csv.exists()


def test_clock_sampler_absent_gives_none():
    assert bench.Clocks(0).stop() is None


def test_traffic_counters_are_reported_only_for_the_profiled_source(monkeypatch):
    """The roofline's DRAM traffic comes from a committed ncu capture and is dropped as soon
    as the kernel sources differ from the ones that capture ran."""
    t = bench.ncu_traffic("k_cg_spmv_dots", "lap3d_160")
    assert t is not None and 0.5 * 424_140_804 < t < 1.5 * 424_140_804
    assert bench.ncu_traffic("k_cg_spmv_dots", "lap3d_999") is None
    monkeypatch.setattr(bench, "kernel_source_sha", lambda: "0" * 16)
    assert bench.ncu_traffic("k_cg_spmv_dots", "lap3d_160") is None


def test_peak_comes_from_the_measured_file():
    peak, kind = bench.measured_peaks()
    if (Path(bench.ROOT) / "MEASURED_PEAKS.json").exists():
        assert kind == "measured" and 5000 < peak < 8000
    else:  # pragma: no cover
        assert (peak, kind) == (6800.0, "fallback")
