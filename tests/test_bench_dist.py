"""The N > 1 path of bench.py (independent replicas) on CPU: two gloo ranks, the job time is
the slowest rank's, the job value sums the replicas, and the reference arm prints on rank 0
only."""
import json
import multiprocessing as mp
import os
import socket
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]
sys.path.insert(0, str(ROOT))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    sys.path.insert(0, str(ROOT))
    import torch.distributed as td

    import bench

    td.init_process_group("gloo", rank=rank, world_size=ws)
    local_ms = 10.0 + 5.0 * rank
    job_ms = bench.max_over_ranks(local_ms, td, "cpu")
    q.put((rank, job_ms, bench.dist(), bench.job_value(ws, 1e9, job_ms * 1e-3)))
    td.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_replica():
    pytest.importorskip("torch")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [15.0, 15.0]          # max over ranks, on every rank
    assert [o[2] for o in out] == [(2, 0, 0), (2, 1, 1)]  # WORLD_SIZE, RANK, LOCAL_RANK
    assert out[0][3] == pytest.approx(2 * 1e9 / 15e-3 / 1e9)  # whole-job GB/s


def test_single_process_needs_no_group():
    import bench

    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.job_value(1, 2e9, 1.0) == pytest.approx(2.0)


def test_reference_arm_prints_on_rank_zero_only(monkeypatch, capsys):
    import bench

    args = bench.argparse.Namespace(k=12, steps=1, warmup=0, gpus=2)
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""
    monkeypatch.setenv("RANK", "0")
    assert bench.run_reference(args) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["n_gpus"] == 2
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
