"""The multi-rank logic of bench.py (torchrun, one replica per GPU) on two
CPU ranks with gloo: every rank gets the slowest rank's time, and the job
rate is all ranks' updates over that time."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        my_ms = 100.0 + 50.0 * rank  # rank 1 is the slow one
        got = bench.max_over_ranks(my_ms, dist, torch.device("cpu"))
        out[rank] = got
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        assert dict(out) == {0: 150.0, 1: 150.0}


def test_whole_job_rate():
    # 2 ranks x 1e6 nodes x 100 steps in 0.1 s = 2 GLUPS
    assert bench.whole_job_rate(1_000_000, 2, 100, 100.0) == pytest.approx(2.0)
    assert bench.max_over_ranks(3.0, None, None) == 3.0


def test_reference_arm_other_ranks_do_no_work(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr("sys.argv", ["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"])
    bench.main()
    assert capsys.readouterr().out == ""


def test_reference_arm_line(monkeypatch, capsys):
    """Rank 0 of the reference arm times the oracle and prints one JSON line."""
    import json
    monkeypatch.delenv("RANK", raising=False)
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    monkeypatch.setattr("sys.argv", ["bench.py", "--impl", "reference", "--steps", "2", "--warmup", "3"])
    bench.main()
    lines = capsys.readouterr().out.strip().splitlines()
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "GLUPS" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["metric"] == bench.METRIC


def test_profiled_traffic_matches_storage_and_source(tmp_path, monkeypatch):
    """The roofline's DRAM traffic comes from the ncu summary of the same
    storage type, taken on the current kernel source, scaled by nodes."""
    good = tmp_path / "good.txt"
    good.write_text(f"kernel_source_sha: {bench.kernel_source_sha()}\ndram_bytes_per_node: 80.0\n")
    stale = tmp_path / "stale.txt"
    stale.write_text("kernel_source_sha: 0000000000000000\ndram_bytes_per_node: 80.0\n")
    monkeypatch.setattr(bench, "PROFILE_SUMMARIES", {"fp32": str(good), "fp16": str(stale)})
    assert bench.profiled_traffic(1000, "fp32") == pytest.approx(80000.0)
    assert bench.profiled_traffic(1000, "fp16") is None   # taken on other sources
    assert bench.profiled_traffic(1000, "bf16") is None   # no summary for this storage
    monkeypatch.setattr(bench, "PROFILE_SUMMARIES", {"fp32": str(tmp_path / "missing.txt")})
    assert bench.profiled_traffic(1000, "fp32") is None
