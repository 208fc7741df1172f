"""The benchmark's host logic on CPU: two gloo ranks (one process each) meet
at the barrier, take the slowest rank's time and report the whole-job rate;
a non-zero rank of the reference arm exits without work; the batched
workload's oracle baseline (one core, then a spawn-started pool)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, q) -> None:
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        ms = bench.max_over_ranks(10.0 + rank, world)  # rank 1 is the slowest
        q.put((rank, ms, bench.whole_job_rate(1000.0, ms, world)))
        bench.barrier(world)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_report_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(60)
    assert [p.exitcode for p in procs] == [0, 0]
    assert [r for r, _, _ in got] == [0, 1]
    for _, ms, rate in got:
        assert ms == 11.0                                 # max over ranks
        assert rate == pytest.approx(2 * 1000.0 / 0.011)  # both ranks' units over the slowest time


def test_single_rank_needs_no_process_group():
    import bench

    assert bench.max_over_ranks(3.5, 1) == 3.5
    bench.barrier(1)
    assert bench.whole_job_rate(500.0, 250.0, 1) == pytest.approx(2000.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    import argparse

    import bench

    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    args = argparse.Namespace(workload="rmat12", steps=1, warmup=0, ref_seconds=0.1)
    assert bench.run_reference(args) == 0  # returns before any work


def test_oracle_batch_sample_single_and_all_cores():
    """The batched workload's CPU baseline: one core, then the same graphs
    over a spawn-started process pool; both count the same edges."""
    import bench

    r = bench.oracle_batch_sample(0.05, 2, limit=3)
    n = int(r["sample"].split("graphs 0..")[1].split(" ")[0]) + 1
    assert 1 <= n <= 3 and r["cores"] == 1 and r["all_cores"]["cores"] == 2
    assert r["value"] > 0 and r["all_cores"]["value"] > 0


def test_host_cpu_is_recorded():
    import bench

    h = bench.host_cpu()
    assert h["nproc"] == os.cpu_count() and h["machine"] and isinstance(h["model"], str)


def test_traffic_guard_covers_the_round1_kernels():
    """The traffic record's hash covers the round-1 kernels' source (found by
    its markers), not the rest of their file."""
    import bench

    sec = bench.round1_section()
    assert "k_round1_count" in sec and "k_round1(" in sec and "tile_rows" in sec
    assert "k_merge_new" not in sec and "k_index_build" not in sec


def test_reference_arm_line_matches_the_main_line_config(monkeypatch, capsys):
    """Rank 0 of the reference arm prints one JSON line whose config carries
    the main line's keys (rounds from the full oracle run: rmat12's largest
    distance is 3) and says what its ms_per_step times."""
    import argparse
    import json

    import bench

    monkeypatch.setenv("WORLD_SIZE", "1")
    monkeypatch.setenv("RANK", "0")
    args = argparse.Namespace(workload="rmat12", steps=1, warmup=0, cpu_seconds=0.2, batch_hubs=0)
    assert bench.run_reference(args) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    cfg = line["config"]
    assert cfg["workload"] == "rmat12" and cfg["labels"] == 82231
    assert cfg["rounds"] == 4 and cfg["parallelism"] == "single" and cfg["batch_hubs"] == 0
    assert "sample" in line["ms_per_step_is"] and line["estimated_ms_per_build"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0
