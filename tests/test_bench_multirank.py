"""The benchmark's multi-GPU bookkeeping (one independent replica per rank)
on CPU with the gloo backend: whole-job time is the slowest rank's, work is
summed, and the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, moves = bench.job_totals(torch, 10.0 + 5.0 * rank, 1000 * (rank + 1), "cpu")
    env = bench.dist_env()
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ms, moves, env))


def test_two_rank_totals_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get() for _ in range(2))
    for rank, ms, moves, env in got:
        assert ms == 15.0 and moves == 3000.0            # max time, summed work
        assert env == (2, rank, rank)


def test_single_process_totals_unchanged():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_totals(torch, 12.5, 77, "cpu") == (12.5, 77.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")

    class A:
        steps, warmup = 1, 3
    bench.run_reference(A())
    assert capsys.readouterr().out == ""


def test_reference_arm_line_on_one_process(monkeypatch, capsys):
    # the oracle timed as the reference arm: one JSON line with the GPU
    # arm's metric, unit and direction, its CPU sample described, no copies
    sys.path.insert(0, ROOT)
    import json
    import bench
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)

    class A:
        steps, warmup = 1, 3
    from paper_1509_04692_gb300 import inputs
    small = inputs.large2d(42, N=1 << 14)            # the headline recipe on a smaller box
    bench.run_reference(A(), system=small, melt=3)
    lines = capsys.readouterr().out.strip().splitlines()
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True and d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 3
    assert d["value"] > 0 and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["host"]["nproc"] >= 1 and d["cpu_baseline"]["host"]["model"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == small.name and d["config"]["melt_sweeps"] == 3
    assert d["cpu_baseline"]["cores"] == os.cpu_count()
    assert bench.WORKLOAD.startswith("2^24 regular pentagons")


def test_clock_sampler_keeps_samples_of_the_timed_region(tmp_path, monkeypatch):
    # a stand-in for nvidia-smi that prints one CSV line per 50 ms, the first
    # one before the timed region starts (left out of the record)
    sys.path.insert(0, ROOT)
    import time
    import bench
    exe = tmp_path / "nvidia-smi"
    exe.write_text("#!/bin/bash\n"
                   "echo '0, 1200, 2070, 90.0, 0x0, Not Active, Not Active, Not Active, Not Active'\n"
                   "while true; do\n"
                   "  echo '0, 2070, 2070, 900.0, 0x4, Not Active, Not Active, Not Active, Active'\n"
                   "  sleep 0.05\n"
                   "done\n")
    exe.chmod(0o755)
    monkeypatch.setenv("PATH", f"{tmp_path}:{os.environ['PATH']}")
    s = bench.ClockSampler(0, period_ms=50)
    time.sleep(0.4)
    c = s.stop()
    assert c["samples"] >= 3 and c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"]
    monkeypatch.setenv("PATH", str(tmp_path / "none"))
    assert bench.ClockSampler(0).stop()["reasons"] == ["nvidia-smi unavailable"]
