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
