"""bench.py's multi-rank logic on the CPU: N independent replicas, one per
GPU, whose job time is the slowest rank's (an all-reduce of one number), and
whose throughput counts every rank's units.  Two gloo ranks on 127.0.0.1 stand
in for two GPUs; no kernel runs."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        job = bench.max_over_ranks(10.0 + 5.0 * rank, world, device="cpu")
        q.put((rank, job, bench.whole_job_rate(1000, 4, world, job)))
    finally:
        dist.destroy_process_group()


def test_job_time_is_slowest_rank_and_rate_counts_all_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert [g[1] for g in got] == [15.0, 15.0]
    # 1000 units x 4 steps x 2 ranks in 15 ms.
    assert all(abs(g[2] - 8000 / 0.015) < 1e-6 for g in got)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5


def test_reference_arm_runs_on_rank_zero_only(capsys):
    import bench
    os.environ["RANK"], os.environ["WORLD_SIZE"] = "1", "2"
    try:
        assert bench.run_reference(None, None) is None  # returns before any work
    finally:
        del os.environ["RANK"], os.environ["WORLD_SIZE"]
    assert capsys.readouterr().out == ""
