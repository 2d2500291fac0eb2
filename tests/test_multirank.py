"""The benchmark's N > 1 host logic on CPU, as two gloo ranks (no GPU).

The path runs replicas (independent solves per rank, no collective on the
data path): the job's time is the slowest rank's, its value counts every
rank's solves, and the reference arm runs on rank 0 only.
"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, q) -> None:
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      LOCAL_RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        # rank 1 is slower in the first time, faster in the second
        got = bench.job_times([10.0 + rank, 3.0 - rank], world, "cpu")
        q.put((rank, got, bench.dist_env()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank_time():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        results = sorted(q.get(timeout=120) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert [p.exitcode for p in procs] == [0, 0]
    assert [r[0] for r in results] == [0, 1]
    for rank, got, env in results:
        assert got == [11.0, 3.0]
        assert env == (rank, rank, 2)


def test_job_rate_counts_every_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_rate(1, 16, 0.5) == 32.0
    assert bench.job_rate(4, 16, 0.5) == 128.0
    assert bench.job_times([1.5, 2.0], 1, "cpu") == [1.5, 2.0]


def test_reference_arm_prints_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2",
                                      "--steps", "1", "--warmup", "0"])
    bench.main()
    assert capsys.readouterr().out == ""
