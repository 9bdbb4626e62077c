"""The benchmark's multi-rank host logic on CPU: two gloo ranks on 127.0.0.1.

Each rank runs its own replica (no exchange in the data path); the only
collective is the max-reduction of the timings, and the whole-job rate counts
every rank's steps over the slowest rank's time.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, times, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "WORLD_SIZE": str(ws),
                       "RANK": str(rank), "LOCAL_RANK": str(rank)})
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import bench
        worst = bench.max_over_ranks(times[rank], device="cpu")
        rate = bench.job_rate(1000, 4, ws, worst)
        out.put((rank, worst, rate))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    times = [0.25, 0.5]
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, times, out), nprocs=2, join=True, start_method="spawn")
    got = sorted(out.get(timeout=60) for _ in range(2))
    for rank, worst, rate in got:
        assert worst == 0.5
        assert rate == pytest.approx(1000 * 4 * 2 / 0.5)


def test_single_process_needs_no_collective(monkeypatch):
    monkeypatch.setenv("WORLD_SIZE", "1")
    import bench
    assert bench.max_over_ranks(0.125) == 0.125
    assert bench.job_rate(2147483648, 20, 1, 0.5) == pytest.approx(2147483648 * 40)
