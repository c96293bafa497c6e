"""Multi-GPU host logic on CPU: two gloo ranks run the bench's cross-rank reduction and the
whole-job rate.  The render path shards by independent rays (replicas, no collective on the data
path); the only collectives are the timing barrier and the max over ranks, tested here."""
from __future__ import annotations

import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r measured (100 + 10 r) ms for 4 steps and an e2e of (0.5 + 0.1 r) s
        total_ms, e2e_s = bench.max_over_ranks([100.0 + 10 * rank, 0.5 + 0.1 * rank], "cpu", world)
        dist.barrier()
        value = bench.whole_job_rate(5_120_000, world, 4, total_ms)
        out.put((rank, total_ms, e2e_s, value))
    finally:
        dist.destroy_process_group()


def test_two_rank_max_and_weak_scaling_rate():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, total_ms, e2e_s, value in res:
        assert total_ms == 110.0 and e2e_s == pytest.approx(0.6)
        # both ranks' rays over the slowest rank's time
        assert value == pytest.approx(2 * 5_120_000 * 4 / 0.110 / 1e6)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks([3.0, 4.0], "cpu", 1) == [3.0, 4.0]
    assert bench.whole_job_rate(1_000_000, 1, 10, 1000.0) == pytest.approx(10.0)
