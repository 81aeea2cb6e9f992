"""The multi-process path of bench.py on CPU: two gloo ranks (replicas, no
data-path collective) agree on the slowest rank's time and the whole-job
throughput counts every rank's frames."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    my_ms = [120.0, 150.0][rank]
    tot = bench.max_over_ranks(my_ms, world, "cpu")
    q.put((rank, tot, bench.job_throughput(world, 10, 1024 * 1024, tot)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[1] for g in got] == [150.0, 150.0]
    # 2 ranks x 10 frames x 1 Mpix in 150 ms
    assert got[0][2] == pytest.approx(2 * 10 * 1024 * 1024 / 0.150 / 1e6)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
