"""The benchmark's N > 1 path (replicas: one independent reconstruction per rank)
on CPU with the gloo backend, world size 2: the job time is the slowest rank's
and the throughput counts every rank's pairs."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 100.0 + 50.0 * rank  # rank 1 is the slow one
    q.put((rank, bench.aggregate_timing(local_ms, 10, world, dist, "cpu")))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_timing_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        total, per_step, value = res[r]
        assert total == 150.0 and per_step == 15.0
        assert value == pytest.approx(2 * 10 / 0.150)


def test_single_rank_timing_needs_no_process_group():
    import bench
    assert bench.aggregate_timing(200.0, 20, 1) == (200.0, 10.0, pytest.approx(100.0))
