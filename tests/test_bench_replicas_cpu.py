"""bench.py's multi-GPU path runs independent replicas (the path shards by grid, but one job
runs on one GPU): the job's time is the slowest rank's and its throughput all ranks' work
over that time.  Checked with two gloo ranks on CPU."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        times = [0.010 + 0.005 * rank, 0.100 - 0.010 * rank]  # rank 1 slower on the first region
        units = [1e9, 2e9]
        q.put((rank, bench.aggregate(times, units, world, device="cpu")))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        times, vals = got[r]
        assert times == pytest.approx([0.015, 0.100])
        assert vals == pytest.approx([2 * 1e9 / 0.015, 2 * 2e9 / 0.100])


def test_single_rank_needs_no_process_group():
    import bench
    times, vals = bench.aggregate([0.5], [1e9], 1)
    assert times == [0.5] and vals == [2e9]
