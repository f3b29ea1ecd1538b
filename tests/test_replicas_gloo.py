"""The multi-rank (replica) path of bench.py on CPU processes with gloo.

Ranks run independent forward solves, so the only cross-rank operations are
the timing and unit reductions; here two gloo ranks check them: the whole-job
throughput is every rank's units over the slowest rank's time.
"""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        seconds = [2.0, 3.0][rank]
        units = [10.0, 20.0][rank]
        value, t, u = bench.aggregate(world, seconds, units)
        q.put((rank, value, t, u))
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation_with_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    for rank, value, t, u in out:
        assert t == 3.0 and u == 30.0 and value == pytest.approx(10.0)


def test_single_rank_aggregation_is_identity():
    import bench
    assert bench.aggregate(1, 2.0, 8.0) == (4.0, 2.0, 8.0)
