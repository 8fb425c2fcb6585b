"""Host logic of bench.py's multi-rank (replica) path on CPU: two gloo ranks
on 127.0.0.1 reduce their timed regions to the maximum and sum their node
updates."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [800.0, 1000.0][rank]
    updates = [4.0e9, 6.0e9][rank]
    value, t_max, w = bench.aggregate(updates, ms, dist)
    q.put((rank, value, t_max, w))
    dist.destroy_process_group()


def test_replica_aggregation_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, t_max, w in out:
        assert w == 2 and t_max == 1000.0
        assert value == pytest.approx((4.0e9 + 6.0e9) / 1.0 / 1e6)


def test_single_process_aggregation():
    import bench
    value, t_max, w = bench.aggregate(1.0e9, 500.0, None)
    assert (w, t_max) == (1, 500.0) and value == pytest.approx(2000.0)
