"""The N>1 path of bench.py on CPU: two gloo ranks, max-over-ranks time and
summed ops (each rank owns independent tables, so there is no data-path
collective to test).  No GPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [100.0, 250.0][rank]
    ops = [1_000_000, 3_000_000][rank]
    got = bench.aggregate(ms, ops, world)
    q.put((rank, got))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(2))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        ms, val = res[r]
        assert ms == 250.0
        assert val == pytest.approx(4_000_000 / 0.25 / 1e9)


def test_single_rank_aggregate():
    import bench
    ms, val = bench.aggregate(50.0, 10_000_000, 1)
    assert ms == 50.0 and val == pytest.approx(0.2)
