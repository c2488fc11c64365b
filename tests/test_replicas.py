"""Multi-process host logic of the replicas-only bench path (gloo, world size 2, CPU).

The solve does not shard: with N ranks each runs an independent replica and the
only collective is the max-over-ranks of the timings, which this test checks.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r "timed" 10 + 5 r ms and 0.2 + 0.1 r s
        ms = bench.replica_max(dist, 10.0 + 5.0 * rank, "cpu")
        e2e = bench.replica_max(dist, 0.2 + 0.1 * rank, "cpu")
        out.put((rank, ms, e2e))
    finally:
        dist.destroy_process_group()


def test_replica_timings_take_the_max_over_ranks():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, e2e in res:
        assert ms == pytest.approx(15.0)
        assert e2e == pytest.approx(0.3)


def test_replica_max_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.replica_max(None, 3.5, "cpu") == 3.5
