"""Multi-rank path of bench.py on CPU (gloo, world size 2): every rank runs an
independent replica; the timed region is the max over ranks and the value is
that time divided by (ranks x steps)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put((rank, bench.aggregate(10.0 * (rank + 1), 5, world, device="cpu")))
    finally:
        dist.destroy_process_group()


def test_replica_aggregation_world2():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        elapsed, value = out[r]
        assert elapsed == 20.0            # max over ranks
        assert value == 20.0 / (5 * 2)    # whole-job ms per decomposition


def test_single_rank_aggregation():
    import bench
    assert bench.aggregate(12.0, 4, 1) == (12.0, 3.0)
