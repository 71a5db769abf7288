"""The bench's multi-rank path on CPU (gloo, world size 2): independent
replicas, job time = max over ranks, work = sum over ranks."""
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

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    # rank r timed steps of (r + 1) ms each; every rank does 1000 units per step
    steps = [float(rank + 1)] * 4
    value, total, w = bench.aggregate(steps, 1000)
    q.put((rank, value, total, w))
    dist.destroy_process_group()


def test_aggregate_over_two_gloo_ranks():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # slowest rank: 4 steps x 2 ms = 8 ms; work: 2 ranks x 4 steps x 1000 units
    for rank, value, total, w in out:
        assert w == 2 and total == pytest.approx(8.0)
        assert value == pytest.approx(2 * 4 * 1000 / 8e-3)


def test_aggregate_single_process():
    import bench

    value, total, w = bench.aggregate([2.0, 2.0], 500)
    assert w == 1 and total == pytest.approx(4.0) and value == pytest.approx(2 * 500 / 4e-3)
