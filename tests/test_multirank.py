"""CPU test of the multi-rank (weak-scaling replica) timing path of bench.py
with the gloo backend, world size 2: the job time is the slowest rank's and
the job throughput counts every rank's units."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r took (r + 1) * 100 ms for 10 steps of 2e6 targets
    ms, value = bench.aggregate_ranks((rank + 1) * 100.0, 10, 2e6, world, "cpu")
    q.put((rank, ms, value))
    dist.destroy_process_group()


def test_aggregate_ranks_gloo_world2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in res:
        assert ms == pytest.approx(20.0)                 # max over ranks: 200 ms / 10 steps
        assert value == pytest.approx(2 * 2e6 / 0.020)   # both ranks' targets


def test_aggregate_ranks_single():
    import bench
    ms, value = bench.aggregate_ranks(50.0, 5, 1e6, 1)
    assert ms == 10.0 and value == pytest.approx(1e8)
