"""The N > 1 path of bench.py on CPU: replicas-only timing aggregation over a
world_size-2 gloo process group (max over ranks, whole-job throughput)."""
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
    my_ms = 1000.0 if rank == 0 else 2500.0  # rank 1 is the slow one
    max_ms, value = bench.aggregate(my_ms, world, steps=5, dist=dist, device=torch.device("cpu"))
    q.put((rank, max_ms, value))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_world_size_2():
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
    for rank, max_ms, value in out:
        assert max_ms == 2500.0
        assert value == pytest.approx(2 * 5 / 2.5)


def test_single_rank_needs_no_collective():
    import bench
    assert bench.aggregate(500.0, 1, 4) == (500.0, 8.0)
