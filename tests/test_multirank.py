"""World-size-2 gloo test of the replica aggregation used by bench.py for N > 1 (CPU only)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    value, t = bench.aggregate(units_per_rank=1000.0, seconds_local=1.0 + rank, dist=dist, device="cpu")
    q.put((rank, value, t))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_throughput_uses_max_over_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    for rank, value, t in res:
        assert t == 2.0                                  # the slowest rank sets the job time
        assert abs(value - world * 1000.0 / 2.0) < 1e-9  # all replicas' units / job time


def test_single_process_aggregate_is_plain_rate():
    import bench
    v, t = bench.aggregate(500.0, 0.25)
    assert (v, t) == (2000.0, 0.25)
