"""bench.py's multi-rank path: independent replicas, aggregated over ranks with
the slowest rank's time and the summed work (world size 2, gloo, CPU)."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=2)
    import bench
    t_dev, t_e2e, work = bench.replica_aggregate(1.0 + rank, 3.0 - rank, 10.0 * (rank + 1))
    q.put((rank, t_dev, t_e2e, work))
    dist.destroy_process_group()


def test_replica_aggregate_two_ranks():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    ps = [mp.Process(target=_worker, args=(r, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in ps:
        p.join(timeout=60)
    for rank, t_dev, t_e2e, work in out:
        assert t_dev == 2.0 and t_e2e == 3.0 and work == 30.0


def test_replica_aggregate_single_process():
    import bench
    assert bench.replica_aggregate(1.5, 2.5, 7.0) == (1.5, 2.5, 7.0)
