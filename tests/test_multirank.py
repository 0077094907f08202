"""Multi-rank logic of the benchmark on CPU (gloo, world size 2): each rank
pushes its own particle set (weak scaling, no collective on the data path);
the job's figures are the slowest rank's time and the summed work."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        T, W = bench.aggregate(1.0 + rank, 100 * (rank + 1))
        assert bench.dist_env() == (ws, rank, rank)
        q.put((rank, T, W))
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, T, W in res:
        assert T == 2.0 and W == 300.0


def test_single_process_aggregation():
    import bench
    assert bench.aggregate(1.5, 42) == (1.5, 42.0)
