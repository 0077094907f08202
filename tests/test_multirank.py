"""Multi-rank logic on CPU (gloo, world size 2): the test-particle push shards
its particle sets (weak scaling, no collective on the data path; the job's
figures are the slowest rank's time and the summed work), and the GRPIC step
shards the particles over a replicated grid, summing the deposit's sources
over the ranks before the field update."""
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


def _pic_worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import numpy as np
    import oracle as O
    from oracle import pic as P
    from paper_2602_07452_gb300 import inputs as I
    from paper_2602_07452_gb300 import parallel as par
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        a = 0.9
        g = I.log_grid(16, 12, 1.5, 20.0)
        n = 2001
        d, qm, w = I.thermal_draws(n, g, 2.0, 15.0, 0.3, seed=7, qm=50.0)
        z = O.seed_fido(1.0, a, d)
        w = np.linspace(0.5, 1.5, n)
        b0, b1 = par.shard_bounds(n, rank, ws)
        # this rank's deposit, summed over the ranks
        part = [torch.from_numpy(x.copy()) for x in P.deposit(1.0, a, g, z[b0:b1], qm[b0:b1], w[b0:b1])]
        par.allreduce_sources(part)
        full = P.deposit(1.0, a, g, z, qm, w)
        err = max(float(np.abs(part[k].numpy() - full[k]).max() / (np.abs(full[k]).max() + 1e-300))
                  for k in range(4))
        # the replicated field update on the summed sources
        st = P.FdtdState(g)
        Fw = O.wald_on_grid(a, 1.0, g)
        for k in range(3):
            st.D0[k][:] = Fw[k]; st.D1[k][:] = Fw[k]; st.B0[k][:] = Fw[3 + k]; st.B1[k][:] = Fw[3 + k]
        po = P.FdtdParams(1.0, a, 1e-3, 1e4, 5.0, 0.9 * g.rn[-1], g.rn[-1])
        P.fdtd(po, st, 1)
        st.rho1 = part[0].numpy().copy()
        st.j1 = [part[k].numpy().copy() for k in (1, 2, 3)]
        P.fdtd(po, st, 2)
        par.assert_replicas_equal([torch.from_numpy(x) for x in st.D0])
        q.put((rank, err, b1 - b0))
    finally:
        dist.destroy_process_group()


def test_two_rank_pic_sources_allreduce():
    """The sharded GRPIC step on two gloo ranks: each rank deposits its half
    of the particles (the oracle's Sec. 2.3 deposit), the four source arrays
    are summed over the ranks and equal the deposit of all particles to
    rounding; the replicated FDTD then leaves bitwise identical fields on
    both ranks."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_pic_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    assert sum(r[2] for r in res) == 2001
    for rank, err, cnt in res:
        assert err < 1e-13
