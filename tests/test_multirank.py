"""Multi-rank logic on CPU (gloo, world size 2): the test-particle push shards
its particle sets (weak scaling, no collective on the data path; the job's
figures are the slowest rank's time and the summed work), and the GRPIC step
shards the particles over a replicated grid, summing the deposit's sources
over the ranks before the field update."""
import os
import socket

import numpy as np

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
    from paper_2602_07452_gb300 import parallel as par
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        T, W = bench.aggregate(1.0 + rank, 100 * (rank + 1))
        assert bench.dist_env() == (ws, rank, rank)
        # the source sum over separate arrays (packed into one all-reduce)
        ts = [torch.full((5 + k,), float(rank + 1) * (k + 1), dtype=torch.float64) for k in range(4)]
        assert par._flat_span(ts) is None
        par.allreduce_sources(ts)
        assert all(torch.equal(t, torch.full_like(t, 3.0 * (k + 1))) for k, t in enumerate(ts))
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


class _OracleLib:
    """CPU stand-in for the library calls GRPIC.step sequences (the oracle's
    push, Sec. 2.3 deposit and FDTD on torch CPU tensors), recording the
    order of the calls; the real fpic.Fields / fpic.Particles hold the data."""

    def __init__(self, a, g, log):
        import oracle as O
        from oracle import pic as P
        from paper_2602_07452_gb300 import fpic as Fb
        self.O, self.P, self.a, self.g, self.log = O, P, a, g, log
        self.Particles, self.Fields = Fb.Particles, Fb.Fields

    def _state(self, fl):
        st = self.P.FdtdState(self.g)
        for nm in ("B0", "B1", "D0", "D1", "j0", "j1", "E", "H", "Bh", "Dw"):
            setattr(st, nm, [t.numpy() for t in getattr(fl, nm)])
        st.rho0, st.rho1 = fl.rho0.numpy(), fl.rho1.numpy()
        return st

    def fpic_fdtd_step(self, ctx, fl, prm, stage):
        self.log.append("fdtd%d" % stage)
        po = self.P.FdtdParams(1.0, self.a, prm.dt, prm.chi0, prm.lam, prm.r_abs, prm.r_max, prm.conserving)
        self.P.fdtd(po, self._state(fl), stage)

    def fpic_push(self, ctx, p, fields, prm):
        import numpy as np
        self.log.append("push")
        z = np.ascontiguousarray(p.state().numpy())
        Hn, alive = p.Hn.numpy().copy(), p.alive.numpy().copy()
        po = self.O.push_params(a=self.a, dt=prm.dt, scheme=self.O.RK4, r_max=prm.r_max, B0pot=prm.B0pot,
                                field_kind=self.O.FIELD_GRID)
        self.O.push(po, z, p.qm.numpy(), p.H0.numpy(), p.D0.numpy(), Hn, alive, self.g,
                    [np.ascontiguousarray(f.numpy()) for f in fields])
        p.set_state(torch.from_numpy(z))
        p.Hn.copy_(torch.from_numpy(Hn))
        p.alive.copy_(torch.from_numpy(alive))

    def fpic_deposit(self, ctx, p, size, out):
        self.log.append("deposit")
        z = p.state().numpy()
        src = self.P.deposit(1.0, self.a, self.g, z, p.qm.numpy(), p.w.numpy(), p.alive.numpy())
        for t, x in zip(out, src):
            t.copy_(torch.from_numpy(x))


def _grpic_worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    import numpy as np
    import oracle as O
    from oracle import pic as P
    from paper_2602_07452_gb300 import fpic as Fb
    from paper_2602_07452_gb300 import grpic, inputs as I, parallel as par
    if ws > 1:
        dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        a, n, steps = 0.9, 1501, 2
        g = I.log_grid(20, 16, 1.5, 20.0)
        d, qm, w = I.thermal_draws(n, g, 2.0, 15.0, 0.3, seed=9, qm=50.0)
        z = O.seed_fido(1.0, a, d)
        w = np.linspace(0.5, 1.5, n) * 1e-3
        H0, _, D0 = O.hamiltonian(1.0, a, 1.0, z, qm)
        b0, b1 = par.shard_bounds(n, rank, ws)
        m = b1 - b0
        store = Fb.Particles.empty(m, device="cpu")
        store.set_state(torch.from_numpy(z[b0:b1]))
        for nm, x in (("qm", qm), ("w", w), ("H0", H0), ("D0", D0), ("Hn", H0)):
            getattr(store, nm).copy_(torch.from_numpy(np.ascontiguousarray(x[b0:b1])))
        store.alive.fill_(1)
        fl = Fb.Fields(g.size, device="cpu")
        Fw = O.wald_on_grid(a, 1.0, g)
        for k in range(3):
            for lvl in ("D0", "D1", "Bh"):
                getattr(fl, lvl)[k].copy_(torch.from_numpy(Fw[k] if lvl != "Bh" else Fw[3 + k]))
            fl.B0[k].copy_(torch.from_numpy(Fw[3 + k])); fl.B1[k].copy_(torch.from_numpy(Fw[3 + k]))
        log = []
        real_allreduce = par.allreduce_sources

        def logged_allreduce(t, group=None):
            log.append("allreduce")
            real_allreduce(t, group)

        grpic.F = _OracleLib(a, g, log)
        grpic.par.allreduce_sources = logged_allreduce
        push_prm = Fb.push_params(1e-3, scheme=Fb.FPIC_RK4, r_max=float(g.rn[-1]), B0pot=1.0)
        fdtd_prm = Fb.fdtd_params(1e-3, 1e4, 5.0, 0.9 * g.rn[-1], g.rn[-1])
        sim = grpic.GRPIC(None, g, fl, store, m, push_prm, fdtd_prm)
        sim.deposit_initial()
        for _ in range(steps):
            sim.step()
        par.assert_replicas_equal(fl.D0 + fl.D1 + fl.B0 + fl.B1)
        # the sources of the last step: the deposit of every rank's particles
        zl = sim.particles.state().numpy()
        al = sim.particles.alive.numpy()
        if ws > 1:
            sizes = [None] * ws
            dist.all_gather_object(sizes, (zl, al))
            zall = np.concatenate([s[0] for s in sizes]); aall = np.concatenate([s[1] for s in sizes])
        else:
            zall, aall = zl, al
        full = P.deposit(1.0, a, g, zall, qm, w, aall)
        src = (fl.rho0, fl.j0[0], fl.j0[1], fl.j0[2])      # after the level swap
        err = max(float(np.abs(src[k].numpy() - full[k]).max() / (np.abs(full[k]).max() + 1e-300)) for k in range(4))
        q.put((rank, log, err, [t.numpy().copy() for t in fl.D0 + fl.B0]))
    finally:
        if ws > 1:
            dist.destroy_process_group()


def test_two_rank_grpic_step_sequence_and_sources():
    """GRPIC.step on two gloo ranks, each with half of the particles, the
    library calls replaced by the oracle's push, deposit and FDTD on CPU:
    each step calls FDTD 1-4, push, deposit, the one source all-reduce and
    FDTD 7-10 in this order; the summed sources equal the deposit of all
    particles; the replicated fields are bitwise equal on both ranks and
    equal those of the same steps run on one rank with every particle
    (up to the summation order of the sources)."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_grpic_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    res = sorted((q.get(timeout=10) for _ in range(2)), key=lambda r: r[0])
    one = ctx.Queue()
    p1 = ctx.Process(target=_grpic_worker, args=(0, 1, port, one))
    p1.start()
    p1.join(300)
    assert p1.exitcode == 0
    _, log1, err1, F1 = one.get(timeout=10)
    step = ["fdtd1", "push", "deposit", "allreduce", "fdtd2"]
    for rank, log, err, Fr in res:
        assert log == ["deposit", "allreduce"] + step * 2, log
        assert err < 1e-12, err
        for x, y in zip(Fr, F1):
            assert np.abs(x - y).max() <= 1e-12 * (np.abs(y).max() + 1e-300)
    for x, y in zip(res[0][3], res[1][3]):
        assert np.array_equal(x, y)


def test_assign_runs_balances_particles():
    """Independent runs over ranks, largest first to the least loaded rank:
    every run on exactly one rank, and no rank above the even share by more
    than the largest run."""
    from paper_2602_07452_gb300 import parallel as par
    counts = [int(x) for x in np.geomspace(1e5, 4e7, 24)]
    for world in (1, 2, 3, 8):
        out = par.assign_runs(counts, world)
        assert sorted(i for r in out for i in r) == list(range(24))
        loads = [sum(counts[i] for i in r) for r in out]
        assert max(loads) <= sum(counts) / world + max(counts)
    assert par.assign_runs([5, 1, 9, 3, 3, 7], 2) == [[2, 3, 4], [0, 1, 5]]
