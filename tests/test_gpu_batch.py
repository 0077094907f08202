"""Batched push: several independent spacetimes (spin, grid, Wald field,
particle count) advanced by one explicit and one persistent implicit launch,
equal to pushing each run on its own and to the oracle; and the batched step
captured in a CUDA graph and replayed."""
import numpy as np
import pytest

import oracle as O
from paper_2602_07452_gb300 import inputs as I
from helpers import cuda_or_skip, dev, fpic, make_particles, to_np

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

RUNS = [(0.5, 48, 1000), (0.7, 64, 20011), (0.9, 96, 137), (0.95, 80, 5003), (0.99, 128, 12000)]
DT, THR = 1e-3, 8e-5


def _build(F):
    ctxs, flds, zs, qs, H0s, D0s, grids, Fos = [], [], [], [], [], [], [], []
    for k, (a, N, n) in enumerate(RUNS):
        g = I.wald_grid(N, a, r_max=30.0)
        ctx = F.fpic_init_metric(1.0, a)
        F.fpic_set_grid(ctx, g)
        Fo = O.wald_on_grid(a, 1.0, g)
        d, q, w = I.thermal_draws(n, g, 1.05 * I.horizon(1.0, a), 28.0, 0.1, seed=40 + k)
        z = O.seed_fido(1.0, a, d)
        H0, _, D0 = O.hamiltonian(1.0, a, 1.0, z, q)
        ctxs.append(ctx); flds.append([dev(f) for f in Fo]); zs.append(z); qs.append(q)
        H0s.append(H0); D0s.append(D0); grids.append(g); Fos.append(Fo)
    return ctxs, flds, zs, qs, H0s, D0s, grids, Fos


@pytest.mark.parametrize("newton", [False, True])
def test_batched_equals_separate_and_oracle(newton):
    """Bitwise equal to the runs pushed one by one, within 1e-12 of the
    oracle, with the IMR in its fixed-point or its Newton form."""
    cuda_or_skip()
    F = fpic()
    ctxs, flds, zs, qs, H0s, D0s, grids, Fos = _build(F)
    z = np.concatenate(zs); q = np.concatenate(qs); H0 = np.concatenate(H0s); D0 = np.concatenate(D0s)
    pb = make_particles(z, q, H0, D0, H0.copy())
    off = np.concatenate([[0], np.cumsum([r[2] for r in RUNS])])
    specs = [(ctxs[k], flds[k], int(off[k]), int(off[k + 1]), float(grids[k].rn[-1]), 1.0) for k in range(len(RUNS))]
    runs = F.make_runs(specs)
    prm = F.push_params(DT, scheme=F.FPIC_HYB1, implicit=F.FPIC_IMR, thr=THR, imr_newton=newton)
    st = F.fpic_push_batched(runs, pb, prm, stats=True)
    zb, Hb, ab, sb, ib, cb = to_np(pb)
    tot_impl = 0
    for k in range(len(RUNS)):
        sl = slice(off[k], off[k + 1])
        p1 = make_particles(zs[k], qs[k], H0s[k], D0s[k], H0s[k].copy())
        prm1 = F.push_params(DT, scheme=F.FPIC_HYB1, implicit=F.FPIC_IMR, thr=THR,
                             r_max=float(grids[k].rn[-1]), B0pot=1.0, imr_newton=newton)
        F.fpic_push(ctxs[k], p1, flds[k], prm1)
        z1, H1, a1, s1, i1, c1 = to_np(p1)
        assert np.array_equal(zb[sl], z1) and np.array_equal(sb[sl], s1) and np.array_equal(cb[sl], c1)
        tot_impl += int(s1.sum())
    assert st["n_implicit"] == tot_impl and st["n_alive_before"] == off[-1]
    # one run against the oracle
    k = 3
    sl = slice(off[k], off[k + 1])
    po = O.push_params(a=RUNS[k][0], dt=DT, scheme=O.HYB1, implicit_kind=O.IMR, thr=THR, r_max=grids[k].rn[-1],
                       B0pot=1.0, field_kind=O.FIELD_GRID, imr_newton=newton)
    zo = np.ascontiguousarray(zs[k].copy()); Ho = H0s[k].copy()
    O.push(po, zo, qs[k], H0s[k], D0s[k], Ho, np.ones(RUNS[k][2], np.uint8), grids[k], Fos[k])
    err = (np.abs(zb[sl] - zo) / (np.abs(zo) + 1)).max()
    assert err <= 1e-12, err


def test_batched_step_in_cuda_graph():
    """Three batched steps captured in a CUDA graph and replayed give the same
    particles as three eager batched steps."""
    cuda_or_skip()
    F = fpic()
    ctxs, flds, zs, qs, H0s, D0s, grids, Fos = _build(F)
    z = np.concatenate(zs); q = np.concatenate(qs); H0 = np.concatenate(H0s); D0 = np.concatenate(D0s)
    off = np.concatenate([[0], np.cumsum([r[2] for r in RUNS])])
    specs = [(ctxs[k], flds[k], int(off[k]), int(off[k + 1]), float(grids[k].rn[-1]), 1.0) for k in range(len(RUNS))]
    runs = F.make_runs(specs)
    prm = F.push_params(DT, scheme=F.FPIC_HYB1, implicit=F.FPIC_IMR, thr=THR)
    pe = make_particles(z, q, H0, D0, H0.copy())
    for _ in range(3):
        F.fpic_push_batched(runs, pe, prm)
    pg = make_particles(z, q, H0, D0, H0.copy())
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        F.fpic_push_batched(runs, pg, prm)        # warm-up outside capture (scratch, tables)
    torch.cuda.synchronize()
    pg2 = make_particles(z, q, H0, D0, H0.copy())
    for name in ("r", "th", "ph", "ur", "uth", "uph", "Hn", "alive"):
        getattr(pg, name).copy_(getattr(pg2, name))
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        for _ in range(3):
            F.fpic_push_batched(runs, pg, prm, stream=s)
    graph.replay()
    torch.cuda.synchronize()
    assert np.array_equal(pg.state().cpu().numpy(), pe.state().cpu().numpy())
    assert np.array_equal(pg.Hn.cpu().numpy(), pe.Hn.cpu().numpy())


@pytest.mark.parametrize("newton", [False, True])
def test_batched_learned_corrector_equals_separate(newton):
    """fpic_push_batched_learned (the corrector form on the batched kernels)
    gives bitwise the particles of fpic_push_learned on each run alone, with
    the same network and configuration (here the zero network: the
    leading-order gap alone), and the scheme choices of the plain batched
    push; the sampled run stays within 1e-12 of the oracle."""
    cuda_or_skip()
    F = fpic()
    ctxs, flds, zs, qs, H0s, D0s, grids, Fos = _build(F)
    z = np.concatenate(zs); q = np.concatenate(qs); H0 = np.concatenate(H0s); D0 = np.concatenate(D0s)
    off = np.concatenate([[0], np.cumsum([r[2] for r in RUNS])])
    specs = [(ctxs[k], flds[k], int(off[k]), int(off[k + 1]), float(grids[k].rn[-1]), 1.0) for k in range(len(RUNS))]
    runs = F.make_runs(specs)
    net0 = F.MLP()
    net0.set_params(torch.zeros(F.MLP.nparams(), dtype=torch.float32, device="cuda"))
    cfg = F.learned_cfg(mode=F.FPIC_LEARN_CORRECT)
    prm = F.push_params(DT, scheme=F.FPIC_HYB1, implicit=F.FPIC_IMR, thr=THR, imr_newton=newton)
    pb = make_particles(z, q, H0, D0, H0.copy())
    st = F.fpic_push_batched_learned(runs, net0, pb, prm, cfg, stats=True)
    zb, Hb, ab, sb, ib, cb = to_np(pb)
    pp = make_particles(z, q, H0, D0, H0.copy())
    F.fpic_push_batched(runs, pp, prm)
    assert np.array_equal(to_np(pp)[3], sb)
    tot_impl = 0
    for k in range(len(RUNS)):
        sl = slice(off[k], off[k + 1])
        p1 = make_particles(zs[k], qs[k], H0s[k], D0s[k], H0s[k].copy())
        prm1 = F.push_params(DT, scheme=F.FPIC_HYB1, implicit=F.FPIC_IMR, thr=THR,
                             r_max=float(grids[k].rn[-1]), B0pot=1.0, imr_newton=newton)
        F.fpic_push_learned(ctxs[k], net0, p1, flds[k], prm1, cfg)
        z1, H1, a1, s1, i1, c1 = to_np(p1)
        assert np.array_equal(zb[sl], z1) and np.array_equal(sb[sl], s1) and np.array_equal(ib[sl], i1)
        tot_impl += int(s1.sum())
    assert st["n_implicit"] == tot_impl > 0
    k = 1
    sl = slice(off[k], off[k + 1])
    po = O.push_params(a=RUNS[k][0], dt=DT, scheme=O.HYB1, implicit_kind=O.IMR, thr=THR, r_max=grids[k].rn[-1],
                       B0pot=1.0, field_kind=O.FIELD_GRID, imr_newton=newton)
    zo = np.ascontiguousarray(zs[k].copy()); Ho = H0s[k].copy()
    O.push(po, zo, qs[k], H0s[k], D0s[k], Ho, np.ones(RUNS[k][2], np.uint8), grids[k], Fos[k])
    err = (np.abs(zb[sl] - zo) / (np.abs(zo) + 1)).max()
    assert err <= 1e-12, err


def test_graph_survives_a_larger_call_on_the_same_context():
    """A plain batched step is captured in a CUDA graph; then a learned
    batched call on the same contexts needs more scratch, and the library
    allocates a larger buffer (device free memory drops) while keeping the
    superseded one alive until fpic_destroy; replaying the first graph
    afterwards gives bitwise the particles of an uncaptured plain step from
    the same state."""
    cuda_or_skip()
    F = fpic()
    ctxs, flds, zs, qs, H0s, D0s, grids, Fos = _build(F)
    z = np.concatenate(zs); q = np.concatenate(qs); H0 = np.concatenate(H0s); D0 = np.concatenate(D0s)
    off = np.concatenate([[0], np.cumsum([r[2] for r in RUNS])])
    specs = [(ctxs[k], flds[k], int(off[k]), int(off[k + 1]), float(grids[k].rn[-1]), 1.0) for k in range(len(RUNS))]
    runs = F.make_runs(specs)
    prm = F.push_params(DT, scheme=F.FPIC_HYB1, implicit=F.FPIC_IMR, thr=THR)
    s = torch.cuda.Stream()
    pg = make_particles(z, q, H0, D0, H0.copy())
    with torch.cuda.stream(s):
        F.fpic_push_batched(runs, pg, prm, stream=s)      # warm-up outside capture (scratch, tables)
    torch.cuda.synchronize()
    p0 = make_particles(z, q, H0, D0, H0.copy())
    for name in ("r", "th", "ph", "ur", "uth", "uph", "Hn", "alive"):
        getattr(pg, name).copy_(getattr(p0, name))
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        F.fpic_push_batched(runs, pg, prm, stream=s)
    torch.cuda.synchronize()
    # a larger call on the same context grows its scratch
    net0 = F.MLP()
    net0.set_params(torch.zeros(F.MLP.nparams(), dtype=torch.float32, device="cuda"))
    cfg = F.learned_cfg(mode=F.FPIC_LEARN_CORRECT)
    pl = make_particles(z, q, H0, D0, H0.copy())
    free0 = torch.cuda.mem_get_info()[0]
    F.fpic_push_batched_learned(runs, net0, pl, prm, cfg)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] < free0 - len(q) * 64      # the learned scratch is new memory
    graph.replay()
    torch.cuda.synchronize()
    pe = make_particles(z, q, H0, D0, H0.copy())
    F.fpic_push_batched(runs, pe, prm)
    torch.cuda.synchronize()
    for x, y in zip(to_np(pg), to_np(pe)):
        assert np.array_equal(x, y)
