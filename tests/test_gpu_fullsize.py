"""Parity at the benchmark's full sizes, in the launch configuration the
benchmark times, on sampled outputs the oracle computes one by one:

* the charged Wald push (2^20 particles, 512 x 512 grid, a = 0.9, Hyb1
  RK4 <-> IMR, dt = 1e-3, the autotuned implicit launch shape): every
  sampled particle's step against the oracle's;
* the deposit of the plasma-filled Wald step (1024 x 1024 grid, 64
  particles per cell, a = 0.99): sampled interior nodes of rho, j^r, j^th,
  j^ph against the oracle's deposit of the particles that can reach them.

Inputs are the seeded draws of the benchmark, turned into states by the
oracle's own seeding (no input comes from the CUDA path)."""
import numpy as np
import pytest

import oracle as O
from oracle import pic as P
from paper_2602_07452_gb300 import inputs as I
from helpers import cuda_or_skip, fields_dev, fpic, make_particles, to_np

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

A, B0, THETA_T, QM, DT, NGRID, THR = 0.9, 1.0, 0.1, 100.0, 1e-3, 512, 3.5e-6


def test_fullsize_charged_push_sampled():
    cuda_or_skip()
    F = fpic()
    n = 1 << 20
    g = I.wald_grid(NGRID, A)
    Fo = O.wald_on_grid(A, B0, g)
    ctx = F.fpic_init_metric(1.0, A)
    F.fpic_set_grid(ctx, g)
    d, q, w = I.thermal_draws(n, g, 1.02 * I.horizon(1.0, A), 49.0, THETA_T, seed=2, qm=QM)
    z = O.seed_fido(1.0, A, d)
    H0, _, D0 = O.hamiltonian(1.0, A, B0, z, q)
    fd = fields_dev(Fo)
    prm = F.push_params(DT, scheme=F.FPIC_HYB1, implicit=F.FPIC_IMR, thr=THR, r_max=float(g.rn[-1]), B0pot=B0)
    p = make_particles(z, q, H0, D0, H0.copy())
    from paper_2602_07452_gb300 import autotune
    autotune.tune_imr_blocks(ctx, p, fd, prm, reps=1)
    st = F.fpic_push(ctx, p, fd, prm, stats=True)
    assert 0.05 < st["n_implicit"] / st["n_alive_before"] < 0.6
    zg, Hg, ag, sg, ig, cg = to_np(p)
    rng = np.random.default_rng(7)
    idx = np.sort(rng.choice(n, 4000, replace=False))
    po = O.push_params(a=A, dt=DT, scheme=O.HYB1, implicit_kind=O.IMR, thr=THR, r_max=g.rn[-1], B0pot=B0,
                       field_kind=O.FIELD_GRID)
    zo = np.ascontiguousarray(z[idx]); Ho = H0[idx].copy(); ao = np.ones(len(idx), np.uint8)
    O.push(po, zo, q[idx], H0[idx], D0[idx], Ho, ao, g, Fo)
    # scheme choice: the oracle's Hyb1 statistic of each sampled particle
    pr = O.push_params(a=A, dt=DT, scheme=O.RK4, r_max=g.rn[-1], B0pot=B0, field_kind=O.FIELD_GRID)
    zr = np.ascontiguousarray(z[idx]); Hr = H0[idx].copy()
    O.push(pr, zr, q[idx], H0[idx], D0[idx], Hr, np.ones(len(idx), np.uint8), g, Fo)
    stat = np.abs(Hr - H0[idx]) / D0[idx] / DT
    near = np.abs(stat - THR) < 1e-9 * THR
    imp = stat >= THR
    assert np.array_equal(sg[idx][~near], imp[~near].astype(np.uint8))
    # the alive flag is bit-exact, except where the state lies within the
    # parity bound of a removal boundary (r_+ or r_max)
    rb = np.array([I.horizon(1.0, A), g.rn[-1]])
    edge = (np.abs(zo[:, 0, None] / rb[None, :] - 1.0) <= 1e-12).any(axis=1)
    ok = ~near & ~edge
    assert edge.sum() <= 1 and np.array_equal(ag[idx][ok], ao[ok])
    live = ok & (ao == 1)
    err = (np.abs(zg[idx] - zo) / (np.abs(zo) + 1.0)).max(axis=1)
    assert err[live].max() <= 1e-12, err[live].max()
    assert np.array_equal(cg[idx][live], O.cell_index(g, zo[live, 0], zo[live, 1]).astype(np.uint32))


def test_fullsize_deposit_sampled_nodes():
    cuda_or_skip()
    F = fpic()
    a, N, ppc = 0.99, 1024, 64
    g = I.wald_grid(N, a)
    ctx = F.fpic_init_metric(1.0, a)
    F.fpic_set_grid(ctx, g)
    d, q, w = I.cell_fill_draws(g, ppc, 0.5, seed=3, qm=QM, r_lo=1.02 * I.horizon(1.0, a))
    z = O.seed_fido(1.0, a, d)
    del d
    n = len(q)
    w = np.full(n, 1e-6)
    p = make_particles(z, q, w=w)
    out = [t.cpu().numpy() for t in F.fpic_deposit(ctx, p, g.size)]
    del p
    # integer cell of every particle (the oracle's), bucketed once, to pick
    # the particles of each sampled node's 4 x 4-cell neighbourhood
    key = (np.searchsorted(g.rn, z[:, 0], side="right") - 1) * g.Nth + \
          (np.searchsorted(g.tn, z[:, 1], side="right") - 1)
    order = np.argsort(key, kind="stable")
    start = np.searchsorted(key[order], np.arange(g.Nr * g.Nth + 1))
    rng = np.random.default_rng(11)
    i_lo = int(np.searchsorted(g.rn, 1.02 * I.horizon(1.0, a))) + 3
    nodes = [(int(rng.integers(i_lo, g.Nr - 3)), int(rng.integers(3, g.Nth - 3))) for _ in range(40)]
    for (i, j) in nodes:
        sel = np.concatenate([order[start[ci * g.Nth + j - 2]:start[ci * g.Nth + j + 2]]
                              for ci in range(i - 2, i + 2)])
        ro = P.deposit(1.0, a, g, z[sel], q[sel], w[sel])
        sc = P.deposit(1.0, a, g, z[sel], np.abs(q[sel]), w[sel])[0]
        o = i * g.ld + j
        scale = sc[o]
        assert scale > 0
        for k in range(4):
            assert abs(out[k][o] - ro[k][o]) <= 1e-10 * scale, (i, j, k, out[k][o], ro[k][o], scale)


def test_fullsize_div_clean():
    """Sec. 2.4 cleaning on the 1024 x 1024 plasma grid (a = 0.99) with the
    paper's 500 Jacobi sweeps, in the benchmark's launch configuration: the
    oracle solves the whole grid, so every entry of the corrected D and of
    phi is compared (1e-10 of their scale)."""
    cuda_or_skip()
    F = fpic()
    a = 0.99
    g = I.wald_grid(1024, a)
    Fo = O.wald_on_grid(a, 1.0, g)
    rng = np.random.default_rng(8)
    D = [Fo[k] + 1e-3 * rng.normal(size=g.size) for k in range(3)]
    rho = 1e-3 * rng.normal(size=g.size)
    ctx = F.fpic_init_metric(1.0, a)
    F.fpic_set_grid(ctx, g)
    Dd = [torch.as_tensor(x, device="cuda") for x in D]
    phi = F.fpic_div_clean(ctx, Dd, torch.as_tensor(rho, device="cuda"), 500, want_phi=True)
    Dc, phio = P.div_clean(1.0, a, g, D, rho, 500)
    for k in range(3):
        got = Dd[k].cpu().numpy()
        sc = np.abs(Dc[k]).max()
        assert np.abs(got - Dc[k]).max() <= 1e-10 * sc, k
    got = phi.cpu().numpy()
    assert np.abs(got - phio).max() <= 1e-10 * np.abs(phio).max()


def test_fullsize_pair_injection():
    """Sec. 3.3 injection on the 1024 x 1024 plasma grid (a = 0.99, 16
    particles per cell, 1.7e7 particles; the benchmark times 64 per cell),
    region r_h .. 6 M, multiplicity 3, n0 = 5, in the benchmark's launch
    configuration: every cell's decision against the oracle's (bit-exact),
    the counts, and a sample of 4096 appended pairs (1e-12)."""
    cuda_or_skip()
    F = fpic()
    a = 0.99
    g = I.wald_grid(1024, a)
    d, q, w = I.cell_fill_draws(g, 16, 0.5, seed=3, qm=QM, r_lo=1.02 * I.horizon(1.0, a))
    z = O.seed_fido(1.0, a, d)
    n = z.shape[0]
    w = np.full(n, 1e-6)
    alive = np.ones(n, np.uint8)
    Fw = O.wald_on_grid(a, 1.0, g)
    dr = I.injection_draws(g, 0.5, seed=9)
    C = g.Nr * g.Nth
    cap = n + 2 * C
    r_lo, r_hi = I.horizon(1.0, a), 6.0
    ctx = F.fpic_init_metric(1.0, a)
    F.fpic_set_grid(ctx, g)
    st = F.Particles.empty(cap)
    st.head(n).set_state(torch.as_tensor(z, device="cuda"))
    st.qm[:n].copy_(torch.as_tensor(q, device="cuda"))
    st.w[:n].fill_(1e-6)
    st.alive[:n].fill_(1)
    prm = F.fpic_inject_params(r_lo, r_hi, 3.0, 5.0, QM, 0.0)
    n_g, K_g, f_g = F.fpic_inject_pairs(ctx, st, n, torch.as_tensor(Fw[3], device="cuda"),
                                        torch.as_tensor(Fw[4], device="cuda"), prm,
                                        torch.as_tensor(dr.ravel(), device="cuda"), want_flags=True)
    zo = np.zeros((cap, 6)); zo[:n] = z
    qo = np.zeros(cap); qo[:n] = q
    wo = np.zeros(cap); wo[:n] = w
    ao = np.zeros(cap, np.uint8); ao[:n] = 1
    zo, qo, wo, ao, n_o, K_o, f_o = P.inject_pairs(1.0, a, g, zo, qo, wo, ao, n, cap, Fw[3], Fw[4], r_lo, r_hi,
                                                   3.0, 5.0, QM, dr)
    assert K_g == K_o > 0 and n_g == n_o
    assert np.array_equal(f_g.cpu().numpy(), f_o)
    rng = np.random.default_rng(0)
    ks = rng.choice(K_o, size=min(4096, K_o), replace=False)
    idx = np.sort(np.r_[n + 2 * ks, n + 2 * ks + 1])
    zg = st.state()[torch.as_tensor(idx, device="cuda")].cpu().numpy()
    assert (np.abs(zg - zo[idx]) / (np.abs(zo[idx]) + 1)).max() <= 1e-12
    wg = st.w[torch.as_tensor(idx, device="cuda")].cpu().numpy()
    assert np.allclose(wg, wo[idx], rtol=1e-12, atol=0)
