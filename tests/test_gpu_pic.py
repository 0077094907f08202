"""GPU parity of the grid side (sort, deposit, FDTD) against the oracle."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from oracle import pic as P
from paper_2602_07452_gb300 import inputs as I
from helpers import cuda_or_skip, dev, fpic, make_particles, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    cuda_or_skip()
    return fpic()


def _plasma(g, n, a, seed, dead_frac=0.1):
    d, q, w = I.thermal_draws(n, g, g.rn[0], g.rn[-1], 0.5, seed=seed)
    z = O.seed_fido(1.0, a, d)
    rng = np.random.default_rng(seed)
    w = rng.uniform(0.5, 2.0, n)
    alive = (rng.random(n) > dead_frac).astype(np.uint8)
    return z, q, w, alive


def test_sort_is_the_stable_argsort(F):
    """fpic_sort = stable sort by cell (removed particles last, in order),
    applied to every array; bit-exact."""
    a = 0.9
    g = I.log_grid(37, 29, 1.5, 30.0)
    ctx = F.fpic_init_metric(1.0, a)
    F.fpic_set_grid(ctx, g)
    n = 20011
    z, q, w, alive = _plasma(g, n, a, 3, dead_frac=0.2)
    p = make_particles(z, q, w=w, alive=alive)
    p.Hn.copy_(dev(np.arange(n, dtype=float)))
    F.fpic_sort(ctx, p)
    cell = O.cell_index(g, z[:, 0], z[:, 1]).astype(np.int64)
    key = np.where(alive == 1, cell, g.Nr * g.Nth)
    perm = np.argsort(key, kind="stable")
    zg = p.state().cpu().numpy()
    assert np.array_equal(zg, z[perm])
    assert np.array_equal(p.Hn.cpu().numpy(), perm.astype(float))
    assert np.array_equal(p.alive.cpu().numpy(), alive[perm])
    assert np.array_equal(p.cell.cpu().numpy().view(np.uint32), cell[perm].astype(np.uint32))
    # sorting the sorted set again (every bucket already in index order, the
    # usual case between PIC steps) leaves every array as it is
    F.fpic_sort(ctx, p)
    assert np.array_equal(p.state().cpu().numpy(), z[perm])
    assert np.array_equal(p.Hn.cpu().numpy(), perm.astype(float))
    assert np.array_equal(p.alive.cpu().numpy(), alive[perm])


def test_deposit_permutes_every_array_like_fpic_sort(F):
    """fpic_deposit permutes the particle arrays in two fused passes through
    its record buffer; fpic_sort, one gather and one copy per array: the
    two leave every array (the 11 FP64 ones, alive / scheme / iters, cell)
    bit for bit alike, removed particles last."""
    a = 0.9
    g = I.log_grid(37, 29, 1.5, 30.0)
    ctx = F.fpic_init_metric(1.0, a)
    F.fpic_set_grid(ctx, g)
    n = 30011
    z, q, w, alive = _plasma(g, n, a, 13, dead_frac=0.2)
    rng = np.random.default_rng(14)
    ps = []
    for _ in range(2):
        p = make_particles(z, q, w=w, alive=alive)
        for nm in ("H0", "D0", "Hn"):
            getattr(p, nm).copy_(dev(np.arange(n, dtype=float) * (1 + 0.5 * len(ps))))
        p.scheme.copy_(dev(np.arange(n) % 251, torch.uint8))
        p.iters.copy_(dev((np.arange(n) * 7) % 253, torch.uint8))
        ps.append(p)
    F.fpic_sort(ctx, ps[0])
    F.fpic_deposit(ctx, ps[1], g.size)
    for nm in ("H0", "D0", "Hn"):
        getattr(ps[0], nm).mul_(1.5)
    for nm in ("r", "th", "ph", "ur", "uth", "uph", "qm", "w", "alive", "scheme", "iters", "cell", "H0", "D0", "Hn"):
        a0, a1 = getattr(ps[0], nm).cpu().numpy(), getattr(ps[1], nm).cpu().numpy()
        assert np.array_equal(a0, a1), nm


@pytest.mark.parametrize("lattice", [1, 0])
@pytest.mark.parametrize("a,nr,nth", [(0.0, 48, 40), (0.9, 48, 40), (0.99, 64, 700)])
def test_deposit_matches_oracle(F, a, nr, nth, lattice):
    """Sec. 2.3 deposit on a coarse 48 x 40 grid (th steps beyond the
    series range of the lattice rotations) and a fine 64 x 700 grid (series
    range), 30011 e-/e+ with random weights and 10 % removed: every node of
    rho, j^r, j^th, j^ph within 1e-10 of the oracle (relative to the node's
    sum of |Q W| scale), and bitwise reproducible; with the trapezoid
    lattices in paired FP32 (1, the default) and in FP64 (0)."""
    g = I.log_grid(nr, nth, 1.2 * I.horizon(1.0, a), 25.0)
    ctx = F.fpic_init_metric(1.0, a)
    F.fpic_set_grid(ctx, g)
    assert F.fpic_get_tuning(ctx, F.FPIC_TUNE_DEP_LATTICE) == 1
    F.fpic_set_tuning(ctx, F.FPIC_TUNE_DEP_LATTICE, lattice)
    n = 30011
    z, q, w, alive = _plasma(g, n, a, 5)
    ro = P.deposit(1.0, a, g, z, q, w, alive)
    scale = P.deposit(1.0, a, g, z, np.abs(q), w, alive)[0]     # sum |Q| W / V per node
    p = make_particles(z, q, w=w, alive=alive)
    out = F.fpic_deposit(ctx, p, g.size)
    got = [t.cpu().numpy() for t in out]
    # rho, j^r, j^th, j^ph; |v| <= 1 so |Q v W| <= |Q| W
    sc = np.maximum(scale, scale.max() * 1e-6)
    for k in range(4):
        mask = np.zeros((g.Nr + 1, g.ld), bool)
        mask[: g.Nr + (0 if k == 1 else 1), : g.Nth + (0 if k == 2 else 1)] = True
        m = mask.ravel()
        err = np.abs(got[k] - ro[k])[m]
        print("lattice", lattice, "component", k, "max err / scale %.3e" % (err.max() / sc.max()))
        assert err.max() <= 1e-10 * sc.max(), (k, err.max())
    # determinism: the same particles deposited again give identical bits
    p2 = make_particles(z, q, w=w, alive=alive)
    out2 = F.fpic_deposit(ctx, p2, g.size)
    for x, y in zip(out, out2):
        assert np.array_equal(x.cpu().numpy(), y.cpu().numpy())


def test_deposit_lattice_arithmetic_changes_only_rounding(F):
    """The paired-FP32 and FP64 trapezoid lattices (FPIC_TUNE_DEP_LATTICE)
    evaluate the same points with the same weights: on the 1024^2 grid's
    spacing near the horizon and far out (a = 0.99, 40000 particles) the
    two deposits agree to 5e-12 of the largest node's |Q W| scale (the
    scale the oracle test uses) -- set by the FP64 form's square root
    (2^-39.6 relative; the paired one is 2^-44) -- while the oracle bound is
    1e-10."""
    a = 0.99
    g = I.wald_grid(1024, a)
    ctx = F.fpic_init_metric(1.0, a)
    F.fpic_set_grid(ctx, g)
    rng = np.random.default_rng(17)
    n = 40000
    lo = 1.02 * I.horizon(1.0, a)
    d, q, w = I.thermal_draws(n, g, lo, 49.0, 0.5, seed=17)
    z = O.seed_fido(1.0, a, d)
    w = rng.uniform(0.5, 2.0, n)
    outs = []
    for lattice in (1, 0):
        F.fpic_set_tuning(ctx, F.FPIC_TUNE_DEP_LATTICE, lattice)
        p = make_particles(z, q, w=w)
        outs.append([t.cpu().numpy() for t in F.fpic_deposit(ctx, p, g.size)])
    p = make_particles(z, np.abs(q), w=w)
    sc = F.fpic_deposit(ctx, p, g.size)[0].cpu().numpy().max()
    for k in range(4):
        rel = np.abs(outs[0][k] - outs[1][k]).max() / sc
        print("component", k, "max |paired - FP64| / scale %.3e" % rel)
        assert rel <= 5e-12, (k, rel)


# (r, th) staggering of the components of each field family
STAG = {"B": [(0, 1), (1, 0), (1, 1)], "D": [(1, 0), (0, 1), (0, 0)]}
FAMILY = {"B0": "B", "B1": "B", "Bh": "B", "H": "B", "D0": "D", "D1": "D", "Dw": "D", "E": "D"}


def valid(g, name, k):
    """Mask of the entries a component actually uses (the rest is padding)."""
    ro, to = STAG[FAMILY[name]][k]
    m = np.zeros((g.Nr + 1, g.ld), bool)
    m[: g.Nr + 1 - ro, : g.Nth + 1 - to] = True
    return m.ravel()


def _fill_random(state, fields, g, seed, sources=True):
    rng = np.random.default_rng(seed)
    names = ["B0", "B1", "D0", "D1"] + (["j0", "j1"] if sources else [])
    for nm in names:
        for k in range(3):
            x = rng.normal(size=g.size)
            getattr(state, nm)[k][:] = x
            getattr(fields, nm)[k].copy_(dev(x))
    if sources:
        for nm in ("rho0", "rho1"):
            x = rng.normal(size=g.size)
            setattr(state, nm, x)
            getattr(fields, nm).copy_(dev(x))


@pytest.mark.parametrize("chi0", [0.0, 1e4])
def test_fdtd_step_matches_oracle(F, chi0):
    """Sub-steps 1-4 and 7-10 of Sec. 2.1 on a 40 x 32 grid with random fields
    and sources (absorbing layer on/off): every array within 1e-12 of the
    oracle relative to its magnitude."""
    a = 0.9
    g = I.log_grid(40, 32, 1.5, 30.0)
    ctx = F.fpic_init_metric(1.0, a)
    F.fpic_set_grid(ctx, g)
    st = P.FdtdState(g)
    fl = F.Fields(g.size)
    _fill_random(st, fl, g, 9)
    dt = 0.003
    po = P.FdtdParams(1.0, a, dt, chi0, 5.0, 0.9 * g.rn[-1], g.rn[-1])
    pg = F.fdtd_params(dt, chi0, 5.0, 0.9 * g.rn[-1], g.rn[-1])
    for stage in (1, 2):
        P.fdtd(po, st, stage)
        F.fpic_fdtd_step(ctx, fl, pg, stage)
        for nm in ("B0", "B1", "D0", "D1", "Bh", "Dw", "E", "H"):
            if stage == 1 and nm in ("Dw",):
                continue
            for k in range(3):
                m = valid(g, nm, k)
                exp = getattr(st, nm)[k][m]
                got = getattr(fl, nm)[k].cpu().numpy()[m]
                sc = np.abs(exp).max() + 1e-300
                assert np.abs(got - exp).max() <= 1e-12 * sc, (stage, nm, k, np.abs(got - exp).max() / sc)


@pytest.mark.parametrize("uneven", [False, True])
def test_full_theta_fdtd_step_matches_oracle(F, uneven):
    """The leapfrog in the full-theta domain (fpic_set_theta_mode FULL,
    periodic in th, Sec. 2.5) on a 40 x 64 grid (and on the oracle pins'
    uneven th table) with random fields and sources, two steps: every
    array within 1e-12 of the oracle's full-theta update relative to its
    magnitude, every column Nth the bitwise image of column 0, and the
    seam columns themselves within the bound."""
    import test_oracle_pic as TO
    a = 0.9
    g = (TO._uneven_full_theta_grid if uneven else I.full_theta_grid)(40, 64, 1.5, 30.0)
    ctx = F.fpic_init_metric(1.0, a)
    F.fpic_set_grid(ctx, g)
    st = P.FdtdState(g)
    fl = F.Fields(g.size)
    rng = np.random.default_rng(19)
    for nm in ("B0", "B1", "D0", "D1", "j0", "j1"):
        for k in range(3):
            x = rng.normal(size=(g.Nr + 1, g.ld))
            x[:, g.Nth] = x[:, 0]
            x = x.ravel()
            getattr(st, nm)[k][:] = x
            getattr(fl, nm)[k].copy_(dev(x))
    for nm in ("rho0", "rho1"):
        x = rng.normal(size=(g.Nr + 1, g.ld))
        x[:, g.Nth] = x[:, 0]
        x = x.ravel()
        setattr(st, nm, x)
        getattr(fl, nm).copy_(dev(x))
    dt = 0.002
    po = P.FdtdParams(1.0, a, dt, 1e4, 5.0, 0.9 * g.rn[-1], g.rn[-1], 0, 1)
    pg = F.fdtd_params(dt, 1e4, 5.0, 0.9 * g.rn[-1], g.rn[-1])
    for step in range(2):
        for stage in (1, 2):
            P.fdtd(po, st, stage)
            F.fpic_fdtd_step(ctx, fl, pg, stage)
            for nm in ("B0", "B1", "D0", "D1", "Bh", "Dw", "E", "H"):
                if stage == 1 and nm == "Dw":
                    continue
                for k in range(3):
                    ro, _ = STAG[FAMILY[nm]][k]
                    exp = getattr(st, nm)[k].reshape(g.Nr + 1, g.ld)[: g.Nr + 1 - ro]
                    got = getattr(fl, nm)[k].cpu().numpy().reshape(g.Nr + 1, g.ld)[: g.Nr + 1 - ro]
                    sc = np.abs(exp).max() + 1e-300
                    err = np.abs(got - exp)
                    assert err.max() <= 1e-12 * sc, (step, stage, nm, k, err.max() / sc)
                    assert err[:, [0, g.Nth - 1]].max() <= 1e-12 * sc
                    assert np.array_equal(got[:, g.Nth], got[:, 0]), (step, stage, nm, k)
        st.swap()
        fl.swap()


def test_full_pic_step_matches_oracle(F):
    """One full GRPIC step in the paper's order (Sec. 2.1): FDTD stage 1,
    RK4 push with D^{n+3/2}, B^{n+3/2}, deposit at n+2, FDTD stage 2 --
    particles within 1e-12, fields within 1e-10 of the oracle."""
    a = 0.9
    g = I.log_grid(32, 28, 1.2 * I.horizon(1.0, a), 20.0)
    ctx = F.fpic_init_metric(1.0, a)
    F.fpic_set_grid(ctx, g)
    Fw = O.wald_on_grid(a, 1.0, g)
    st = P.FdtdState(g)
    fl = F.Fields(g.size)
    for k in range(3):
        for nm, src in (("D0", Fw[k]), ("D1", Fw[k]), ("B0", Fw[3 + k]), ("B1", Fw[3 + k])):
            getattr(st, nm)[k][:] = src
            getattr(fl, nm)[k].copy_(dev(src))
    n = 8009
    z, q, w, alive = _plasma(g, n, a, 12, dead_frac=0.0)
    dt = 1e-3
    po = P.FdtdParams(1.0, a, dt, 1e4, 5.0, 0.9 * g.rn[-1], g.rn[-1])
    pg = F.fdtd_params(dt, 1e4, 5.0, 0.9 * g.rn[-1], g.rn[-1])
    # oracle
    P.fdtd(po, st, 1)
    Fpush = [st.D1[0], st.D1[1], st.D1[2], st.Bh[0], st.Bh[1], st.Bh[2]]
    pp = O.push_params(a=a, dt=dt, scheme=O.RK4, field_kind=O.FIELD_GRID, r_max=g.rn[-1])
    zo = np.ascontiguousarray(z.copy()); H0, _, D0 = O.hamiltonian(1.0, a, 0.0, z, q); Hn = H0.copy()
    ao = np.ones(n, np.uint8)
    O.push(pp, zo, q, H0, D0, Hn, ao, g, [np.ascontiguousarray(x) for x in Fpush])
    rho, jr, jt, jp = P.deposit(1.0, a, g, zo, q, w, ao)
    st.j1 = [jr, jt, jp]; st.rho1 = rho
    P.fdtd(po, st, 2)
    # GPU
    p = make_particles(z, q, H0, D0, H0.copy(), w=w)
    F.fpic_fdtd_step(ctx, fl, pg, 1)
    F.fpic_push(ctx, p, fl.push_fields(), F.push_params(dt, scheme=F.FPIC_RK4, r_max=float(g.rn[-1])))
    F.fpic_deposit(ctx, p, g.size, out=(fl.rho1, fl.j1[0], fl.j1[1], fl.j1[2]))
    F.fpic_fdtd_step(ctx, fl, pg, 2)
    # the deposit sorted the GPU particles: compare after sorting the oracle's the same way
    cell = O.cell_index(g, zo[:, 0], zo[:, 1]).astype(np.int64)
    key = np.where(ao == 1, cell, g.Nr * g.Nth)
    perm = np.argsort(key, kind="stable")
    zg = p.state().cpu().numpy()
    err = (np.abs(zg - zo[perm]) / (np.abs(zo[perm]) + 1)).max()
    assert err <= 1e-12, err
    for nm in ("D0", "Dw", "B0", "Bh"):
        for k in range(3):
            m = valid(g, nm, k)
            exp = getattr(st, nm)[k][m]; got = getattr(fl, nm)[k].cpu().numpy()[m]
            assert np.abs(got - exp).max() <= 1e-10 * (np.abs(exp).max() + 1e-300), (nm, k)


def test_split_monopole_field_and_bz_power_match_oracle(F):
    """Sec. 3.4 / App. B.2 field sampled by the library vs the oracle (1e-12
    relative), and Eq. (Pbz) from the auxiliary fields of one FDTD stage vs
    the oracle's quadrature of the same arrays (1e-12 relative)."""
    import torch
    a = 0.9
    g = I.log_grid(48, 64, 1.5, 30.0)
    ctx = F.fpic_init_metric(1.0, a)
    F.fpic_set_grid(ctx, g)
    fo = P.split_monopole_on_grid(1.0, a, 2.0, 1e3, g)
    fd = [torch.zeros(g.size, dtype=torch.float64, device="cuda") for _ in range(6)]
    F.fpic_init_split_monopole(ctx, fd, 2.0, 1e3)
    for k in range(6):
        got = fd[k].cpu().numpy()
        sc = np.abs(fo[k]).max() + 1e-300
        assert np.abs(got - fo[k]).max() <= 1e-12 * sc, k
    # BZ power of random auxiliary fields (the arrays the FDTD leaves in E, H)
    fl = F.Fields(g.size)
    rng = np.random.default_rng(21)
    E = [rng.normal(size=g.size) for _ in range(3)]
    H = [rng.normal(size=g.size) for _ in range(3)]
    for k in range(3):
        fl.E[k].copy_(dev(E[k]))
        fl.H[k].copy_(dev(H[k]))
    for i in (0, 17, g.Nr - 1):
        got = float(F.fpic_bz_power(ctx, fl, i).item())
        ref = P.bz_power(g, E, H, i)
        assert abs(got - ref) <= 1e-12 * (np.pi * 4), (i, got, ref)
    with pytest.raises(F.FpicError):
        F.fpic_bz_power(ctx, fl, g.Nr)


@pytest.mark.parametrize("a,Nr,Nth,n_iter", [(0.9, 48, 64, 0), (0.9, 48, 64, 1), (0.9, 48, 64, 500),
                                             (0.0, 33, 300, 37), (0.99, 20, 513, 200)])
def test_div_clean_matches_oracle(F, a, Nr, Nth, n_iter):
    """Sec. 2.4 (Eq. phi) cleaning of a random D against random rho: the
    corrected D^r, D^th, D^ph and phi agree with the oracle to 1e-10 of
    their scale (grids whose theta rows span one to three blocks of the
    sweep kernel, ragged tails; 0 sweeps is the no-op phi = 0)."""
    import torch
    g = I.log_grid(Nr, Nth, 1.5, 30.0)
    ctx = F.fpic_init_metric(1.0, a)
    F.fpic_set_grid(ctx, g)
    rng = np.random.default_rng(31 + Nr)
    D = [rng.normal(size=g.size) for _ in range(3)]
    rho = rng.normal(size=g.size) * 0.1
    Dd = [dev(x) for x in D]
    phi = F.fpic_div_clean(ctx, Dd, dev(rho), n_iter, want_phi=True)
    torch.cuda.synchronize()
    Dc, phio = P.div_clean(1.0, a, g, D, rho, n_iter)
    sc = max(np.abs(x).max() for x in Dc)
    for k in range(3):
        got = Dd[k].cpu().numpy()
        assert np.abs(got - Dc[k]).max() <= 1e-10 * sc, k
    got = phi.cpu().numpy()
    assert np.abs(got - phio).max() <= 1e-10 * (np.abs(phio).max() + 1e-300)
    # a second cleaning of the same input (the sweep chain replayed) is bitwise identical
    Dd2 = [dev(x) for x in D]
    F.fpic_div_clean(ctx, Dd2, dev(rho), n_iter)
    for k in range(3):
        assert torch.equal(Dd[k], Dd2[k])
    with pytest.raises(F.FpicError):
        F.fpic_div_clean(ctx, Dd, dev(rho), -1)


def _inject_case(g, a, n, seed, dead_frac=0.1):
    """Plasma particles (unit weights, some removed), the Wald B^r, B^th, the
    injection draws, and a multiplicity placing about half of the eligible
    cells below it (calibrated from the particle counts, not from the
    library)."""
    z, q, w, alive = _plasma(g, n, a, seed, dead_frac)
    w = np.ones(n)
    Fw = O.wald_on_grid(a, 1.0, g)
    d = I.injection_draws(g, 0.5, seed=seed + 1)
    return z, q, w, alive, Fw[3], Fw[4], d


def _gpu_store(F, z, q, w, alive, cap):
    import torch
    n = z.shape[0]
    st = F.Particles.empty(cap)
    zz = np.zeros((cap, 6)); zz[:n] = z
    st.set_state(dev(zz))
    for name, x in (("qm", q), ("w", w)):
        v = np.zeros(cap); v[:n] = x
        getattr(st, name).copy_(dev(v))
    al = np.zeros(cap, np.uint8); al[:n] = alive
    st.alive.copy_(torch.as_tensor(al, device="cuda"))
    return st


@pytest.mark.parametrize("a,Nr,Nth,n,extra", [(0.9, 40, 48, 20011, None), (0.99, 33, 70, 5003, 5),
                                              (0.9, 24, 20, 0, None)])
def test_inject_pairs_matches_oracle(F, a, Nr, Nth, n, extra):
    """Sec. 3.3 / 3.4 injection: the per-cell decisions bit-exact (cells
    within 1e-9 of the threshold excluded), the wanted count and the new
    particle count equal, every appended particle's state, q/m, weight,
    H0, D0 within 1e-12 of the oracle (cell order, e- then e+), the cell
    index written, the existing particles untouched; `extra` limits the
    capacity to that many pairs (cell-order truncation)."""
    import torch
    g = I.log_grid(Nr, Nth, 1.2 * I.horizon(1.0, a), 20.0)
    ctx = F.fpic_init_metric(1.0, a)
    F.fpic_set_grid(ctx, g)
    z, q, w, alive, Br, Bt, d = _inject_case(g, a, max(n, 1), 40 + Nr)
    z, q, w, alive = z[:n], q[:n], w[:n], alive[:n]
    r_lo, r_hi, n0, qm_e = I.horizon(1.0, a), 6.0, 5.0, 100.0
    C = g.Nr * g.Nth
    # calibration: weight per new particle at n0 = 1 -> per-cell threshold on sum w |q/m|
    zc, qc, wc, ac, nc, Kc, fc = P.inject_pairs(1.0, a, g, np.zeros((2 * C, 6)), np.zeros(2 * C), np.zeros(2 * C),
                                                np.zeros(2 * C, np.uint8), 0, 2 * C, Br, Bt, r_lo, r_hi, 1e300,
                                                1.0, qm_e, d)
    S = np.zeros(C)
    if n:
        cell = O.cell_index(g, z[:, 0], z[:, 1]).astype(np.int64)
        np.add.at(S, cell[alive == 1], (w * np.abs(q))[alive == 1])
    thr1 = np.zeros(C)
    thr1[np.flatnonzero(fc)] = 2 * qm_e * wc[0:2 * Kc:2]            # = V e n_GJ per cell
    el = thr1 > 0
    ratio = S[el] / thr1[el]
    mult = float(np.median(ratio)) * (1 + 1e-6) if n else 3.0
    cap = n + (2 * C if extra is None else 2 * extra + 1)
    zo, qo, wo, ao, n_o, K_o, f_o = P.inject_pairs(1.0, a, g, np.vstack([z, np.zeros((cap - n, 6))]),
                                                   np.r_[q, np.zeros(cap - n)], np.r_[w, np.zeros(cap - n)],
                                                   np.r_[alive, np.zeros(cap - n, np.uint8)], n, cap, Br, Bt,
                                                   r_lo, r_hi, mult, n0, qm_e, d)
    st = _gpu_store(F, z, q, w, alive, cap)
    prm = F.fpic_inject_params(r_lo, r_hi, mult, n0, qm_e, 0.0)
    n_g, K_g, f_g = F.fpic_inject_pairs(ctx, st, n, dev(Br), dev(Bt), prm, dev(d.ravel()), want_flags=True)
    f_g = f_g.cpu().numpy()
    tie = np.zeros(C, bool)
    tie[el] = np.abs(S[el] / (mult * thr1[el]) - 1) < 1e-9
    assert tie.sum() <= 1
    assert np.array_equal(f_g[~tie], f_o[~tie])
    assert K_g == K_o and n_g == n_o
    if n:
        assert 0 < f_o[el].sum() < el.sum()
    h = st.head(n_g)
    zg = h.state().cpu().numpy()
    assert np.array_equal(zg[:n], z)
    new = slice(n, n_g)
    err = (np.abs(zg[new] - zo[new]) / (np.abs(zo[new]) + 1)).max() if n_g > n else 0.0
    assert err <= 1e-12
    assert np.array_equal(h.qm.cpu().numpy()[new], qo[new])
    assert np.allclose(h.w.cpu().numpy()[new], wo[new], rtol=1e-12, atol=0)
    assert np.all(h.alive.cpu().numpy()[new] == 1)
    H, _, D0 = O.hamiltonian(1.0, a, 0.0, zo[new], qo[new])
    assert np.allclose(h.H0.cpu().numpy()[new], H, rtol=1e-12, atol=1e-14)
    assert np.allclose(h.D0.cpu().numpy()[new], D0, rtol=1e-12, atol=1e-14)
    cells = np.repeat(np.flatnonzero(f_o)[:(n_g - n) // 2], 2)
    assert np.array_equal(h.cell.cpu().numpy()[new].view(np.uint32), cells.astype(np.uint32))
    with pytest.raises(F.FpicError):
        F.fpic_inject_pairs(ctx, st, cap + 1, dev(Br), dev(Bt), prm, dev(d.ravel()))


def _moves_gpu(g, n, seed, frac=0.4):
    rng = np.random.default_rng(seed)
    i = rng.integers(0, g.Nr, n); j = rng.integers(0, g.Nth, n)
    r = g.rn[i] + rng.random(n) * (g.rn[i + 1] - g.rn[i])
    t = g.tn[j] + rng.random(n) * (g.tn[j + 1] - g.tn[j])
    z0 = np.stack([r, t, rng.uniform(0, 6, n), rng.normal(size=n), rng.normal(size=n), rng.normal(size=n)], 1)
    z1 = z0.copy()
    z1[:, 0] += frac * rng.uniform(-1, 1, n) * (g.rn[np.minimum(i + 1, g.Nr)] - g.rn[i])
    z1[:, 1] += frac * rng.uniform(-1, 1, n) * (g.tn[np.minimum(j + 1, g.Nth)] - g.tn[j])
    z1[:, 3:] += 0.1 * rng.normal(size=(n, 3))
    q = np.where(rng.random(n) < 0.5, -1.0, 1.0) * rng.uniform(0.5, 2, n)
    alive = (rng.random(n) > 0.1).astype(np.uint8)
    return z0, z1, q, rng.uniform(0.5, 2, n), alive


@pytest.mark.parametrize("a,Nr,Nth,n", [(0.9, 40, 48, 20011), (0.0, 33, 300, 5003)])
def test_conserving_deposit_matches_oracle(F, a, Nr, Nth, n):
    """Charge-conserving deposit of random moves (up to 0.4 cell, crossing
    nodes, some out of the grid and clamped, 10 % removed): rho and the three
    currents within 1e-10 of the oracle's (relative to each array's scale),
    bitwise reproducible, and the GPU's own output meets the node-wise
    continuity sqrtg d rho + dt Yee-div(sqrtg J) = 0 to rounding."""
    import torch
    g = I.log_grid(Nr, Nth, 1.5, 30.0)
    ctx = F.fpic_init_metric(1.0, a)
    F.fpic_set_grid(ctx, g)
    z0, z1, q, w, alive = _moves_gpu(g, n, 50 + Nr)
    dt = 0.05
    ro = P.deposit_conserving(1.0, a, g, z0, z1, q, w, alive, dt)
    r0o = P.deposit_conserving(1.0, a, g, z0, z0, q, w, alive, dt)[0]
    before = make_particles(z0, q, w=w, alive=alive)
    after = make_particles(z1, q, w=w, alive=alive)
    out, sk = F.fpic_deposit_conserving(ctx, before, after, dt, want_skipped=True)
    assert sk == ro[4] == 0
    got = [t.cpu().numpy() for t in out]
    for k in range(4):
        sc = np.abs(ro[k]).max() + 1e-300
        assert np.abs(got[k] - ro[k]).max() <= 1e-10 * sc, (k, np.abs(got[k] - ro[k]).max() / sc)
    out2 = F.fpic_deposit_conserving(ctx, before, after, dt)
    for x, y in zip(out, out2):
        assert torch.equal(x, y)
    # continuity on the GPU's arrays (interior and boundary nodes)
    rho_b = F.fpic_deposit_conserving(ctx, before, before, dt)[0].cpu().numpy()
    sgn = O.metric(1.0, a, np.repeat(g.rn, g.ld), np.tile(g.tn, g.Nr + 1))[:, 12].reshape(g.Nr + 1, g.ld)
    Jr = got[1].reshape(g.Nr + 1, g.ld); Jt = got[2].reshape(g.Nr + 1, g.ld)
    sr = O.metric(1.0, a, np.repeat(g.rh, g.ld), np.tile(g.tn, g.Nr))[:, 12].reshape(g.Nr, g.ld)
    st_ = O.metric(1.0, a, np.repeat(g.rn, g.Nth), np.tile(g.th, g.Nr + 1))[:, 12].reshape(g.Nr + 1, g.Nth)
    fr = np.zeros((g.Nr + 2, g.ld)); fr[1:g.Nr + 1] = sr * Jr[:g.Nr]
    ft = np.zeros((g.Nr + 1, g.ld + 1)); ft[:, 1:g.Nth + 1] = st_ * Jt[:, :g.Nth]
    drd = np.r_[g.rh, g.rn[-1]] - np.r_[g.rn[0], g.rh]
    dtd = np.r_[g.th, math.pi] - np.r_[0.0, g.th]
    div = (fr[1:] - fr[:-1]) / drd[:, None] + (ft[:, 1:] - ft[:, :-1]) / dtd[None, :]
    lhs = sgn * (got[0] - rho_b).reshape(g.Nr + 1, g.ld)
    assert np.abs(lhs + dt * div).max() <= 1e-13 * np.abs(lhs).max()


def test_conserving_pic_loop_matches_oracle(F):
    """Six steps of the GRPIC loop with the conserving deposit and the
    conserving FDTD mode (RK4 push, no absorbing layer): D^{n+1/2} after the
    run within 1e-10 of the oracle's loop, and the GPU's Gauss residual
    Yee-div(sqrtg D) - 4 pi sqrtg rho unchanged at the interior nodes."""
    import torch
    a = 0.9
    g = I.log_grid(24, 20, 1.5, 20.0)
    ctx = F.fpic_init_metric(1.0, a)
    F.fpic_set_grid(ctx, g)
    n = 3000
    rng = np.random.default_rng(4)
    d, q, _ = I.thermal_draws(n, g, 3.0, 12.0, 0.3, seed=5, qm=50.0)
    d[:, 1] = rng.uniform(0.5, math.pi - 0.5, n)
    z = O.seed_fido(1.0, a, d)
    w = np.full(n, 1e-3)
    Fw = O.wald_on_grid(a, 1.0, g)
    dt = 2e-3
    # oracle loop
    st = P.FdtdState(g)
    for k in range(3):
        st.D0[k][:] = Fw[k]; st.D1[k][:] = Fw[k]; st.B0[k][:] = Fw[3 + k]; st.B1[k][:] = Fw[3 + k]
    po = P.FdtdParams(1.0, a, dt, 0.0, 5.0, g.rn[-1], g.rn[-1], 1)
    al = np.ones(n, np.uint8)
    st.rho1 = P.deposit_conserving(1.0, a, g, z, z, q, w, al, dt)[0]
    H0, _, D0 = O.hamiltonian(1.0, a, 0.0, z, q)
    pp = O.push_params(a=a, dt=dt, scheme=O.RK4, field_kind=O.FIELD_GRID, r_max=g.rn[-1])
    zo = z.copy()
    # GPU loop
    fl = F.Fields(g.size)
    for k in range(3):
        for nm, src in (("D0", Fw[k]), ("D1", Fw[k]), ("B0", Fw[3 + k]), ("B1", Fw[3 + k])):
            getattr(fl, nm)[k].copy_(dev(src))
    p = make_particles(z, q, H0, D0, H0.copy(), w=w)
    prev = make_particles(z, q, H0, D0, H0.copy(), w=w)
    F.fpic_deposit_conserving(ctx, p, p, dt, out=(fl.rho1, fl.j1[0], fl.j1[1], fl.j1[2]))
    pg = F.fdtd_params(dt, 0.0, 5.0, g.rn[-1], g.rn[-1], conserving=True)
    pprm = F.push_params(dt, scheme=F.FPIC_RK4, r_max=float(g.rn[-1]))
    sel = np.zeros((g.Nr + 1, g.ld), bool)
    sel[2:g.Nr - 1, 2:g.Nth - 1] = True
    sg = O.metric(1.0, a, np.repeat(g.rn, g.ld), np.tile(g.tn, g.Nr + 1))[:, 12]

    def resid(D, rho_):
        _, dD = P.div(1.0, a, g, [np.zeros(g.size)] * 3, D)
        return (dD - 4 * math.pi * sg * rho_).reshape(g.Nr + 1, g.ld)[sel]

    R0 = resid([x.cpu().numpy() for x in fl.D1], fl.rho1.cpu().numpy())
    for step in range(6):
        P.fdtd(po, st, 1)
        zold = zo.copy()
        O.push(pp, zo, q, H0, D0, H0.copy(), al, g, [st.D1[0], st.D1[1], st.D1[2], st.Bh[0], st.Bh[1], st.Bh[2]])
        rho, Jr, Jt, Jp, _ = P.deposit_conserving(1.0, a, g, zold, zo, q, w, np.ones(n, np.uint8), dt)
        st.j1 = [Jr, Jt, Jp]; st.rho1 = rho
        P.fdtd(po, st, 2)
        st.swap()
        F.fpic_fdtd_step(ctx, fl, pg, 1)
        for nm in ("r", "th", "ph", "ur", "uth", "uph", "alive"):
            getattr(prev, nm).copy_(getattr(p, nm))
        F.fpic_push(ctx, p, fl.push_fields(), pprm)
        F.fpic_deposit_conserving(ctx, prev, p, dt, out=(fl.rho1, fl.j1[0], fl.j1[1], fl.j1[2]))
        F.fpic_fdtd_step(ctx, fl, pg, 2)
        fl.swap()
    Dg = [x.cpu().numpy() for x in fl.D1]
    for k in range(3):
        m = valid(g, "D0", k)
        sc = np.abs(st.D1[k][m]).max()
        assert np.abs(Dg[k][m] - st.D1[k][m]).max() <= 1e-10 * sc, k
    R = resid(Dg, fl.rho0.cpu().numpy())
    scale = np.abs(4 * math.pi * sg.reshape(g.Nr + 1, g.ld)[sel] * fl.rho0.cpu().numpy().reshape(g.Nr + 1, g.ld)[sel]).max()
    assert np.abs(R - R0).max() <= 1e-11 * scale


def test_deposit_thread_tuning_changes_no_result(F):
    """FPIC_TUNE_DEP_THREADS only reshapes the deposit's per-particle launch:
    rho and the currents are bitwise the same for 64, 128 and 256 threads per
    block; other values are rejected; the autotuner leaves a valid choice."""
    import torch
    from paper_2602_07452_gb300 import autotune
    a = 0.9
    g = I.log_grid(40, 32, 1.2 * I.horizon(1.0, a), 25.0)
    ctx = F.fpic_init_metric(1.0, a)
    F.fpic_set_grid(ctx, g)
    z, q, w, alive = _plasma(g, 30011, a, 8)
    outs = []
    for v in (64, 128, 256):
        F.fpic_set_tuning(ctx, F.FPIC_TUNE_DEP_THREADS, v)
        p = make_particles(z, q, w=w, alive=alive)
        outs.append([t.cpu().numpy() for t in F.fpic_deposit(ctx, p, g.size)])
    for o in outs[1:]:
        for x, y in zip(outs[0], o):
            assert np.array_equal(x, y)
    with pytest.raises(F.FpicError):
        F.fpic_set_tuning(ctx, F.FPIC_TUNE_DEP_THREADS, 96)
    p = make_particles(z, q, w=w, alive=alive)
    times = autotune.tune_deposit_threads(ctx, p, g.size, reps=1)
    assert set(times) == {64, 128, 256}
    assert F.fpic_get_tuning(ctx, F.FPIC_TUNE_DEP_THREADS) == min(times, key=times.get)


def test_new_grid_entry_points_edge_cases(F):
    """Degenerate inputs of the grid-side extensions: an empty particle set
    deposits zeros (conserving deposit) and injects into every eligible cell
    of an empty store; a store without room injects nothing but still counts
    the wanted pairs; the cleaning runs on the smallest grid (2 x 2) and on
    zero sweeps leaves D unchanged when rho matches div D; a zero-length
    move is a rest (no current)."""
    import torch
    a = 0.9
    g = I.log_grid(6, 5, 1.5, 10.0)
    ctx = F.fpic_init_metric(1.0, a)
    F.fpic_set_grid(ctx, g)
    empty = make_particles(np.zeros((0, 6)), np.zeros(0))
    rho, jr, jt, jp = F.fpic_deposit_conserving(ctx, empty, empty, 0.1)
    assert not rho.any() and not jr.any() and not jt.any() and not jp.any()
    Br = dev(np.full(g.size, 1.0)); Bt = dev(np.zeros(g.size))
    d = dev(I.injection_draws(g, 0.5, seed=1).ravel())
    prm = F.fpic_inject_params(0.0, 1e9, 3.0, 5.0, 10.0, 0.0)
    st = F.Particles.empty(2 * g.Nr * g.Nth)
    n_new, K, fl = F.fpic_inject_pairs(ctx, st, 0, Br, Bt, prm, d, want_flags=True)
    assert K == int(fl.sum().item()) > 0 and n_new == 2 * K
    full = F.Particles.empty(5)
    n2, K2, _ = F.fpic_inject_pairs(ctx, full, 5, Br, Bt, prm, d)
    assert n2 == 5 and K2 == K
    z = np.array([[2.5, 1.0, 0.0, 0.1, 0.0, 0.5]])
    p = make_particles(z, np.array([1.0]))
    _, jr, jt, jp = F.fpic_deposit_conserving(ctx, p, p, 0.1)
    assert not jr.any() and not jt.any()
    g2 = I.log_grid(2, 2, 1.5, 10.0)
    ctx2 = F.fpic_init_metric(1.0, a)
    F.fpic_set_grid(ctx2, g2)
    D = [dev(np.random.default_rng(0).normal(size=g2.size)) for _ in range(3)]
    D0 = [x.clone() for x in D]
    rho2 = dev(np.zeros(g2.size))
    F.fpic_div_clean(ctx2, D, rho2, 10)
    Dc, _ = P.div_clean(1.0, a, g2, [x.cpu().numpy() for x in D0], np.zeros(g2.size), 10)
    for k in range(3):
        assert np.abs(D[k].cpu().numpy() - Dc[k]).max() <= 1e-12 * (np.abs(Dc[k]).max() + 1e-300)
    D = [x.clone() for x in D0]
    F.fpic_div_clean(ctx2, D, rho2, 0)
    Dc0, _ = P.div_clean(1.0, a, g2, [x.cpu().numpy() for x in D0], np.zeros(g2.size), 0)
    for k in range(3):
        assert np.abs(D[k].cpu().numpy() - Dc0[k]).max() <= 1e-12 * (np.abs(Dc0[k]).max() + 1e-300)


def test_grpic_conserving_loop_with_injection_keeps_gauss(F):
    """The GRPIC sequencer (grpic.py) with the conserving deposit, the FDTD in
    its conserving mode and pair injection every other step: the injected
    pairs are neutral at one point, so Yee-div(sqrtg D) - 4 pi sqrtg rho at
    the interior nodes stays what it was, over 6 steps, while the particle
    count grows."""
    from paper_2602_07452_gb300.grpic import GRPIC
    a = 0.9
    g = I.log_grid(24, 20, 1.5, 20.0)
    ctx = F.fpic_init_metric(1.0, a)
    F.fpic_set_grid(ctx, g)
    n = 3000
    rng = np.random.default_rng(4)
    d, q, _ = I.thermal_draws(n, g, 3.0, 12.0, 0.3, seed=5, qm=50.0)
    d[:, 1] = rng.uniform(0.5, math.pi - 0.5, n)
    z = O.seed_fido(1.0, a, d)
    Fw = O.wald_on_grid(a, 1.0, g)
    fl = F.Fields(g.size)
    for k in range(3):
        for nm, src in (("D0", Fw[k]), ("D1", Fw[k]), ("B0", Fw[3 + k]), ("B1", Fw[3 + k])):
            getattr(fl, nm)[k].copy_(dev(src))
    cap = n + 4 * g.Nr * g.Nth
    store = F.Particles.empty(cap)
    head = store.head(n)
    head.set_state(dev(z)); head.qm.copy_(dev(q)); head.w.fill_(1e-3); head.alive.fill_(1)
    dt = 2e-3
    inj = (2, F.fpic_inject_params(3.5, 8.0, 1e30, 0.05, 50.0, 0.0), dev(I.injection_draws(g, 0.3, seed=7).ravel()))
    sim = GRPIC(ctx, g, fl, store, n, F.push_params(dt, scheme=F.FPIC_RK4, r_max=float(g.rn[-1])),
                F.fdtd_params(dt, 0.0, 5.0, g.rn[-1], g.rn[-1]), conserving=True, inject=inj)
    sim.deposit_initial()
    sel = np.zeros((g.Nr + 1, g.ld), bool)
    sel[2:g.Nr - 1, 2:g.Nth - 1] = True
    sg = O.metric(1.0, a, np.repeat(g.rn, g.ld), np.tile(g.tn, g.Nr + 1))[:, 12]

    def resid():
        _, dD = P.div(1.0, a, g, [np.zeros(g.size)] * 3, [x.cpu().numpy() for x in fl.D1])
        return (dD - 4 * math.pi * sg * fl.rho1.cpu().numpy()).reshape(g.Nr + 1, g.ld)[sel]

    R0 = resid()
    scale = np.abs(4 * math.pi * sg.reshape(g.Nr + 1, g.ld)[sel] * fl.rho1.cpu().numpy().reshape(g.Nr + 1, g.ld)[sel]).max()
    for _ in range(6):
        sim.step()
        # after the swap the step's sources sit in the "0" slot: pair D1 with rho0
        _, dD = P.div(1.0, a, g, [np.zeros(g.size)] * 3, [x.cpu().numpy() for x in fl.D1])
        R = (dD - 4 * math.pi * sg * fl.rho0.cpu().numpy()).reshape(g.Nr + 1, g.ld)[sel]
        assert np.abs(R - R0).max() <= 1e-11 * scale
    assert sim.n > n and sim.pairs > 0
