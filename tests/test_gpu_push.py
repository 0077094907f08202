"""GPU parity of the push path against the oracle, element by element, on the
same seeded inputs, through the C ABI.

Bar (per step from an identical state): |z_gpu - z_oracle| <= 1e-12 (|z| + 1)
per component; cell indices and plain-path scheme choices bit-exact (except
states within 1e-12 relative of a node or of the threshold, counted)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2602_07452_gb300 import inputs as I
from helpers import (assert_state_close, cuda_or_skip, dev, fields_dev, fpic, make_particles,
                     thermal_state, to_np)

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
TOL = 1e-12


@pytest.fixture(scope="module")
def F():
    cuda_or_skip()
    return fpic()


def _ctx(F, a, g=None):
    ctx = F.fpic_init_metric(1.0, a)
    if g is not None:
        F.fpic_set_grid(ctx, g)
    return ctx


@pytest.fixture(scope="module")
def wald128(F):
    a = 0.9
    g = I.wald_grid(128, a, r_max=50.0)
    Fo = O.wald_on_grid(a, 1.0, g)
    ctx = _ctx(F, a, g)
    return a, g, Fo, ctx


def test_wald_on_grid_matches_oracle(F, wald128):
    a, g, Fo, ctx = wald128
    Fg = [dev(np.zeros_like(f)) for f in Fo]
    F.fpic_init_wald(ctx, Fg, 1.0)
    for k in range(6):
        got = Fg[k].cpu().numpy()
        scale = np.abs(Fo[k]).max()
        assert np.abs(got - Fo[k]).max() <= 1e-13 * scale, k


def test_hamiltonian_matches_oracle(F, wald128):
    a, g, Fo, ctx = wald128
    d, z, q = thermal_state(3001, g, a)
    p = make_particles(z, q)
    H, L = F.fpic_hamiltonian(ctx, p, B0pot=1.0)
    Ho, Lo, _ = O.hamiltonian(1.0, a, 1.0, z, q)
    assert np.abs(H.cpu().numpy() - Ho).max() <= 1e-13 * (np.abs(Ho).max())
    assert np.abs(L.cpu().numpy() - Lo).max() <= 1e-13 * (np.abs(Lo).max())


def test_cell_index_bit_exact(F, wald128):
    a, g, Fo, ctx = wald128
    rng = np.random.default_rng(7)
    r = np.concatenate([rng.uniform(g.rn[0] * 0.5, g.rn[-1] * 1.5, 5000), g.rn,
                        np.nextafter(g.rn, 0), np.nextafter(g.rn, 1e9)])
    t = np.concatenate([rng.uniform(-0.2, math.pi + 0.2, 5000), rng.choice(g.tn, 3 * g.rn.size)])
    t[5000:5000 + g.tn.size] = g.tn
    z = np.zeros((r.size, 6)); z[:, 0] = r; z[:, 1] = t
    p = make_particles(z, np.zeros(r.size))
    got = F.fpic_cell_index(ctx, p).cpu().numpy().view(np.uint32)
    assert np.array_equal(got, O.cell_index(g, r, t))


def test_seeding_matches_oracle(F):
    a = 0.9
    ctx = _ctx(F, a)
    cand = I.orbit_candidates(777, seed=1)
    zo, bad = O.seed_orbits(1.0, a, cand)
    p = make_particles(np.zeros((777, 6)), np.zeros(777))
    F.fpic_init_particles(ctx, p, F.FPIC_SEED_ORBIT, dev(cand), K=cand.shape[1])
    zg = p.state().cpu().numpy()
    assert bad == 0 and p.alive.cpu().numpy().all()
    assert_state_close(zg, zo, 1e-13)
    H0 = O.hamiltonian(1.0, a, 0.0, zo, 0.0)
    assert np.abs(p.H0.cpu().numpy() - H0[0]).max() < 1e-14
    g = I.wald_grid(64, a)
    d, q, w = I.thermal_draws(1001, g, 1.5, 40.0, 0.1, seed=5)
    zo = O.seed_fido(1.0, a, d)
    p = make_particles(np.zeros((1001, 6)), q)
    F.fpic_init_particles(ctx, p, F.FPIC_SEED_FIDO, dev(d), B0pot=1.0)
    assert_state_close(p.state().cpu().numpy(), zo, 1e-13)
    Ho, _, Do = O.hamiltonian(1.0, a, 1.0, zo, q)
    assert np.abs(p.H0.cpu().numpy() - Ho).max() <= 1e-13 * np.abs(Ho).max()
    assert np.abs(p.D0.cpu().numpy() - Do).max() <= 1e-13 * np.abs(Do).max()


def _one_step(F, ctx, g, Fo, z, q, scheme, dt, thr=1e-12, implicit=None, B0pot=1.0, r_max=None,
              max_iter=50, alive=None, tol=1e-14, dt_imp=0.0, t=None, newton=False):
    n = z.shape[0]
    H0, _, D0 = O.hamiltonian(1.0, _A[id(ctx)], B0pot, z, q)
    Hn = H0 * (1.0 + 1e-9 * np.cos(np.arange(n)))
    implicit = implicit if implicit is not None else F.FPIC_IMR
    r_max = r_max if r_max is not None else (g.rn[-1] if g is not None else 1e300)
    alive = np.ones(n, np.uint8) if alive is None else alive
    p = make_particles(z, q, H0, D0, Hn, alive)
    prm = F.push_params(dt, scheme=scheme, implicit=implicit, thr=thr, tol=tol, max_iter=max_iter,
                        r_max=r_max, B0pot=B0pot, dt_implicit=dt_imp, t=t, imr_newton=newton)
    st = F.fpic_push(ctx, p, fields_dev(Fo) if Fo is not None else None, prm, stats=True)
    po = O.push_params(a=_A[id(ctx)], dt=dt, scheme=scheme, implicit_kind=implicit, thr=thr, tol=tol,
                       max_iter=max_iter, r_max=r_max, B0pot=B0pot, dt_imp=dt_imp, imr_newton=newton,
                       field_kind=O.FIELD_GRID if Fo is not None else O.FIELD_NONE)
    zo = np.ascontiguousarray(z.copy()); Ho = Hn.copy(); ao = alive.copy()
    nc, so, io = O.push(po, zo, q, H0, D0, Ho, ao, g, Fo)
    return p, st, (zo, Ho, ao, so, io, nc), (H0, D0, Hn)


_A = {}


def _check_iterations(ig, io, newton):
    """Implicit iteration counts, GPU against oracle.  Fixed-point form: the
    same successive-update stop on both sides, so the counts agree except
    where the last update sits at the tolerance within rounding (at most
    1 % of the solves, by one iteration).  Newton form: the kernel also
    stops when its a-posteriori bound passes the tolerance, which the
    oracle does not use; it stops no later than the oracle (up to the same
    rounding) and usually one iteration earlier."""
    d = io.astype(int) - ig.astype(int)
    if not newton:
        assert np.abs(d).max() <= 1 and (d != 0).mean() <= 0.01, (np.abs(d).max(), (d != 0).mean())
    else:
        assert d.min() >= -1 and d.max() <= 2 and (d < 0).mean() <= 0.01, (d.min(), d.max(), (d < 0).mean())
        assert d.mean() > 0.3, d.mean()


def _mk(F, a, g=None):
    ctx = _ctx(F, a, g)
    _A[id(ctx)] = a
    return ctx


@pytest.mark.parametrize("scheme,newton", [("RK4", False), ("IMR", False), ("HYB1", False), ("HYB2", False),
                                           ("IMR", True), ("HYB1", True), ("HYB2", True)])
def test_charged_push_one_step_matches_oracle(F, scheme, newton):
    """Wald field on a 128 x 128 (ln r, th) grid, e-/e+ q/m = -/+100,
    4741 particles (37 blocks of 128 plus a ragged tail), dt = 1e-3; the
    IMR solved by the fixed-point update or by the Newton iteration
    (imr_newton) on both sides."""
    a = 0.9
    g = I.wald_grid(128, a)
    Fo = O.wald_on_grid(a, 1.0, g)
    ctx = _mk(F, a, g)
    d, z, q = thermal_state(4741, g, a, theta=0.1, seed=11)
    sch = getattr(F, "FPIC_" + scheme)
    thr = {"HYB1": 8e-5, "HYB2": 8e-8}.get(scheme, 1e-12)
    p, st, (zo, Ho, ao, so, io, nc), (H0, D0, Hn) = _one_step(F, ctx, g, Fo, z, q, sch, 1e-3, thr=thr,
                                                             newton=newton)
    zg, Hg, ag, sg, ig, cg = to_np(p)
    assert np.array_equal(ag, ao)
    if newton:
        assert io[so == 1].mean() < 6.0
    if scheme.startswith("HYB"):
        # exclude particles whose test statistic lies within 1e-12 of the threshold
        pr = O.push_params(a=a, dt=1e-3, scheme=O.RK4, B0pot=1.0, field_kind=O.FIELD_GRID, r_max=g.rn[-1])
        zr = np.ascontiguousarray(z.copy()); Hr = Hn.copy()
        O.push(pr, zr, q, H0, D0, Hr, np.ones(len(q), np.uint8), g, Fo)
        Ht1 = np.abs(Hr - H0) / D0
        stat = Ht1 if scheme == "HYB2" else (Ht1 - np.abs(Hn - H0) / D0) / 1e-3
        near = np.abs(stat - thr) <= 1e-12 * abs(thr) + 1e-12 * np.abs(stat)
        assert near.sum() <= 2
        assert np.array_equal(sg[~near], so[~near])
        frac = so.mean()
        assert 0.02 < frac < 0.8, frac
        assert st["n_implicit"] == int(so.sum())
        ok = ~near
    else:
        ok = np.ones(len(q), bool)
        assert np.array_equal(sg, so)
    assert_state_close(zg, zo, TOL, ok)
    assert np.abs(Hg - Ho)[ok].max() <= 1e-12 * np.abs(Ho).max()
    # cells bit-exact except states within 1e-12 of a node
    rel = np.minimum(np.abs(zo[:, 0, None] / g.rn[None, :] - 1).min(1),
                     np.abs(zo[:, 1, None] - g.tn[None, :]).min(1))
    cell_o = O.cell_index(g, zo[:, 0], zo[:, 1])
    far = rel > 1e-11
    assert np.array_equal(cg[far & (ao == 1)], cell_o[far & (ao == 1)])
    if scheme in ("IMR",) or scheme.startswith("HYB"):
        _check_iterations(ig[so == 1], io[so == 1], newton)


@pytest.mark.parametrize("scheme", ["RK4", "HAM", "HYB2"])
def test_neutral_push_one_step_matches_oracle(F, scheme):
    """Geodesics (no fields), bound-orbit seeds, a = 0.9, dt = 0.5 and 1.0;
    hybrid partner = the discrete-gradient scheme.  Every step within 1e-12
    (the quotients are taken in closed form, so the discrete-gradient solve
    converges to the tolerance on both sides)."""
    a = 0.9
    ctx = _mk(F, a)
    cand = I.orbit_candidates(1000, seed=3)
    z, bad = O.seed_orbits(1.0, a, cand)
    q = np.zeros(len(z))
    H0 = O.hamiltonian(1.0, a, 0.0, z, q)[0]
    for dt in (0.5, 1.0):
        sch = getattr(F, "FPIC_" + scheme)
        pr = O.push_params(a=a, dt=dt, scheme=O.RK4)
        zr = np.ascontiguousarray(z.copy()); Hr = H0.copy()
        O.push(pr, zr, q, H0, H0, Hr, np.ones(len(q), np.uint8))
        stat = np.abs(Hr - H0) / H0
        thr = float(np.median(stat))
        p, st, (zo, Ho, ao, so, io, nc), _ = _one_step(F, ctx, None, None, z, q, sch, dt, thr=thr,
                                                      implicit=F.FPIC_HAM, B0pot=0.0, tol=1e-15)
        zg, Hg, ag, sg, ig, cg = to_np(p)
        near = np.abs(stat - thr) <= 1e-10 * thr + 1e-15
        if scheme == "HYB2":
            assert near.sum() <= 10
            assert np.array_equal(sg[~near], so[~near])
            assert 0 < so.sum() < len(q)
        else:
            near[:] = False
            assert np.array_equal(sg, so)
        bound = np.full(len(q), TOL)
        err = (np.abs(zg - zo) / (np.abs(zo) + 1.0)).max(axis=1)
        assert np.all(err[~near] <= bound[~near]), (err / bound).max()
        if scheme == "HAM":
            assert np.abs(Hg - H0).max() < 2e-14


def test_removal_reflection_and_edges(F):
    """Boundaries: particles falling through r_+ or crossing r_max are removed,
    pole crossings reflect; particles outside the grid use the clamped gather;
    dead particles are left untouched; n = 0 is a no-op."""
    a = 0.5
    g = I.log_grid(40, 30, 1.0, 20.0)
    Fo = O.wald_on_grid(a, 1.0, g)
    ctx = _mk(F, a, g)
    z = np.array([[1.9, 0.3, 0.0, -3.0, 0.0, 0.0],
                  [6.0, 0.002, 0.0, 0.0, -2.0, 0.0],
                  [19.99, 1.0, 0.0, 5.0, 0.0, 0.0],
                  [8.0, 0.01, 0.0, 0.1, 0.3, 0.2],        # between the pole and the first node
                  [7.0, 1.0, 0.0, 0.1, 0.1, 0.1]])
    q = np.array([0.0, 0.0, 1.0, 10.0, -10.0])
    alive = np.array([1, 1, 1, 1, 0], np.uint8)
    p, st, (zo, Ho, ao, so, io, nc), _ = _one_step(F, ctx, g, Fo, z, q, F.FPIC_RK4, 0.1, r_max=20.0,
                                                  alive=alive)
    zg, Hg, ag, sg, ig, cg = to_np(p)
    assert ag.tolist() == [0, 1, 0, 1, 0] == ao.tolist()
    assert_state_close(zg, zo, TOL)
    assert np.array_equal(zg[4], z[4])
    assert st["n_removed"] == 2 and st["n_alive_before"] == 4
    p0 = make_particles(np.zeros((0, 6)), np.zeros(0))
    assert F.fpic_push(ctx, p0, None, F.push_params(0.1), stats=True)["n_alive_before"] == 0


def test_iteration_cap_is_reported(F):
    """An implicit solve stopped by max_iter is counted (FPIC_ENOTCONVERGED),
    and the state equals the oracle's capped iterate."""
    a = 0.9
    g = I.wald_grid(64, a)
    Fo = O.wald_on_grid(a, 1.0, g)
    ctx = _mk(F, a, g)
    d, z, q = thermal_state(300, g, a, seed=4)
    p, st, (zo, Ho, ao, so, io, nc), _ = _one_step(F, ctx, g, Fo, z, q, F.FPIC_IMR, 1e-3, max_iter=2)
    assert st["n_notconv"] == nc > 0
    assert_state_close(to_np(p)[0], zo, TOL)


def test_invalid_arguments_raise(F):
    ctx = _mk(F, 0.9)
    p = make_particles(np.ones((3, 6)), np.zeros(3))
    with pytest.raises(F.FpicError):
        F.fpic_push(ctx, p, None, F.push_params(float("nan")))
    with pytest.raises(F.FpicError):
        F.fpic_push(ctx, p, None, F.push_params(0.1, scheme=9))
    with pytest.raises(F.FpicError):
        F.fpic_push(ctx, p, None, F.push_params(0.1, max_iter=0))
    with pytest.raises(F.FpicError):
        F.fpic_init_metric(1.0, 1.5)
    with pytest.raises(F.FpicError):
        F.fpic_cell_index(ctx, p)   # no grid


@pytest.mark.parametrize("newton", [False, True])
def test_full_size_charged_workload_sampled(F, newton):
    """Charged Wald workload at full size (512 x 512 grid, 2^20 particles,
    hybrid RK4 <-> IMR, dt = 1e-3) in the launch configuration the benchmark
    times (IMR by the fixed-point update and by the Newton iteration); 3000
    sampled particles are recomputed by the oracle."""
    a = 0.9
    n = 1 << 20
    g = I.wald_grid(512, a)
    ctx = _mk(F, a, g)
    Fg = [dev(np.zeros(g.size)) for _ in range(6)]
    F.fpic_init_wald(ctx, Fg, 1.0)
    d, q, w = I.thermal_draws(n, g, 1.02 * I.horizon(1.0, a), 49.0, 0.1, seed=2)
    p = make_particles(np.zeros((n, 6)), q)
    F.fpic_init_particles(ctx, p, F.FPIC_SEED_FIDO, dev(d), B0pot=1.0)
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(n, 3000, replace=False))
    z0 = p.state().cpu().numpy()[idx]
    H0 = p.H0.cpu().numpy()[idx]; D0 = p.D0.cpu().numpy()[idx]; Hn = p.Hn.cpu().numpy()[idx]
    thr = 5e-6
    prm = F.push_params(1e-3, scheme=F.FPIC_HYB1, implicit=F.FPIC_IMR, thr=thr, r_max=g.rn[-1], B0pot=1.0,
                        imr_newton=newton)
    st = F.fpic_push(ctx, p, Fg, prm, stats=True)
    zg, Hg, ag, sg, ig, cg = to_np(p)
    Fo = [f.cpu().numpy() for f in Fg]
    po = O.push_params(a=a, dt=1e-3, scheme=O.HYB1, implicit_kind=O.IMR, thr=thr, r_max=g.rn[-1],
                       B0pot=1.0, field_kind=O.FIELD_GRID, imr_newton=newton)
    zo = np.ascontiguousarray(z0.copy()); Ho = Hn.copy(); ao = np.ones(len(idx), np.uint8)
    O.push(po, zo, q[idx], H0, D0, Ho, ao, g, Fo)
    assert_state_close(zg[idx], zo, TOL)
    assert st["n_alive_before"] == n


@pytest.mark.parametrize("newton", [False, True])
def test_imr_launch_shape_changes_no_result(newton):
    """FPIC_TUNE_IMR_BLOCKS_PER_SM only reshapes the persistent implicit
    launch: every particle's step is bitwise the same for 1 and 4 resident
    blocks per SM (either IMR iteration); out-of-range values are rejected."""
    cuda_or_skip()
    F = fpic()
    a = 0.9
    g = I.wald_grid(96, a)
    Fo = O.wald_on_grid(a, 1.0, g)
    ctx = F.fpic_init_metric(1.0, a)
    F.fpic_set_grid(ctx, g)
    d, z, q = thermal_state(20000, g, a, theta=0.1, seed=12)
    H0, _, D0 = O.hamiltonian(1.0, a, 1.0, z, q)
    prm = F.push_params(1e-3, scheme=F.FPIC_HYB1, implicit=F.FPIC_IMR, thr=8e-5, r_max=float(g.rn[-1]),
                        B0pot=1.0, imr_newton=newton)
    outs = []
    for v in (1, 4):
        F.fpic_set_tuning(ctx, F.FPIC_TUNE_IMR_BLOCKS_PER_SM, v)
        assert F.fpic_get_tuning(ctx, F.FPIC_TUNE_IMR_BLOCKS_PER_SM) == v
        p = make_particles(z, q, H0, D0, H0.copy())
        st = F.fpic_push(ctx, p, fields_dev(Fo), prm, stats=True)
        assert st["n_implicit"] > 100
        outs.append(to_np(p))
    for x, y in zip(*outs):
        assert np.array_equal(x, y)
    for bad in (0, 5):
        with pytest.raises(F.FpicError):
            F.fpic_set_tuning(ctx, F.FPIC_TUNE_IMR_BLOCKS_PER_SM, bad)


@pytest.mark.parametrize("n", [0, 3, 20011])
@pytest.mark.parametrize("pinned,staging", [(True, 0), (True, 1), (False, 0)])
def test_host_buffer_push_equals_device_push(n, pinned, staging):
    """fpic_push_host gives bitwise the device push's results, for ragged
    chunk sizes and removed particles, on pinned host arrays (read and
    written in place by the kernels, or DMA-staged with
    FPIC_TUNE_HOST_STAGING) and on pageable ones (chunked copies
    overlapping the explicit pass); the host arrays hold the result
    afterwards."""
    cuda_or_skip()
    F = fpic()
    a = 0.9
    g = I.wald_grid(96, a)
    Fo = O.wald_on_grid(a, 1.0, g)
    ctx = F.fpic_init_metric(1.0, a)
    F.fpic_set_grid(ctx, g)
    F.fpic_set_tuning(ctx, F.FPIC_TUNE_HOST_STAGING, staging)
    prm = F.push_params(1e-3, scheme=F.FPIC_HYB1, implicit=F.FPIC_IMR, thr=8e-5, r_max=float(g.rn[-1]),
                        B0pot=1.0)
    if n:
        d, z, q = thermal_state(n, g, a, theta=0.1, seed=13)
        H0, _, D0 = O.hamiltonian(1.0, a, 1.0, z, q)
    else:
        z, q, H0, D0 = np.zeros((0, 6)), np.zeros(0), np.zeros(0), np.zeros(0)
    alive = (np.arange(n) % 7 != 3).astype(np.uint8)
    p = make_particles(z, q, H0, D0, H0.copy(), alive.copy())
    F.fpic_push(ctx, p, fields_dev(Fo), prm)
    hp = F.HostParticles(n)
    if not pinned:
        import torch
        for f in F.HostParticles.FIELDS_D + F.HostParticles.FIELDS_B + ("cell",):
            t = getattr(hp, f)
            setattr(hp, f, torch.zeros(t.shape, dtype=t.dtype))
    for k, col in zip(("r", "th", "ph", "ur", "uth", "uph"), range(6)):
        getattr(hp, k).copy_(torch_from(z[:, col]))
    hp.qm.copy_(torch_from(q)); hp.H0.copy_(torch_from(H0)); hp.D0.copy_(torch_from(D0))
    hp.Hn.copy_(torch_from(H0)); hp.alive.copy_(torch_from(alive))
    F.fpic_push_host(ctx, hp, fields_dev(Fo), prm)
    zs, Hn, al, sc, it, cell = to_np(p)
    zh = np.stack([getattr(hp, k).numpy() for k in ("r", "th", "ph", "ur", "uth", "uph")], 1)
    assert np.array_equal(zh, zs)
    assert np.array_equal(hp.Hn.numpy(), Hn)
    assert np.array_equal(hp.alive.numpy(), al)
    assert np.array_equal(hp.scheme.numpy(), sc)
    assert np.array_equal(hp.iters.numpy(), it)
    assert np.array_equal(hp.cell.numpy().view(np.uint32), cell)


def torch_from(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x))


@pytest.mark.parametrize("scheme", ["HYB1", "HYB2"])
def test_adaptive_implicit_step_matches_oracle(F, scheme):
    """Sec. 3.1.2 / Tab. C.2 adaptive steps on the charged Wald workload
    (4741 particles, dt = 1e-3, the IMR partner with dt_implicit = 3e-3):
    states 1e-12, choices bit-exact (threshold ties excluded), and the
    per-particle time advanced by dt or dt_implicit as each particle's
    scheme says (removed-at-start particles keep their time)."""
    import torch
    a = 0.9
    g = I.wald_grid(128, a)
    Fo = O.wald_on_grid(a, 1.0, g)
    ctx = _mk(F, a, g)
    d, z, q = thermal_state(4741, g, a, theta=0.1, seed=13)
    n = len(q)
    alive = (np.arange(n) % 97 != 5).astype(np.uint8)
    t0 = np.linspace(0.0, 1.0, n)
    tg = torch.as_tensor(t0.copy(), device="cuda")
    thr = {"HYB1": 8e-5, "HYB2": 8e-8}[scheme]
    sch = getattr(F, "FPIC_" + scheme)
    p, st, (zo, Ho, ao, so, io, nc), (H0, D0, Hn) = _one_step(F, ctx, g, Fo, z, q, sch, 1e-3, thr=thr,
                                                              alive=alive, dt_imp=3e-3, t=tg)
    zg, Hg, ag, sg, ig, cg = to_np(p)
    assert np.array_equal(ag, ao)
    pr = O.push_params(a=a, dt=1e-3, scheme=O.RK4, B0pot=1.0, field_kind=O.FIELD_GRID, r_max=g.rn[-1])
    zr = np.ascontiguousarray(z.copy()); Hr = Hn.copy()
    O.push(pr, zr, q, H0, D0, Hr, np.ones(n, np.uint8), g, Fo)
    Ht1 = np.abs(Hr - H0) / D0
    stat = Ht1 if scheme == "HYB2" else (Ht1 - np.abs(Hn - H0) / D0) / 1e-3
    near = np.abs(stat - thr) <= 1e-12 * abs(thr) + 1e-12 * np.abs(stat)
    ok = ~near & (alive == 1)
    assert near.sum() <= 2
    assert np.array_equal(sg[ok], so[ok]) and 0 < so[alive == 1].sum() < alive.sum()
    assert_state_close(zg, zo, TOL, ok)
    t_exp = t0 + np.where(alive == 1, np.where(so == 1, 3e-3, 1e-3), 0.0)
    assert np.array_equal(tg.cpu().numpy()[ok | (alive == 0)], t_exp[ok | (alive == 0)])


def test_adaptive_step_dg_partner_matches_oracle(F):
    """Neutral geodesics with the discrete-gradient partner at dt = 0.5,
    dt_implicit = 1.0 (the a.0 column of Tab. C.2 takes 1.0 for the
    Hamiltonian steps): states within 1e-12, choices bit-exact, H conserved
    by the implicit steps."""
    a = 0.9
    ctx = _mk(F, a)
    z, bad = O.seed_orbits(1.0, a, I.orbit_candidates(1000, seed=4))
    q = np.zeros(len(z))
    H0 = O.hamiltonian(1.0, a, 0.0, z, q)[0]
    dt, dti = 0.5, 1.0
    pr = O.push_params(a=a, dt=dt, scheme=O.RK4)
    zr = np.ascontiguousarray(z.copy()); Hr = H0.copy()
    O.push(pr, zr, q, H0, H0, Hr, np.ones(len(q), np.uint8))
    stat = np.abs(Hr - H0) / H0
    thr = float(np.median(stat))
    p, st, (zo, Ho, ao, so, io, nc), _ = _one_step(F, ctx, None, None, z, q, F.FPIC_HYB2, dt, thr=thr,
                                                  implicit=F.FPIC_HAM, B0pot=0.0, tol=1e-15, dt_imp=dti)
    zg, Hg, ag, sg, ig, cg = to_np(p)
    near = np.abs(stat - thr) <= 1e-10 * thr + 1e-15
    assert near.sum() <= 10 and np.array_equal(sg[~near], so[~near]) and 0 < so.sum() < len(q)
    bound = np.full(len(q), TOL)
    err = (np.abs(zg - zo) / (np.abs(zo) + 1.0)).max(axis=1)
    assert np.all(err[~near] <= bound[~near]), (err / bound).max()
    imp = (so == 1) & ~near & (ag == 1)
    assert np.abs(Hg[imp] - H0[imp]).max() < 2e-14


@pytest.mark.parametrize("scheme", ["RK4", "IMR", "IMR_NEWTON", "HAM", "HYB2"])
def test_analytic_wald_push_matches_oracle(F, scheme):
    """Charged particles in the analytic Wald field (fields = NULL, B0field):
    RK4 / IMR / the discrete-gradient scheme in canonical momenta (an
    extension) / Hyb2 with the discrete-gradient partner, one step of 3001
    e-/e+ and neutral particles, a = 0.9, dt = 0.05: states within 1e-12 of
    the oracle (choices bit-exact away from threshold ties); the
    discrete-gradient steps keep H to 1e-14."""
    a, B0, dt = 0.9, 1.0, 0.05
    ctx = _mk(F, a)
    rng = np.random.default_rng(21)
    n = 3001
    z = np.stack([rng.uniform(4, 9, n), rng.uniform(0.7, 2.4, n), rng.uniform(0, 6, n),
                  rng.normal(size=n) * 0.3, rng.normal(size=n) * 0.5, rng.normal(size=n) * 2], 1)
    q = np.choose(np.arange(n) % 3, [np.full(n, -2.0), np.full(n, 2.0), np.zeros(n)])
    H0, _, D0 = O.hamiltonian(1.0, a, B0, z, q)
    Hn = H0.copy()
    newton = scheme == "IMR_NEWTON"
    scheme = "IMR" if newton else scheme
    sch = getattr(F, "FPIC_" + scheme)
    thr = 1e-12
    if scheme == "HYB2":
        pr = O.push_params(a=a, dt=dt, scheme=O.RK4, field_kind=O.FIELD_WALD, B0field=B0, B0pot=B0)
        zr = np.ascontiguousarray(z.copy()); Hr = Hn.copy()
        O.push(pr, zr, q, H0, D0, Hr, np.ones(n, np.uint8))
        stat = np.abs(Hr - H0) / D0
        thr = float(np.median(stat))
    p = make_particles(z, q, H0, D0, Hn)
    prm = F.push_params(dt, scheme=sch, implicit=F.FPIC_HAM, thr=thr, tol=1e-15, max_iter=100, B0pot=B0,
                        B0field=B0, imr_newton=newton)
    F.fpic_push(ctx, p, None, prm)
    po = O.push_params(a=a, dt=dt, scheme=sch, implicit_kind=O.HAM, thr=thr, tol=1e-15, max_iter=100, B0pot=B0,
                       field_kind=O.FIELD_WALD, B0field=B0, imr_newton=newton)
    zo = np.ascontiguousarray(z.copy()); Ho = Hn.copy(); ao = np.ones(n, np.uint8)
    nc, so, io = O.push(po, zo, q, H0, D0, Ho, ao)
    zg, Hg, ag, sg, ig, cg = to_np(p)
    assert np.array_equal(ag, ao)
    ok = np.ones(n, bool)
    if scheme == "HYB2":
        ok = np.abs(stat - thr) > 1e-10 * thr
        assert (~ok).sum() <= 2 and np.array_equal(sg[ok], so[ok]) and 0 < so.sum() < n
    assert_state_close(zg, zo, TOL, ok)
    if scheme in ("HAM", "HYB2"):
        imp = (so == 1) & ok
        Hnew = O.hamiltonian(1.0, a, B0, zg[imp], q[imp])[0]
        assert np.abs(Hnew - H0[imp]).max() <= 1e-14 * np.abs(H0).max()


def test_static_fields_reuse_changes_no_result():
    """FPIC_TUNE_STATIC_FIELDS reuses the interpolation coefficients while the
    field pointers stay the same: two pushes with it on give bitwise the
    results of two pushes with it off; new field arrays are picked up; the
    flag only takes 0 or 1."""
    cuda_or_skip()
    F = fpic()
    a = 0.9
    g = I.wald_grid(96, a)
    Fo = O.wald_on_grid(a, 1.0, g)
    ctx = F.fpic_init_metric(1.0, a)
    F.fpic_set_grid(ctx, g)
    d, z, q = thermal_state(3001, g, a, theta=0.1, seed=17)
    H0, _, D0 = O.hamiltonian(1.0, a, 1.0, z, q)
    prm = F.push_params(1e-3, scheme=F.FPIC_HYB1, implicit=F.FPIC_IMR, thr=8e-5, r_max=float(g.rn[-1]),
                        B0pot=1.0)
    fd = fields_dev(Fo)
    res = []
    for flag in (0, 1):
        F.fpic_set_tuning(ctx, F.FPIC_TUNE_STATIC_FIELDS, flag)
        assert F.fpic_get_tuning(ctx, F.FPIC_TUNE_STATIC_FIELDS) == flag
        p = make_particles(z, q, H0, D0, H0.copy())
        F.fpic_push(ctx, p, fd, prm)
        F.fpic_push(ctx, p, fd, prm)
        res.append(to_np(p)[0])
    assert np.array_equal(res[0], res[1])
    # a second, scaled field set through new arrays is used at once
    fd2 = fields_dev([2.0 * f for f in Fo])
    pa = make_particles(z, q, H0, D0, H0.copy())
    F.fpic_push(ctx, pa, fd2, prm)
    F.fpic_set_tuning(ctx, F.FPIC_TUNE_STATIC_FIELDS, 0)
    pb = make_particles(z, q, H0, D0, H0.copy())
    F.fpic_push(ctx, pb, fd2, prm)
    assert np.array_equal(to_np(pa)[0], to_np(pb)[0])
    with pytest.raises(F.FpicError):
        F.fpic_set_tuning(ctx, F.FPIC_TUNE_STATIC_FIELDS, 2)


def test_newton_imr_mixed_charges_is_deterministic_and_matches_oracle(F):
    """The Newton form of the IMR with grid fields on a mix of e-, e+ and
    neutral particles (the neutral ones take the field-free Newton matrix):
    one IMR step of 3001 particles within 1e-12 of the oracle, and two runs
    from the same state bitwise equal (no value of a previous particle or
    launch leaks into a solve)."""
    a = 0.9
    g = I.wald_grid(96, a)
    Fo = O.wald_on_grid(a, 1.0, g)
    ctx = _mk(F, a, g)
    d, z, q = thermal_state(3001, g, a, theta=0.1, seed=31)
    q = q * (np.arange(len(q)) % 3 != 2)          # every third particle neutral
    outs = []
    for _ in range(2):
        p, st, (zo, Ho, ao, so, io, nc), _ = _one_step(F, ctx, g, Fo, z, q, F.FPIC_IMR, 1e-3, newton=True)
        outs.append(to_np(p))
    for x, y in zip(*outs):
        assert np.array_equal(x, y)
    zg, Hg, ag, sg, ig, cg = outs[0]
    assert np.array_equal(ag, ao) and nc == 0
    assert_state_close(zg, zo, TOL)
    _check_iterations(ig, io, True)
    assert io[q == 0].mean() < io[q != 0].mean()


@pytest.mark.parametrize("newton", [False, True])
def test_unconverged_solve_returns_smallest_update_iterate(F, newton):
    """At a step far too long for the IMR map to contract (dt = 0.05,
    q/m = 100), every solve stops at max_iter = 4 and returns the iterate
    with the smallest update, as the oracle does: states within 1e-12 of the
    oracle, every particle counted as not converged (fixed-point form).  The
    Newton form converges for some of them (the kernel, with its a-posteriori
    stop, for at least as many as the oracle); either way GPU and oracle
    agree."""
    a = 0.9
    g = I.wald_grid(64, a)
    Fo = O.wald_on_grid(a, 1.0, g)
    ctx = _mk(F, a, g)
    d, z, q = thermal_state(1001, g, a, theta=0.1, seed=17)
    p, st, (zo, Ho, ao, so, io, nc), _ = _one_step(F, ctx, g, Fo, z, q, F.FPIC_IMR, 0.05, max_iter=4,
                                                   newton=newton, r_max=1e300)
    zg, Hg, ag, sg, ig, cg = to_np(p)
    if not newton:
        assert nc == len(q)
        assert st["n_notconv"] == nc
    else:
        # the kernel's a-posteriori stop accepts some solves the oracle's
        # successive-update test runs to the cap: those states still agree
        assert 0 < st["n_notconv"] <= nc
    ok = (ao == 1) & (ag == 1)
    assert ok.mean() > 0.9
    assert_state_close(zg, zo, TOL, ok)


@pytest.mark.parametrize("newton", [False, True])
def test_slope_reuse_matches_oracle_every_step(F, newton):
    """FPIC_TUNE_REUSE_SLOPE: each step's first RK4 stage comes from the
    right-hand side the previous step left at the particle's new state.
    Over five Hyb1 steps (grid Wald field, 4741 particles, ~15 % implicit)
    every step stays within 1e-12 of the oracle's step from the same input
    state, choices bit-exact away from threshold ties; between steps the
    state of every seventh particle is changed (its cached slope no longer
    applies), the particles are permuted, and the field pointers replaced
    by copies: the cache notices each change and the results stay within
    the bound."""
    a = 0.9
    g = I.wald_grid(128, a)
    Fo = O.wald_on_grid(a, 1.0, g)
    ctx = _mk(F, a, g)
    F.fpic_set_tuning(ctx, F.FPIC_TUNE_STATIC_FIELDS, 1)
    F.fpic_set_tuning(ctx, F.FPIC_TUNE_REUSE_SLOPE, 1)
    assert F.fpic_get_tuning(ctx, F.FPIC_TUNE_REUSE_SLOPE) == 1
    d, z, q = thermal_state(4741, g, a, theta=0.1, seed=37)
    n = len(q)
    H0, _, D0 = O.hamiltonian(1.0, a, 1.0, z, q)
    p = make_particles(z, q, H0, D0, H0.copy())
    fd = fields_dev(Fo)
    thr = 8e-5
    prm = F.push_params(1e-3, scheme=F.FPIC_HYB1, implicit=F.FPIC_IMR, thr=thr, r_max=g.rn[-1], B0pot=1.0,
                        imr_newton=newton)
    po = O.push_params(a=a, dt=1e-3, scheme=O.HYB1, implicit_kind=O.IMR, thr=thr, r_max=g.rn[-1], B0pot=1.0,
                       field_kind=O.FIELD_GRID, imr_newton=newton)
    pr = O.push_params(a=a, dt=1e-3, scheme=O.RK4, B0pot=1.0, field_kind=O.FIELD_GRID, r_max=g.rn[-1])
    implicit_seen = 0
    for step in range(5):
        if step == 2:
            ur = p.ur.clone()
            ur[::7] += 1e-3
            p.ur.copy_(ur)
        if step == 3:
            perm = torch.randperm(n, generator=torch.Generator().manual_seed(5)).cuda()
            for name in ("r", "th", "ph", "ur", "uth", "uph", "qm", "H0", "D0", "Hn", "alive"):
                t = getattr(p, name)
                t.copy_(t[perm])
        if step == 4:
            fd = [f.clone() for f in fd]
        zs, Hs, als, _, _, _ = to_np(p)
        q_s, H0_s, D0_s = (t.cpu().numpy() for t in (p.qm, p.H0, p.D0))
        st = F.fpic_push(ctx, p, fd, prm, stats=True)
        zg, Hg, ag, sg, ig, cg = to_np(p)
        zo = np.ascontiguousarray(zs.copy()); Ho = Hs.copy(); ao = als.copy()
        nc, so, io = O.push(po, zo, q_s, H0_s, D0_s, Ho, ao, g, Fo)
        zr = np.ascontiguousarray(zs.copy()); Hr = Hs.copy()
        O.push(pr, zr, q_s, H0_s, D0_s, Hr, als.copy(), g, Fo)
        stat = (np.abs(Hr - H0_s) - np.abs(Hs - H0_s)) / D0_s / 1e-3
        near = np.abs(stat - thr) <= 1e-12 * abs(thr) + 1e-12 * np.abs(stat)
        ok = ~near & (als == 1)
        assert near.sum() <= 2, step
        assert np.array_equal(ag[ok], ao[ok]) and np.array_equal(sg[ok], so[ok]), step
        assert_state_close(zg, zo, TOL, ok & (ao == 1))
        implicit_seen += int(so[ok].sum())
    assert implicit_seen > 0.05 * 5 * n


@pytest.mark.parametrize("scheme", ["RK4", "HYB1"])
def test_field_tile_staging_changes_no_result(F, scheme):
    """FPIC_TUNE_STAGE_FIELDS: the explicit pass stages the coefficient
    tiles of each block's cells in shared memory by TMA.  On a plasma
    filling every cell of a 96 x 96 grid (64 particles per cell, sorted by
    fpic_sort, a = 0.99 Wald field) almost every block stages its tile, and
    two steps give bitwise the particles of the unstaged push (the tile
    holds the same bytes; gathers outside it read global memory); a sample
    stays within 1e-12 of the oracle.  Unsorted, the same particles stage
    few tiles and still give bitwise the unstaged results."""
    a = 0.99
    g = I.wald_grid(96, a)
    Fo = O.wald_on_grid(a, 1.0, g)
    ctx = _mk(F, a, g)
    d, q, w = I.cell_fill_draws(g, 64, 0.5, seed=41, qm=100.0, r_lo=1.02 * I.horizon(1.0, a))
    z = O.seed_fido(1.0, a, d)
    n = len(q)
    H0, _, D0 = O.hamiltonian(1.0, a, 1.0, z, q)
    fd = fields_dev(Fo)
    thr = 8e-5
    prm = F.push_params(1e-3, scheme=getattr(F, "FPIC_" + scheme), implicit=F.FPIC_IMR, thr=thr, r_max=g.rn[-1],
                        B0pot=1.0, imr_newton=True)
    rng = np.random.default_rng(43)
    for sort in (True, False):
        zz = z if sort else z[rng.permutation(n)]
        ps, pu = make_particles(zz, q, H0, D0, H0.copy()), make_particles(zz, q, H0, D0, H0.copy())
        F.fpic_cell_index(ctx, ps)
        F.fpic_cell_index(ctx, pu)
        if sort:
            F.fpic_sort(ctx, ps)
            F.fpic_sort(ctx, pu)
        if sort:
            z_in, q_in, H0_in, D0_in = (t.cpu().numpy() for t in (ps.state(), ps.qm, ps.H0, ps.D0))
        staged = 0
        for step in range(2):
            F.fpic_set_tuning(ctx, F.FPIC_TUNE_STAGE_FIELDS, 1)
            st = F.fpic_push(ctx, ps, fd, prm, stats=True)
            staged += st["n_tiles_staged"]
            F.fpic_set_tuning(ctx, F.FPIC_TUNE_STAGE_FIELDS, 0)
            su = F.fpic_push(ctx, pu, fd, prm, stats=True)
            assert su["n_tiles_staged"] == 0
            for x, y in zip(to_np(ps), to_np(pu)):
                assert np.array_equal(x, y)
        blocks = 2 * ((n + 127) // 128)
        if sort:
            assert staged > 0.85 * blocks, (staged, blocks)
        else:
            assert staged < 0.05 * blocks, (staged, blocks)
    # one staged step from the sorted input against the oracle on a sample
    pt = make_particles(z_in, q_in, H0_in, D0_in, H0_in.copy())
    F.fpic_cell_index(ctx, pt)
    F.fpic_set_tuning(ctx, F.FPIC_TUNE_STAGE_FIELDS, 1)
    F.fpic_push(ctx, pt, fd, prm)
    F.fpic_set_tuning(ctx, F.FPIC_TUNE_STAGE_FIELDS, 0)
    zg, Hg, ag, sg, ig, cg = to_np(pt)
    idx = np.sort(rng.choice(n, 3000, replace=False))
    po = O.push_params(a=a, dt=1e-3, scheme=getattr(O, scheme), implicit_kind=O.IMR, thr=thr, r_max=g.rn[-1],
                       B0pot=1.0, field_kind=O.FIELD_GRID, imr_newton=True)
    zo = np.ascontiguousarray(z_in[idx]); Ho = H0_in[idx].copy(); ao = np.ones(len(idx), np.uint8)
    nc, so, io = O.push(po, zo, q_in[idx], H0_in[idx], D0_in[idx], Ho, ao, g, Fo)
    ok = (ao == 1) & (ag[idx] == 1)
    if scheme == "HYB1":
        ok &= so == sg[idx]
        assert (so != sg[idx]).sum() <= 2
    assert ok.mean() > 0.95
    assert_state_close(zg[idx], zo, TOL, ok)


def _axis_state(n, seed):
    rng = np.random.default_rng(seed)
    th = np.exp(rng.uniform(np.log(1e-5), np.log(3e-4), n))
    north = rng.random(n) < 0.5
    th = np.where(north, th, np.pi - th)
    uth = rng.uniform(0.3, 3.0, n) * np.where(north, -1.0, 1.0)
    z = np.stack([rng.uniform(1.5, 5.0, n), th, rng.uniform(0, 6, n), rng.normal(size=n) * 0.5, uth,
                  rng.normal(size=n) * 2e-4], 1)
    q = np.where(np.arange(n) % 2 == 0, -100.0, 100.0)
    return np.ascontiguousarray(z), q


@pytest.mark.parametrize("field,newton", [("wald", True), ("wald", False), ("grid", True)])
def test_unconverged_solves_redone_in_substeps_match_oracle(F, field, newton):
    """Particles within 3e-4 rad of a pole heading for it (601 e-/e+,
    dt = 1e-3, IMR): most full-step solves do not converge; with
    imr_substeps = 8 the library redoes them in 2, 4, ... substeps as the
    oracle does.  Solves that converge on their own match at 1e-12; the
    substepped ones (up to 256 sequential solves near the axis) match the
    oracle's to 1e-10 except where the two sides take a different level
    (a solve converging at the max_iter edge, at most 2 %), and the counts
    of unconverged solves agree to the same margin."""
    a, B0, dt = 0.9, 1.0, 1e-3
    z, q = _axis_state(601, 43)
    n = len(q)
    H0, _, D0 = O.hamiltonian(1.0, a, B0, z, q)
    if field == "wald":
        ctx = _mk(F, a)
        fd, Fo, g = None, None, None
        okw = dict(field_kind=O.FIELD_WALD, B0field=B0)
        gkw = dict(B0field=B0)
    else:
        g = I.wald_grid(256, a)
        Fo = O.wald_on_grid(a, B0, g)
        ctx = _mk(F, a, g)
        fd = fields_dev(Fo)
        okw = dict(field_kind=O.FIELD_GRID)
        gkw = {}
    r_max = g.rn[-1] if g is not None else 1e300
    for K, tol_s in ((0, 0.0), (8, 0.0), (8, 1e-6)):
        p = make_particles(z, q, H0, D0, H0.copy())
        prm = F.push_params(dt, scheme=F.FPIC_IMR, B0pot=B0, imr_newton=newton, r_max=r_max,
                            imr_substeps=K, substep_tol=tol_s, **gkw)
        st = F.fpic_push(ctx, p, fd, prm, stats=True)
        po = O.push_params(a=a, dt=dt, scheme=O.IMR, B0pot=B0, imr_newton=newton, r_max=r_max, imr_substeps=K,
                           substep_tol=tol_s, **okw)
        zo = np.ascontiguousarray(z.copy()); Ho = H0.copy(); ao = np.ones(n, np.uint8)
        nc, so, io, fo = O.push(po, zo, q, H0, D0, Ho, ao, g, Fo, flags=True)
        zg = to_np(p)[0]
        err = (np.abs(zg - zo) / (np.abs(zo) + 1.0)).max(axis=1)
        if K == 0:
            fail = fo == 1
            z_full = zo.copy()
            assert fail.mean() > 0.2
            assert err[~fail].max() <= 1e-12
            continue
        # steps redone: the unconverged ones and, with an H condition, the
        # converged ones whose end point misses it (H^n = H0 here)
        dH_full = np.abs(O.hamiltonian(1.0, a, B0, z_full, q)[0] - H0) / D0
        trig = fail | ((dH_full > tol_s) if tol_s > 0 else False)
        edge = np.abs(dH_full - tol_s) <= 1e-9 * tol_s if tol_s > 0 else np.zeros(n, bool)
        assert err[~trig & ~edge].max() <= 1e-12
        bad = err[trig] > 1e-10
        print(f"K={K} tol={tol_s}: {trig.sum()} substepped ({fail.sum()} unconverged), {bad.sum()} beyond 1e-10, "
              f"median err {np.median(err[trig]):.1e}, notconv gpu {st['n_notconv']} oracle {nc}")
        assert bad.mean() <= 0.02, (bad.sum(), trig.sum())
        assert abs(st["n_notconv"] - nc) <= max(2, 0.02 * fail.sum())
        assert nc < 0.1 * fail.sum()


def test_full_theta_wald_field_matches_oracle(F):
    """fpic_init_wald on a full-theta grid (fpic_set_theta_mode FULL): every
    Yee component at th in (pi, 2 pi) from the continued closed forms, and
    column Nth the exact image of column 0, as the oracle samples it."""
    a = 0.9
    g = I.full_theta_grid(64, 96, 0.9 * I.horizon(1.0, a), 40.0)
    ctx = _mk(F, a, g)
    Fo = O.wald_on_grid(a, 1.0, g)
    Fg = [dev(np.zeros_like(f)) for f in Fo]
    F.fpic_init_wald(ctx, Fg, 1.0)
    for k in range(6):
        got = Fg[k].cpu().numpy().reshape(g.Nr + 1, g.ld)
        exp = Fo[k].reshape(g.Nr + 1, g.ld)
        rows = g.Nr if k in (0, 4, 5) else g.Nr + 1
        assert np.array_equal(got[:rows, g.Nth], got[:rows, 0])
        assert np.abs(got[:rows] - exp[:rows]).max() <= 1e-13 * np.abs(exp).max(), k


@pytest.mark.parametrize("scheme", ["RK4", "HYB1"])
def test_full_theta_push_matches_oracle(F, scheme):
    """Charged particles (q/m = -/+100) over the whole period of a
    full-theta grid (96 x 128, a = 0.9 Wald field on it), some next to the
    wrap at tn[0] and tn[0] + 2 pi and next to th = pi, plus meridional
    geodesics crossing the poles: three steps, each within 1e-12 of the
    oracle's full-theta step from the same state (periodic gather with the
    half-node wrap cell, periodic particle boundary), cells and alive flags
    bit-exact, scheme choices bit-exact away from threshold ties; slope
    reuse on from the second step."""
    a = 0.9
    g = I.full_theta_grid(96, 128, 0.9 * I.horizon(1.0, a), 40.0)
    Fo = O.wald_on_grid(a, 1.0, g)
    ctx = _mk(F, a, g)
    F.fpic_set_tuning(ctx, F.FPIC_TUNE_STATIC_FIELDS, 1)
    F.fpic_set_tuning(ctx, F.FPIC_TUNE_REUSE_SLOPE, 1)
    d, z, q = thermal_state(3000, g, a, theta=0.1, seed=61)
    rng = np.random.default_rng(62)
    t0 = g.tn[0]
    edge = np.concatenate([t0 + rng.uniform(1e-6, 2e-3, 150), t0 + 2 * np.pi - rng.uniform(1e-6, 2e-3, 150),
                           np.pi + rng.choice([-1.0, 1.0], 150) * rng.uniform(1e-3, 4e-3, 150)])
    z[:450, 1] = edge
    north = rng.random(200) < 0.5
    zm = np.stack([rng.uniform(6.0, 12.0, 200),
                   np.where(north, t0 + rng.uniform(0, 3e-5, 200), np.pi - rng.uniform(0, 3e-5, 200)),
                   rng.uniform(0, 6, 200), rng.normal(size=200) * 0.2, np.where(north, -2.0, 2.0),
                   np.zeros(200)], 1)
    z = np.ascontiguousarray(np.concatenate([z, zm]))
    q = np.concatenate([q, np.zeros(200)])
    n = len(q)
    H0, _, D0 = O.hamiltonian(1.0, a, 1.0, z, q)
    p = make_particles(z, q, H0, D0, H0.copy())
    fd = fields_dev(Fo)
    sch = getattr(F, "FPIC_" + scheme)
    thr = 8e-5
    prm = F.push_params(1e-3, scheme=sch, implicit=F.FPIC_IMR, thr=thr, r_max=g.rn[-1], B0pot=1.0, imr_newton=True)
    po = O.push_params(a=a, dt=1e-3, scheme=getattr(O, scheme), implicit_kind=O.IMR, thr=thr, r_max=g.rn[-1],
                       B0pot=1.0, field_kind=O.FIELD_GRID, imr_newton=True, grid=g)
    pr = O.push_params(a=a, dt=1e-3, scheme=O.RK4, r_max=g.rn[-1], B0pot=1.0, field_kind=O.FIELD_GRID, grid=g)
    wrapped = 0
    for step in range(3):
        zs, Hs, als, _, _, _ = to_np(p)
        F.fpic_push(ctx, p, fd, prm)
        zg, Hg, ag, sg, ig, cg = to_np(p)
        zo = np.ascontiguousarray(zs.copy()); Ho = Hs.copy(); ao = als.copy()
        nc, so, io = O.push(po, zo, q, H0, D0, Ho, ao, g, Fo)
        ok = als == 1
        if scheme == "HYB1":
            zr = np.ascontiguousarray(zs.copy()); Hr = Hs.copy()
            O.push(pr, zr, q, H0, D0, Hr, als.copy(), g, Fo)
            stat = (np.abs(Hr - H0) - np.abs(Hs - H0)) / D0 / 1e-3
            near = np.abs(stat - thr) <= 1e-12 * abs(thr) + 1e-12 * np.abs(stat)
            assert near.sum() <= 2
            ok &= ~near
            assert np.array_equal(sg[ok], so[ok])
        assert np.array_equal(ag[ok], ao[ok])
        live = ok & (ao == 1)
        assert_state_close(zg, zo, TOL, live)
        rel = np.minimum(np.abs(zo[:, 0, None] / g.rn[None, :] - 1).min(1), np.abs(zo[:, 1, None] - g.tn[None, :]).min(1))
        far = live & (rel > 1e-11)
        assert np.array_equal(cg[far], O.cell_index(g, zo[far, 0], zo[far, 1]))
        assert ((zg[live, 1] >= t0) & (zg[live, 1] < t0 + 2 * np.pi)).all()
        wrapped += int((np.abs(zg[live, 1] - zs[live, 1]) > np.pi).sum())
    assert wrapped > 0


def test_full_theta_rejects_the_grid_side_solvers(F):
    """In the full-theta domain the deposits, cleaning and injection are not
    built: they refuse with FPIC_EINVAL instead of running."""
    a = 0.9
    g = I.full_theta_grid(16, 32, 0.9 * I.horizon(1.0, a), 40.0)
    ctx = _mk(F, a, g)
    z = np.ascontiguousarray(np.tile([[8.0, 1.0, 0.0, 0.0, 0.0, 3.0]], (10, 1)))
    p = make_particles(z, np.ones(10))
    with pytest.raises(F.FpicError, match="full-theta"):
        F.fpic_deposit(ctx, p, g.size)
    with pytest.raises(F.FpicError, match="full-theta"):
        F.fpic_deposit_conserving(ctx, p, make_particles(z, np.ones(10)), 1e-3)
    fl = F.Fields(g.size)
    with pytest.raises(F.FpicError, match="full-theta"):
        F.fpic_div_clean(ctx, fl.D1, fl.rho1, 5)
    F.fpic_set_theta_mode(ctx, F.FPIC_THETA_HALF)
    F.fpic_deposit(ctx, p, g.size)          # the half-theta reading of the same tables


@pytest.mark.parametrize("scheme", ["RK4", "HYB1"])
def test_push_writes_the_state_it_starts_from(F, scheme):
    """fpic_push_params.before: the explicit pass stores every particle's
    r, th, ur, uth, uph and alive at the start of the step (removed ones
    included, their flag 0) -- bitwise the state before the push -- and
    leaves the other arrays of `before` alone; the pushed result is the
    same as without it.  The batched, learned, host and allocation-free
    pushes refuse it."""
    a = 0.9
    g = I.wald_grid(64, a)
    Fo = O.wald_on_grid(a, 1.0, g)
    ctx = _mk(F, a, g)
    d, z, q = thermal_state(4001, g, a, theta=0.1, seed=71)
    n = len(q)
    H0, _, D0 = O.hamiltonian(1.0, a, 1.0, z, q)
    alive = np.ones(n, np.uint8)
    alive[::7] = 0
    p = make_particles(z, q, H0, D0, H0.copy(), alive=alive)
    p2 = make_particles(z, q, H0, D0, H0.copy(), alive=alive)
    before = make_particles(np.full((n, 6), -1.0), np.full(n, -3.0))
    before.alive.fill_(7)
    fd = fields_dev(Fo)
    sch = getattr(F, "FPIC_" + scheme)
    prm = F.push_params(1e-3, scheme=sch, implicit=F.FPIC_IMR, thr=8e-5, r_max=g.rn[-1], B0pot=1.0, imr_newton=True)
    F.fpic_push(ctx, p2, fd, prm)
    F.set_push_before(prm, before)
    F.fpic_push(ctx, p, fd, prm)
    zb = before.state().cpu().numpy()
    ab = before.alive.cpu().numpy()
    assert np.array_equal(ab, alive)
    live = alive == 1
    for i in (0, 1, 3, 4, 5):
        assert np.array_equal(zb[live, i], z[live, i]), i
    assert np.all(zb[:, 2] == -1.0) and np.all(zb[~live] == -1.0)
    assert np.all(before.qm.cpu().numpy() == -3.0)
    assert np.array_equal(p.state().cpu().numpy(), p2.state().cpu().numpy())
    with pytest.raises(F.FpicError, match="before"):
        F.fpic_push_noalloc(1.0, a, p, prm)
    short = make_particles(np.ones((n - 1, 6)), np.ones(n - 1))
    F.set_push_before(prm, short)
    with pytest.raises(F.FpicError, match="fewer"):
        F.fpic_push(ctx, p, fd, prm)
    F.set_push_before(prm, None)
    F.fpic_push(ctx, p, fd, prm)


def test_async_stats_and_host_push_match_the_synchronous_ones(F):
    """FPIC_TUNE_ASYNC: fpic_push with stats assembled on the device and
    copied to pinned memory without a wait, and fpic_push_host on pinned
    arrays returning before its results land, give -- once the stream is
    synchronised -- bitwise the synchronous calls' states and stats over
    three steps each."""
    import torch
    a = 0.9
    g = I.wald_grid(96, a)
    Fo = O.wald_on_grid(a, 1.0, g)
    ctx = _mk(F, a, g)
    d, z, q = thermal_state(6007, g, a, theta=0.1, seed=83)
    n = len(q)
    H0, _, D0 = O.hamiltonian(1.0, a, 1.0, z, q)
    alive = (np.arange(n) % 9 != 4).astype(np.uint8)
    fd = fields_dev(Fo)
    prm = F.push_params(1e-3, scheme=F.FPIC_HYB1, implicit=F.FPIC_IMR, thr=8e-5, r_max=float(g.rn[-1]),
                        B0pot=1.0, imr_newton=True)
    p1 = make_particles(z, q, H0, D0, H0.copy(), alive.copy())
    p2 = make_particles(z, q, H0, D0, H0.copy(), alive.copy())
    ref = [F.fpic_push(ctx, p1, fd, prm, stats=True) for _ in range(3)]
    F.fpic_set_tuning(ctx, F.FPIC_TUNE_ASYNC, 1)
    assert F.fpic_get_tuning(ctx, F.FPIC_TUNE_ASYNC) == 1
    outs = torch.zeros((3, 8), dtype=torch.int64).pin_memory()
    for i in range(3):
        assert F.fpic_push(ctx, p2, fd, prm, stats_out=outs[i]) is None
    torch.cuda.synchronize()
    assert [F.stats_dict(outs[i]) for i in range(3)] == ref
    assert np.array_equal(p1.state().cpu().numpy(), p2.state().cpu().numpy())
    assert ref[0]["n_implicit"] > 0

    def host_set():
        hp = F.HostParticles(n)
        for k, col in zip(("r", "th", "ph", "ur", "uth", "uph"), range(6)):
            getattr(hp, k).copy_(torch_from(z[:, col]))
        hp.qm.copy_(torch_from(q)); hp.H0.copy_(torch_from(H0)); hp.D0.copy_(torch_from(D0))
        hp.Hn.copy_(torch_from(H0)); hp.alive.copy_(torch_from(alive))
        return hp
    F.fpic_set_tuning(ctx, F.FPIC_TUNE_ASYNC, 0)
    hs = host_set()
    ref_h = [F.fpic_push_host(ctx, hs, fd, prm, stats=True) for _ in range(3)]
    F.fpic_set_tuning(ctx, F.FPIC_TUNE_ASYNC, 1)
    ha = host_set()
    outs.zero_()
    for i in range(3):
        F.fpic_push_host(ctx, ha, fd, prm, stats_out=outs[i])
    torch.cuda.synchronize()
    assert [F.stats_dict(outs[i]) for i in range(3)] == ref_h
    for k in ("r", "th", "ph", "ur", "uth", "uph", "Hn", "alive", "scheme", "iters"):
        assert np.array_equal(getattr(hs, k).numpy(), getattr(ha, k).numpy()), k
    F.fpic_set_tuning(ctx, F.FPIC_TUNE_ASYNC, 0)


def test_pushes_with_async_stats_replay_from_a_cuda_graph(F):
    """Three hybrid pushes captured in one CUDA graph, each with its stats
    copied asynchronously into its own pinned slot (FPIC_TUNE_ASYNC), then
    replayed twice: states and every stat bitwise those of six eager pushes
    from the same start."""
    import torch
    a = 0.9
    g = I.wald_grid(96, a)
    Fo = O.wald_on_grid(a, 1.0, g)
    ctx = _mk(F, a, g)
    F.fpic_set_tuning(ctx, F.FPIC_TUNE_STATIC_FIELDS, 1)
    d, z, q = thermal_state(5003, g, a, theta=0.1, seed=91)
    H0, _, D0 = O.hamiltonian(1.0, a, 1.0, z, q)
    fd = fields_dev(Fo)
    prm = F.push_params(1e-3, scheme=F.FPIC_HYB1, implicit=F.FPIC_IMR, thr=8e-5, r_max=float(g.rn[-1]),
                        B0pot=1.0, imr_newton=True)
    p1 = make_particles(z, q, H0, D0, H0.copy())
    p2 = make_particles(z, q, H0, D0, H0.copy())
    ref = [F.fpic_push(ctx, p1, fd, prm, stats=True) for _ in range(7)]
    F.fpic_set_tuning(ctx, F.FPIC_TUNE_ASYNC, 1)
    slots = torch.zeros((3, 8), dtype=torch.int64).pin_memory()
    F.fpic_push(ctx, p2, fd, prm, stats_out=slots[0])          # eager: scratch in place before capture
    torch.cuda.synchronize()
    assert F.stats_dict(slots[0]) == ref[0]
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        for i in range(3):
            F.fpic_push(ctx, p2, fd, prm, stats_out=slots[i])
    got = []
    for _ in range(2):
        graph.replay()
        torch.cuda.synchronize()
        got += [F.stats_dict(slots[i]) for i in range(3)]
    assert got == ref[1:]
    assert np.array_equal(p1.state().cpu().numpy(), p2.state().cpu().numpy())
    assert np.array_equal(p1.alive.cpu().numpy(), p2.alive.cpu().numpy())
    F.fpic_set_tuning(ctx, F.FPIC_TUNE_ASYNC, 0)
