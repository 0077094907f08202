"""GPU tests of the learned implicit guess wired into the push: features,
samples taken from the plain method, and the learned hybrid push (parity of
every step with the oracle's own schemes, and the gain in right-hand-side
evaluations over the plain hybrid)."""
import numpy as np
import pytest

import oracle as O
from paper_2602_07452_gb300 import inputs as I
from helpers import cuda_or_skip, dev, fields_dev, fpic, make_particles, thermal_state, to_np

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
A, DT, THR = 0.9, 1e-3, 8e-5


@pytest.fixture(scope="module")
def setup():
    cuda_or_skip()
    F = fpic()
    g = I.wald_grid(128, A)
    Fo = O.wald_on_grid(A, 1.0, g)
    ctx = F.fpic_init_metric(1.0, A)
    F.fpic_set_grid(ctx, g)
    return F, g, Fo, ctx


def _parts(n, g, seed):
    d, z, q = thermal_state(n, g, A, theta=0.1, seed=seed)
    H0, _, D0 = O.hamiltonian(1.0, A, 1.0, z, q)
    return z, q, H0, D0


def test_features_match_definition(setup):
    """The 14 FP32 features equal their FP64 definitions (ln r, th, u_i, the
    gathered D^i, B^i, the energy error (H^n - H_0)/D_0, the fractional r
    position in the cell, (q/m) dt) to FP32 accuracy."""
    F, g, Fo, ctx = setup
    z, q, H0, D0 = _parts(3001, g, 4)
    Hn = H0 * (1 + 1e-7 * np.sin(np.arange(len(q))))
    p = make_particles(z, q, H0, D0, Hn)
    X = F.fpic_features(ctx, p, fields_dev(Fo), DT).cpu().numpy().astype(np.float64)
    DB = O.gather(g, Fo, z[:, 0], z[:, 1])
    i = np.searchsorted(g.rn, z[:, 0], side="right") - 1
    wr = (z[:, 0] - g.rn[i]) / (g.rn[i + 1] - g.rn[i])
    ref = np.concatenate([np.log(z[:, :1]), z[:, 1:2], z[:, 3:6], DB, ((Hn - H0) / D0)[:, None], wr[:, None],
                          (q * DT)[:, None]], 1)
    err = np.abs(X[:, :14] - ref) / (np.abs(ref).max(0) + 1e-30)
    assert err.max() < 1e-5, err.max(0)
    assert np.all(X[:, 14:] == 0)


def test_samples_are_the_plain_method(setup):
    """Targets = the converged IMR step (started from the RK4 trial) minus z^n,
    labels = the plain Hyb1 verdict; the particles are left unchanged."""
    F, g, Fo, ctx = setup
    n = 4097
    z, q, H0, D0 = _parts(n, g, 5)
    p = make_particles(z, q, H0, D0, H0.copy())
    prm = F.push_params(DT, scheme=F.FPIC_HYB1, implicit=F.FPIC_IMR, thr=THR, r_max=float(g.rn[-1]), B0pot=1.0)
    X, T, S = F.fpic_learn_sample(ctx, p, fields_dev(Fo), prm)
    assert np.array_equal(p.state().cpu().numpy(), z)
    # oracle: IMR from z (converges to the same fixed point) and the Hyb1 verdict
    po = O.push_params(a=A, dt=DT, scheme=O.IMR, field_kind=O.FIELD_GRID, r_max=g.rn[-1], B0pot=1.0)
    zi = np.ascontiguousarray(z.copy()); Hx = H0.copy()
    O.push(po, zi, q, H0, D0, Hx, np.ones(n, np.uint8), g, Fo)
    inc = T[:, :6].double().cpu().numpy()
    assert np.abs(inc - (zi - z)).max() <= 1e-6 * np.abs(zi - z).max() + 1e-12
    pr = O.push_params(a=A, dt=DT, scheme=O.RK4, field_kind=O.FIELD_GRID, r_max=g.rn[-1], B0pot=1.0)
    zr = np.ascontiguousarray(z.copy()); Hr = H0.copy()
    O.push(pr, zr, q, H0, D0, Hr, np.ones(n, np.uint8), g, Fo)
    stat = (np.abs(Hr - H0) / D0 - 0.0) / DT
    rej = (stat >= THR).astype(float)
    near = np.abs(stat - THR) < 1e-9 * THR
    assert np.array_equal(S.cpu().numpy()[~near], rej[~near])
    assert 0.05 < rej.mean() < 0.8


def test_learned_push_parity_and_gain(setup):
    """Train briefly on samples of the plain pusher, then one learned step:
    every particle's result is the oracle's (IMR for those sent implicit,
    RK4 for the rest, whose H test passes), and the learned push spends
    fewer right-hand-side evaluations than the plain hybrid."""
    from paper_2602_07452_gb300 import learned as L
    F, g, Fo, ctx = setup
    n = 1 << 16
    z, q, H0, D0 = _parts(n, g, 6)
    fd = fields_dev(Fo)
    prm = F.push_params(DT, scheme=F.FPIC_HYB1, implicit=F.FPIC_IMR, thr=THR, r_max=float(g.rn[-1]), B0pot=1.0)
    p = make_particles(z, q, H0, D0, H0.copy())
    cfg = L.fit_cfg(ctx, p, fd, prm, p_skip=0.7)
    X, T, S = L.generate(ctx, p, fd, prm, cfg, steps=10)
    net, P, hist = L.train(X, T, S, steps=2500, batch=8192, lr=3e-3, log_every=500)
    assert hist[-1][1] < hist[0][1]
    # one step from identical states: plain vs learned
    zs = p.state().cpu().numpy(); Hn = p.Hn.cpu().numpy(); al = p.alive.cpu().numpy()
    pp = make_particles(zs, q, H0, D0, Hn.copy(), al.copy())
    pl = make_particles(zs, q, H0, D0, Hn.copy(), al.copy())
    st_p = F.fpic_push(ctx, pp, fd, prm, stats=True)
    st_l = F.fpic_push_learned(ctx, net, pl, fd, prm, cfg, stats=True)
    zl, Hl, alv, sl, il, _ = to_np(pl)
    live = al == 1
    # oracle per particle with the scheme the learned push took
    imp = (sl == 1) & live
    exp_ = (sl == 0) & live
    po = O.push_params(a=A, dt=DT, scheme=O.IMR, field_kind=O.FIELD_GRID, r_max=g.rn[-1], B0pot=1.0)
    zi = np.ascontiguousarray(zs[imp]); Hi = Hn[imp].copy()
    O.push(po, zi, q[imp], H0[imp], D0[imp], Hi, np.ones(imp.sum(), np.uint8), g, Fo)
    err_i = (np.abs(zl[imp] - zi) / (np.abs(zi) + 1)).max()
    pr = O.push_params(a=A, dt=DT, scheme=O.RK4, field_kind=O.FIELD_GRID, r_max=g.rn[-1], B0pot=1.0)
    ze = np.ascontiguousarray(zs[exp_]); He = Hn[exp_].copy()
    O.push(pr, ze, q[exp_], H0[exp_], D0[exp_], He, np.ones(exp_.sum(), np.uint8), g, Fo)
    err_e = (np.abs(zl[exp_] - ze) / (np.abs(ze) + 1)).max()
    assert err_i <= 1e-12 and err_e <= 1e-12, (err_i, err_e)
    stat = (np.abs(He - H0[exp_]) - np.abs(Hn[exp_] - H0[exp_])) / D0[exp_] / DT
    assert np.all(stat < THR * (1 + 1e-9))          # every kept RK4 step passed the plain test
    ev_p = st_p["n_rhs_evals"] / st_p["n_alive_before"]
    ev_l = st_l["n_rhs_evals"] / st_l["n_alive_before"]
    assert ev_l < ev_p, (ev_l, ev_p, st_p, st_l)


# ---------------------------------------------------------------------------
# Corrector form: the network corrects the implicit guess of rejected trials
# ---------------------------------------------------------------------------
def _slope(g, Fo, z, q):
    DB = O.gather(g, Fo, z[:, 0], z[:, 1])
    return O.rhs(1.0, A, z, q, DB[:, :3], DB[:, 3:])


def _match_rows(X, z):
    """Row -> particle, by the ln r feature (FP32) nearest to the particles'
    own value; must be a permutation."""
    key = np.log(z[:, 0])
    idx = np.empty(X.shape[0], np.int64)
    for b in range(0, X.shape[0], 512):
        idx[b:b + 512] = np.abs(X[b:b + 512, None, 12] - key[None, :]).argmin(1)
    assert np.unique(idx).size == X.shape[0]
    return idx


def test_corrector_samples_are_the_plain_method(setup):
    """Corrector form: one row per implicit-queue slot (every alive particle
    in sampling); features = per-component dt (k3 - k2) and dt (k4 - 2 k2 +
    k1) over s = |.| + |.|, then ln r and ln(|A| / |z_RK4 - z^n|) over u_r, u_th;
    targets = (z_IMR - z_RK4 -
    (2/3 A - 1/6 B)) / s, the gap left by the leading-order term; labels =
    the plain Hyb1 verdict.  Row by row against the oracle's
    right-hand side (RK4 stages of Sec. 2.2.1) and IMR; the particles are
    left unchanged."""
    F, g, Fo, ctx = setup
    n = 2048
    z, q, H0, D0 = _parts(n, g, 7)
    fd = fields_dev(Fo)
    p = make_particles(z, q, H0, D0, H0.copy())
    prm = F.push_params(DT, scheme=F.FPIC_HYB1, implicit=F.FPIC_IMR, thr=THR, r_max=float(g.rn[-1]), B0pot=1.0)
    X, T, S = F.fpic_learn_sample(ctx, p, fd, prm, F.learned_cfg(mode=F.FPIC_LEARN_CORRECT))
    assert np.array_equal(p.state().cpu().numpy(), z)
    X, T, S = (t.double().cpu().numpy() for t in (X, T, S))
    idx = _match_rows(X, z)
    zz, qq = z[idx], q[idx]
    k1 = _slope(g, Fo, zz, qq)
    k2 = _slope(g, Fo, zz + 0.5 * DT * k1, qq)
    k3 = _slope(g, Fo, zz + 0.5 * DT * k2, qq)
    k4 = _slope(g, Fo, zz + DT * k3, qq)
    zr = zz + DT / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
    Av, Bv = DT * (k3 - k2), DT * (k4 - 2 * k2 + k1)
    s = np.abs(Av) + np.abs(Bv)
    safe = np.where(s > 0, s, 1.0)
    assert np.abs(X[:, :6] - np.where(s > 0, Av / safe, 0)).max() < 1e-5
    assert np.abs(X[:, 6:12] - np.where(s > 0, Bv / safe, 0)).max() < 1e-5
    e = np.log(np.abs(Av[:, 3:5]).sum(1) / np.abs(zr[:, 3:5] - zz[:, 3:5]).sum(1))
    assert np.abs(X[:, 13] - e).max() < 1e-4 * np.abs(e).max()
    assert np.all(X[:, 14:] == 0)
    po = O.push_params(a=A, dt=DT, scheme=O.IMR, field_kind=O.FIELD_GRID, r_max=g.rn[-1], B0pot=1.0)
    zi = np.ascontiguousarray(zz.copy()); Hx = H0[idx].copy()
    O.push(po, zi, qq, H0[idx], D0[idx], Hx, np.ones(n, np.uint8), g, Fo)
    lead = 2.0 / 3.0 * Av - Bv / 6.0            # leading-order IMR - RK4 gap
    gap = (zi - zr - lead) / safe
    ok = (s > 1e-12 * (np.abs(zz) + 1)) & (np.abs(gap) < 3.9)
    assert ok.mean() > 0.8
    assert np.abs(T[:, :6] - gap)[ok].max() <= 1e-4 * np.abs(gap[ok]).max() + 1e-6
    # labels: the plain verdict of each row's particle
    stat = (np.abs(_rk4_H(g, Fo, zr, qq) - H0[idx]) / D0[idx]) / DT
    near = np.abs(stat - THR) < 1e-9 * THR
    assert np.array_equal(S[~near], (stat >= THR).astype(float)[~near])


def _rk4_H(g, Fo, zr, q):
    H, _, _ = O.hamiltonian(1.0, A, 1.0, zr, q)
    return H


@pytest.mark.parametrize("newton", [False, True])
def test_corrector_push_parity_and_gain(setup, newton):
    """Train the corrector briefly on the plain pusher's rejected trials, then
    one step from the same state with the plain and the learned push: the
    scheme choices are identical (the trial and the test are the plain
    ones), every particle matches the plain push and the oracle to 1e-12
    (the IMR in its fixed-point or Newton form on both sides),
    and the implicit solves need fewer iterations."""
    from paper_2602_07452_gb300 import learned as L
    F, g, Fo, ctx = setup
    n = 1 << 16
    z, q, H0, D0 = _parts(n, g, 8)
    fd = fields_dev(Fo)
    prm = F.push_params(DT, scheme=F.FPIC_HYB1, implicit=F.FPIC_IMR, thr=THR, r_max=float(g.rn[-1]), B0pot=1.0,
                        imr_newton=newton)
    p = make_particles(z, q, H0, D0, H0.copy())
    cfg = L.fit_cfg(ctx, p, fd, prm, mode=F.FPIC_LEARN_CORRECT)
    X, T, S = L.generate(ctx, p, fd, prm, cfg, steps=10)
    assert X.shape[0] > 10000 and float(S.min()) == 1.0
    net, P, hist = L.train(X, T, S, steps=2500, batch=8192, lr=3e-3, log_every=500)
    assert hist[-1][1] < hist[0][1]
    zs = p.state().cpu().numpy(); Hn = p.Hn.cpu().numpy(); al = p.alive.cpu().numpy()
    pp = make_particles(zs, q, H0, D0, Hn.copy(), al.copy())
    pl = make_particles(zs, q, H0, D0, Hn.copy(), al.copy())
    st_p = F.fpic_push(ctx, pp, fd, prm, stats=True)
    st_l = F.fpic_push_learned(ctx, net, pl, fd, prm, cfg, stats=True)
    zp, _, alp, sp, ip, _ = to_np(pp)
    zl, Hl, alv, sl, il, _ = to_np(pl)
    assert np.array_equal(sp, sl) and np.array_equal(alp, alv)
    assert st_l["n_implicit"] == st_p["n_implicit"]
    live = al == 1
    assert (np.abs(zl - zp) / (np.abs(zp) + 1))[live].max() <= 1e-12
    imp = (sl == 1) & live
    po = O.push_params(a=A, dt=DT, scheme=O.IMR, field_kind=O.FIELD_GRID, r_max=g.rn[-1], B0pot=1.0,
                       imr_newton=newton)
    zi = np.ascontiguousarray(zs[imp]); Hi = Hn[imp].copy()
    O.push(po, zi, q[imp], H0[imp], D0[imp], Hi, np.ones(imp.sum(), np.uint8), g, Fo)
    assert (np.abs(zl[imp] - zi) / (np.abs(zi) + 1)).max() <= 1e-12
    # the leading-order term alone (network output zero) as the reference
    net0 = F.MLP()
    net0.set_params(torch.zeros_like(P))
    p0 = make_particles(zs, q, H0, D0, Hn.copy(), al.copy())
    st_0 = F.fpic_push_learned(ctx, net0, p0, fd, prm, cfg, stats=True)
    assert np.array_equal(to_np(p0)[3], sp)
    it_p = st_p["n_iter_total"] / st_p["n_implicit"]
    it_0 = st_0["n_iter_total"] / st_0["n_implicit"]
    it_l = st_l["n_iter_total"] / st_l["n_implicit"]
    print("IMR iterations per implicit step: plain %.3f leading-order %.3f learned %.3f" % (it_p, it_0, it_l))
    assert it_l < it_p and it_0 < it_p, (it_l, it_0, it_p)
