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
