"""Pins of the oracle's equations of motion, pushers and hybrid switch against
what the paper and the mathematics fix (no GPU)."""
import math

import numpy as np
import pytest

import oracle as O
from conftest import golden
from paper_2602_07452_gb300 import inputs as I


def _fd_grad(fun, z, h=1e-4):
    g = np.zeros(6)
    for k in range(6):
        e = np.zeros(6)
        e[k] = h
        g[k] = (4 * (fun(z + e / 2) - fun(z - e / 2)) / h - (fun(z + e) - fun(z - e)) / (2 * h)) / 3
    return g


def _H(a, qm=0.0, B0=0.0):
    return lambda z: O.hamiltonian(1.0, a, B0, z[None, :], qm)[0][0]


@pytest.mark.parametrize("a", [0.0, 0.9, 0.999])
def test_geodesic_rhs_is_hamiltons_equations(a):
    """Eqs. (p1)-(p2): dx/dt = dH/du, du/dt = -dH/dx (q = 0), checked against
    finite differences of H."""
    rng = np.random.default_rng(11)
    for _ in range(8):
        z = np.array([rng.uniform(1.6, 30), rng.uniform(0.2, 2.9), rng.uniform(0, 6),
                      rng.normal(), rng.normal() * 3, rng.normal() * 3])
        f = O.rhs(1.0, a, z, 0.0)[0]
        g = _fd_grad(_H(a), z)
        exp = np.concatenate([g[3:], -g[:3]])
        assert np.abs(f - exp).max() < 1e-8 * (np.abs(exp).max() + 1)


@pytest.mark.parametrize("a", [0.0, 0.7, 0.9])
@pytest.mark.parametrize("qm", [-100.0, 1.0, 100.0])
def test_conserved_H_L_in_exact_wald_field(a, qm):
    """Sec. 3.1.3: in the static Wald field H = -u_0 - (q/m) A_0 and
    L = u_ph + (q/m) A_ph are integrals of the motion, so grad H . dz/dt = 0
    and grad L . dz/dt = 0 pointwise (pins the Lorentz force and its signs)."""
    rng = np.random.default_rng(12)
    B0 = 1.0
    for _ in range(6):
        z = np.array([rng.uniform(1.9, 20), rng.uniform(0.2, 2.9), 0.3,
                      rng.normal(), rng.normal() * 2, rng.normal() * 2])
        _, _, D, _, _ = O.wald(a, B0, z[:1], z[1:2])
        B = O.wald(a, B0, z[:1], z[1:2])[0]
        f = O.rhs(1.0, a, z, qm, D, B)[0]
        gH = _fd_grad(lambda y: O.hamiltonian(1.0, a, B0, y[None, :], qm)[0][0], z)
        gL = _fd_grad(lambda y: O.hamiltonian(1.0, a, B0, y[None, :], qm)[1][0], z)
        sH = np.abs(gH * f).sum()
        sL = np.abs(gL * f).sum()
        assert abs(gH @ f) < 1e-8 * sH
        assert abs(gL @ f) < 1e-8 * sL


def _run(p, z0, steps, qm=0.0, g=None, F=None):
    z = np.ascontiguousarray(np.atleast_2d(z0).astype(float))
    n = z.shape[0]
    qmv = np.full(n, qm)
    H0, _, D0 = O.hamiltonian(p.M, p.a, p.B0pot, z, qmv)
    Hn = H0.copy()
    alive = np.ones(n, np.uint8)
    for _ in range(steps):
        O.push(p, z, qmv, H0, D0, Hn, alive, g, F)
    return z, H0, Hn, alive


def _kerr_orbit_state():
    return np.array([8.0, 1.2, 0.0, 0.05, 0.4, 3.3])


def _ref(a, z0, T):
    p = O.push_params(a=a, dt=T / 4000, scheme=O.RK4)
    return _run(p, z0, 4000)[0][0]


@pytest.mark.parametrize("scheme,order", [(O.RK4, 4), (O.IMR, 2), (O.HAM, 2)])
def test_convergence_order(scheme, order):
    """RK4 is 4th order (Sec. 2.2.1); the IMR and the discrete-gradient scheme
    are 2nd order (Secs. 2.2.2, 2.2.3).  Global error at fixed T, dt halved."""
    a, T = 0.9, 4.0
    z0 = _kerr_orbit_state()
    ref = _ref(a, z0, T)
    errs = []
    for nsteps in (20, 40, 80):
        p = O.push_params(a=a, dt=T / nsteps, scheme=scheme)
        z = _run(p, z0, nsteps)[0][0]
        errs.append(np.abs(z - ref).max())
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(abs(q - order) < 0.35 for q in rates), rates


@pytest.mark.parametrize("scheme", [O.IMR, O.HAM])
def test_implicit_schemes_are_time_symmetric(scheme):
    """Both implicit schemes are symmetric: a step of +dt followed by -dt
    returns to the start (to the iteration tolerance)."""
    z0 = _kerr_orbit_state()
    p = O.push_params(a=0.9, dt=0.3, scheme=scheme, tol=1e-15)
    z1 = _run(p, z0, 1)[0]
    p2 = O.push_params(a=0.9, dt=-0.3, scheme=scheme, tol=1e-15, r_max=1e300)
    z2 = _run(p2, z1[0], 1)[0][0]
    assert np.abs(z2 - z0).max() < 1e-12


@pytest.mark.parametrize("a", [0.0, 0.9, 0.995])
@pytest.mark.parametrize("dt", [0.01, 0.3, 1.0])
def test_discrete_gradient_conserves_H_exactly(a, dt):
    """Sec. 2.2.3: the Hamiltonian scheme conserves H to round-off for any dt
    (the paper reports |dH|/H <~ 1e-15); u_ph never changes."""
    z0 = np.array([9.0, 1.4, 0.0, 0.12, 0.3, 3.1])
    p = O.push_params(a=a, dt=dt, scheme=O.HAM, tol=1e-15)
    z, H0, Hn, alive = _run(p, z0, 30)
    assert alive[0] == 1
    assert abs(Hn[0] - H0[0]) / H0[0] < 2e-14
    assert z[0, 5] == z0[5]


def test_discrete_gradient_identity():
    """Each telescoped ordering satisfies sum G_v (z1_v - z0_v) = H(z1) - H(z0);
    so does the symmetrised average."""
    rng = np.random.default_rng(5)
    for a in (0.0, 0.9):
        for _ in range(10):
            z0 = np.array([rng.uniform(3, 15), rng.uniform(0.4, 2.7), 0.1,
                           rng.normal() * 0.3, rng.normal(), 2 + rng.random()])
            z1 = z0 + rng.normal(size=6) * 0.05
            z1[5] = z0[5]
            G = O.dg_grad(1.0, a, z0, z1)
            dH = _H(a)(z1) - _H(a)(z0)
            assert abs(G @ (z1 - z0) - dH) < 1e-14


def test_table_c1_neutral_orbits_energy_drift():
    """Sec. 3.1.1 / Fig. part0: the three neutral orbits of Table C.1 keep H
    at round-off with the Hamiltonian scheme (dt = 0.1) and at small drift
    with RK4 over t = 200 M."""
    for name, (a, E, L, r0, ur, ut, up) in golden("table_c1_neutral.txt"):
        z0 = np.array([r0, math.pi / 2, 0.0, ur, ut, up])
        pH = O.push_params(a=a, dt=0.1, scheme=O.HAM, tol=1e-15)
        _, H0, Hn, _ = _run(pH, z0, 2000)
        assert abs(Hn[0] - H0[0]) / H0[0] < 1e-13, name
        pR = O.push_params(a=a, dt=0.1, scheme=O.RK4)
        _, H0, Hn, _ = _run(pR, z0, 2000)
        assert abs(Hn[0] - H0[0]) / H0[0] < 1e-6, name


def _circular(a, r):
    """Bardeen, Press & Teukolsky (1972): prograde equatorial circular orbit."""
    s = r ** 1.5 - 3 * r ** 0.5 + 2 * a
    E = (r ** 1.5 - 2 * r ** 0.5 + a) / (r ** 0.75 * math.sqrt(s))
    L = (r * r - 2 * a * r ** 0.5 + a * a) / (r ** 0.75 * math.sqrt(s))
    Om = 1.0 / (r ** 1.5 + a)
    return E, L, Om


@pytest.mark.parametrize("a,r", [(0.9, 6.0), (0.9, 3.0), (0.0, 8.0)])
def test_circular_orbit_closed_form(a, r):
    """Kerr circular equatorial orbits (textbook closed forms; KS and BL share
    r, E = -u_t, L = u_ph and dph/dt at fixed r): the orbit seeded with dr/dt = 0
    stays at r and advances ph at Omega.  Printed values (a=0.9, r=6):
    E=0.922599626, L=2.794278361, Omega=0.064115147."""
    E, L, Om = _circular(a, r)
    if (a, r) == (0.9, 6.0):
        assert abs(E - 0.922599626) < 1e-9 and abs(L - 2.794278361) < 1e-9
        assert abs(Om - 0.064115147) < 1e-9
    m = O.metric(1.0, a, [r], [math.pi / 2])[0]
    al2, be, grr, grp = m[2] ** 2, m[3], m[8], m[9]
    ur = (be * E - al2 * grp * L) / (al2 * grr - be * be)      # dr/dt = 0
    z0 = np.array([r, math.pi / 2, 0.0, ur, 0.0, L])
    assert abs(_H(a)(z0) - E) < 1e-13
    T = 100.0
    p = O.push_params(a=a, dt=0.02, scheme=O.RK4)
    z, H0, Hn, _ = _run(p, z0, int(T / 0.02))
    assert abs(z[0, 0] - r) < 1e-6 * r
    assert abs(z[0, 2] - Om * T) < 1e-6 * Om * T
    assert abs(z[0, 1] - math.pi / 2) < 1e-12


def _kappa_r(a, r):
    """Radial epicyclic frequency of a prograde circular equatorial Kerr orbit
    in coordinate time (M = 1; e.g. Okazaki, Kato & Fukue 1987):
    kappa_r^2 = Omega^2 (1 - 6/r + 8 a / r^1.5 - 3 a^2 / r^2)."""
    Om = 1.0 / (r ** 1.5 + a)
    return Om * math.sqrt(1 - 6 / r + 8 * a / r ** 1.5 - 3 * a * a / (r * r))


def _isco(a):
    """Bardeen, Press & Teukolsky (1972): prograde ISCO radius (M = 1)."""
    z1 = 1 + (1 - a * a) ** (1 / 3) * ((1 + a) ** (1 / 3) + (1 - a) ** (1 / 3))
    z2 = math.sqrt(3 * a * a + z1 * z1)
    return 3 + z2 - math.sqrt((3 - z1) * (3 + z1 + 2 * z2))


def _circular_state(a, r):
    E, L, Om = _circular(a, r)
    m = O.metric(1.0, a, [r], [math.pi / 2])[0]
    al2, be, grr, grp = m[2] ** 2, m[3], m[8], m[9]
    ur = (be * E - al2 * grp * L) / (al2 * grr - be * be)      # dr/dt = 0
    return np.array([r, math.pi / 2, 0.0, ur, 0.0, L])


def _radial_jacobian(a, r):
    """Linearisation of the oracle's right-hand side (Eqs. p1, p2) in the
    (r, u_r) plane about the circular orbit (th = pi/2, u_th = 0, u_ph = L
    fixed; ph does not enter): central differences of dr/dt and du_r/dt."""
    z0 = _circular_state(a, r)
    J = np.zeros((2, 2))
    for col, k in enumerate((0, 3)):
        h = 1e-5 * (abs(z0[k]) + 1.0)
        zp, zm = z0.copy(), z0.copy()
        zp[k] += h
        zm[k] -= h
        d = (O.rhs(1.0, a, zp, 0.0)[0] - O.rhs(1.0, a, zm, 0.0)[0]) / (2 * h)
        J[:, col] = d[[0, 3]]
    return z0, J


@pytest.mark.parametrize("a,r", [(0.9, 6.0), (0.9, 3.0), (0.0, 8.0), (0.5, 5.0)])
def test_radial_epicyclic_frequency(a, r):
    """App. A metric through Eqs. (p1)-(p2) at second order: the circular
    orbit is a fixed point of the (r, u_r) flow, and the linearised flow
    about it oscillates at the closed-form radial epicyclic frequency
    (eigenvalues +-i kappa_r: zero trace, determinant kappa_r^2).  Printed
    values (a = 0.9): kappa_r = 0.041669812 at r = 6, 0.055782688 at r = 3."""
    if (a, r) == (0.9, 6.0):
        assert abs(_kappa_r(a, r) - 0.041669812) < 1e-9
    if (a, r) == (0.9, 3.0):
        assert abs(_kappa_r(a, r) - 0.055782688) < 1e-9
    z0, J = _radial_jacobian(a, r)
    f0 = O.rhs(1.0, a, z0, 0.0)[0]
    assert abs(f0[0]) < 1e-14 and abs(f0[3]) < 1e-14
    k = _kappa_r(a, r)
    assert abs(np.trace(J)) < 1e-8 * k
    assert abs(math.sqrt(np.linalg.det(J)) - k) < 1e-7 * k, (math.sqrt(np.linalg.det(J)), k)


def test_radial_oscillation_period_of_a_perturbed_circular_orbit():
    """A circular orbit (a = 0.9, r = 6) kicked radially (u_r + 1e-4) and
    pushed with RK4 (dt = 0.1) oscillates in r with period 2 pi / kappa_r
    (upward crossings of its mean radius over two periods, 1e-4 relative)."""
    a, r, dt = 0.9, 6.0, 0.1
    z = np.ascontiguousarray(_circular_state(a, r)[None, :])
    z[0, 3] += 1e-4
    p = O.push_params(a=a, dt=dt, scheme=O.RK4)
    qm = np.zeros(1)
    H0, _, D0 = O.hamiltonian(1.0, a, 0.0, z, qm)
    Hn, alive = H0.copy(), np.ones(1, np.uint8)
    T = 2.0 * math.pi / _kappa_r(a, r)
    rs = [z[0, 0]]
    for _ in range(int(2.3 * T / dt)):
        O.push(p, z, qm, H0, D0, Hn, alive)
        rs.append(z[0, 0])
    rs = np.array(rs)
    x = rs - 0.5 * (rs.max() + rs.min())
    up = np.nonzero((x[:-1] < 0) & (x[1:] >= 0))[0]
    tc = (up + x[up] / (x[up] - x[up + 1])) * dt
    assert len(tc) >= 2
    period = (tc[-1] - tc[0]) / (len(tc) - 1)
    assert abs(period - T) < 1e-4 * T, (period, T)


@pytest.mark.parametrize("a", [0.0, 0.5, 0.9])
def test_isco_is_where_the_radial_restoring_force_vanishes(a):
    """The innermost stable circular orbit is where the oracle's linearised
    radial flow stops oscillating (det J = kappa_r^2 changes sign): found by
    bisection on the oracle's right-hand side, it equals the Bardeen-Press-
    Teukolsky radius (printed: 2.320883 for a = 0.9; 6 for a = 0)."""
    rI = _isco(a)
    if a == 0.9:
        assert abs(rI - 2.320883) < 1e-6
    if a == 0.0:
        assert abs(rI - 6.0) < 1e-12
    lo, hi = rI - 0.3, rI + 0.3
    assert np.linalg.det(_radial_jacobian(a, lo)[1]) < 0 < np.linalg.det(_radial_jacobian(a, hi)[1])
    for _ in range(40):
        mid = 0.5 * (lo + hi)
        if np.linalg.det(_radial_jacobian(a, mid)[1]) < 0:
            lo = mid
        else:
            hi = mid
    assert abs(0.5 * (lo + hi) - rI) < 1e-6, (0.5 * (lo + hi), rI)


def test_charged_orbit_exact_wald_conserves_H_L():
    """Sec. 3.1.3: charged orbits (Table C.1 RKA initial states) in the exact
    Wald field conserve H and L; RK4 at dt = 1e-3 keeps both to ~1e-10."""
    for name, (a, B0, r0, dth, ur, ut, up) in golden("table_c1_charged.txt"):
        z0 = np.array([r0, math.pi / 2 - dth, 0.0, ur, ut, up])
        p = O.push_params(a=a, dt=1e-3, scheme=O.RK4, B0pot=B0, field_kind=O.FIELD_WALD,
                          B0field=B0)
        z, H0, Hn, alive = _run(p, z0, 3000, qm=1.0)
        assert alive[0] == 1
        L0 = O.hamiltonian(1.0, a, B0, z0[None, :], 1.0)[1][0]
        L1 = O.hamiltonian(1.0, a, B0, z, 1.0)[1][0]
        assert abs(Hn[0] - H0[0]) < 1e-10 * abs(H0[0]), name
        assert abs(L1 - L0) < 1e-10 * abs(L0), name


def test_interpolation_dominates_charged_error():
    """Sec. 3.1.3 (Fig. 3d discussion): with the Wald field sampled on the grid
    the H error is set by the interpolation: it falls with the resolution N
    and does not change when dt is halved."""
    a, B0 = 0.9, 1.0
    z0 = np.array([6.0, 1.2, 0.0, 0.3, 0.5, 0.8])
    errs = {}
    for N in (64, 128, 256):
        g = I.log_grid(N, N, 1.3, 12.0)
        F = O.wald_on_grid(a, B0, g)
        for dt in (2e-3, 1e-3):
            p = O.push_params(a=a, dt=dt, scheme=O.RK4, B0pot=B0, field_kind=O.FIELD_GRID)
            _, H0, Hn, _ = _run(p, z0, int(round(2.0 / dt)), qm=10.0, g=g, F=F)
            errs[N, dt] = abs(Hn[0] - H0[0])
    assert errs[64, 1e-3] > 1.8 * errs[128, 1e-3] > 1.8 * 1.8 * errs[256, 1e-3]
    for N in (64, 128, 256):
        assert abs(errs[N, 1e-3] - errs[N, 2e-3]) < 0.01 * errs[N, 1e-3]


def test_gather_exact_for_bilinear_fields():
    """The (r, th)-bilinear gather reproduces fields bilinear in (r, th) on every
    staggered sub-grid, and extrapolates as a constant beyond the end nodes."""
    g = I.log_grid(13, 9, 1.5, 30.0)
    F = []
    coef = [(0.3, -1.2, 0.7, 0.05), (1.0, 0.2, -0.4, 0.3), (-0.5, 0.1, 0.9, -0.2),
            (2.0, 0.0, 1.0, 0.1), (0.1, 0.3, 0.0, 0.5), (0.0, -0.7, 0.2, 0.02)]
    roff, toff = [1, 0, 0, 0, 1, 1], [0, 1, 0, 1, 0, 1]
    for k in range(6):
        X = g.rh if roff[k] else g.rn
        Y = g.th if toff[k] else g.tn
        f = np.zeros((g.Nr + 1, g.ld))
        c = coef[k]
        f[:X.size, :Y.size] = c[0] + c[1] * X[:, None] + c[2] * Y[None, :] + c[3] * X[:, None] * Y[None, :]
        F.append(f.ravel())
    rng = np.random.default_rng(3)
    r = rng.uniform(g.rh[0], g.rh[-1], 200)
    t = rng.uniform(g.th[0], g.th[-1], 200)
    out = O.gather(g, F, r, t)
    for k in range(6):
        c = coef[k]
        exp = c[0] + c[1] * r + c[2] * t + c[3] * r * t
        assert np.abs(out[:, k] - exp).max() < 1e-12
    # constant extrapolation below the first half node in r
    t0 = g.th[0]
    o2 = O.gather(g, F, np.array([g.rn[0]]), np.array([t0]))
    c = coef[4]
    assert abs(o2[0, 4] - (c[0] + c[1] * g.rh[0] + c[2] * t0 + c[3] * g.rh[0] * t0)) < 1e-12


def test_cell_index_brute_force():
    """Cell location: the cell (i, j) with r_i <= r < r_{i+1}, th_j <= th <
    th_{j+1} (clamped), found by exhaustive search over the nodes; points on
    nodes belong to the upper cell."""
    g = I.log_grid(7, 5, 1.2, 9.0)
    rng = np.random.default_rng(4)
    r = np.concatenate([rng.uniform(0.5, 12, 300), g.rn, g.rn[:-1] * (1 + 1e-16)])
    t = np.concatenate([rng.uniform(-0.1, 3.3, 300), rng.choice(g.tn, g.rn.size), rng.choice(g.tn, g.rn.size - 1)])
    got = O.cell_index(g, r, t)
    for k in range(r.size):
        i = max([ii for ii in range(g.Nr) if g.rn[ii] <= r[k]] or [0])
        j = max([jj for jj in range(g.Nth) if g.tn[jj] <= t[k]] or [0])
        assert got[k] == i * g.Nth + j


@pytest.mark.parametrize("scheme", [O.HYB1, O.HYB2])
def test_hybrid_choice_equals_brute_force(scheme):
    """Sec. 3.1.2: the hybrid accepts the RK4 trial iff its H-violation test
    passes (Hyb2: Ht < Ht_max; Hyb1: dHt/dt < max) and otherwise returns the
    implicit step from z^n (here the discrete-gradient scheme, which then
    leaves H where it was); recomputed from separate RK4 pushes and H."""
    a, dt = 0.9, 0.5
    cand = I.orbit_candidates(64, seed=9)
    z0, bad = O.seed_orbits(1.0, a, cand)
    assert bad == 0
    n = z0.shape[0]
    qm = np.zeros(n)
    H0, _, D0 = O.hamiltonian(1.0, a, 0.0, z0, qm)
    Hprev = H0 * (1 + 1e-10 * np.sin(np.arange(n)))
    pr = O.push_params(a=a, dt=dt, scheme=O.RK4)
    zr = z0.copy(); Hr = Hprev.copy()
    O.push(pr, zr, qm, H0, D0, Hr, np.ones(n, np.uint8))
    Ht1 = np.abs(Hr - H0) / D0
    stat = Ht1 if scheme == O.HYB2 else (Ht1 - np.abs(Hprev - H0) / D0) / dt
    thr = float(np.median(stat))
    acc = stat < thr
    ph = O.push_params(a=a, dt=dt, scheme=scheme, implicit_kind=O.HAM, thr=thr, tol=1e-15)
    zh = z0.copy(); Hh = Hprev.copy()
    _, sch, its = O.push(ph, zh, qm, H0, D0, Hh, np.ones(n, np.uint8))
    assert np.array_equal(sch == 0, acc)
    assert 0 < acc.sum() < n
    assert np.array_equal(zh[acc], zr[acc])
    assert np.abs(Hh[~acc] - H0[~acc]).max() < 1e-14 * np.abs(H0).max()
    assert np.all(its[~acc] > 0) and np.all(its[acc] == 0)


def test_seeding_orbits_and_fido():
    """Seeding: orbit candidates give H = E exactly (to round-off) with
    u_th = 0, u_ph = L; FIDO-frame momenta give Gamma = sqrt(1 + |uhat|^2)."""
    cand = I.orbit_candidates(256, seed=1)
    z, bad = O.seed_orbits(1.0, 0.9, cand)
    assert bad == 0
    H = O.hamiltonian(1.0, 0.9, 0.0, z, 0.0)[0]
    Es = np.array([cand[p, [k for k in range(cand.shape[1])
                            if abs(cand[p, k, 0] - z[p, 0]) == 0][0], 2] for p in range(256)])
    assert np.abs(H - Es).max() < 1e-12
    g = I.wald_grid(32, 0.9)
    d, q, w = I.thermal_draws(500, g, 1.6, 40.0, 0.1, seed=3)
    zf = O.seed_fido(1.0, 0.9, d)
    m = O.metric(1.0, 0.9, zf[:, 0], zf[:, 1])
    u = zf[:, 3:]
    quad = m[:, 8] * u[:, 0] ** 2 + 2 * m[:, 9] * u[:, 0] * u[:, 2] + m[:, 10] * u[:, 1] ** 2 + m[:, 11] * u[:, 2] ** 2
    assert np.allclose(quad, (d[:, 3:] ** 2).sum(1), rtol=1e-12, atol=1e-15)


def test_particle_boundaries():
    """Sec. 2.5: particles inside r_h or beyond r_max are removed; crossing a
    pole reflects (th -> -th, u_th -> -u_th, ph -> ph + pi)."""
    a = 0.5
    z = np.array([[1.5, 0.3, 0.0, -3.0, 0.0, 0.0],       # falls in
                  [6.0, 0.002, 0.0, 0.0, -2.0, 0.0],     # crosses th = 0
                  [19.99, 1.0, 0.0, 5.0, 0.0, 0.0]])     # leaves r_max = 20
    p = O.push_params(a=a, dt=0.1, scheme=O.RK4, r_max=20.0)
    z1, _, _, alive = _run(p, z, 3)
    assert alive.tolist() == [0, 1, 0]
    assert z1[1, 1] > 0 and z1[1, 4] > 0 and abs(z1[1, 2] - math.pi) < 1e-3


@pytest.mark.parametrize("partner,charged", [(O.IMR, False), (O.HAM, False), (O.IMR, True)])
def test_adaptive_implicit_step_is_the_standalone_step(partner, charged):
    """Sec. 3.1.2 / Tab. C.2 adaptive steps: a hybrid whose test rejects every
    trial returns, for every particle, the standalone implicit step of size
    dt_imp from z^n (independently started at z^n), to the iteration
    tolerance; a test that accepts everything returns the RK4 step of size
    dt, whatever dt_imp; dt_imp = dt is bit-identical to dt_imp = 0."""
    a, dt, dti = 0.9, 0.05, 0.15
    if charged:
        d, q, _ = I.thermal_draws(48, I.log_grid(8, 8, 1.5, 30.0), 3.0, 12.0, 0.1, seed=4, qm=1.0)
        z0 = O.seed_fido(1.0, a, d)
        kw = dict(field_kind=O.FIELD_WALD, B0field=1.0, B0pot=1.0)
    else:
        # generic bound states away from turning points (u_th != 0), where
        # the discrete-gradient iteration reaches 1e-14
        rng = np.random.default_rng(12)
        m_ = 48
        z0 = np.stack([rng.uniform(6, 12, m_), rng.uniform(0.8, 2.3, m_), np.zeros(m_), rng.uniform(-0.1, 0.1, m_),
                       rng.choice([-1, 1], m_) * rng.uniform(0.1, 0.4, m_), rng.uniform(2.5, 3.5, m_)], 1)
        q = np.zeros(m_)
        kw = {}
    n = z0.shape[0]
    H0, _, D0 = O.hamiltonian(1.0, a, kw.get("B0pot", 0.0), z0, q)

    def run(**p):
        z = z0.copy(); Hn = H0.copy(); al = np.ones(n, np.uint8)
        _, sch, its = O.push(O.push_params(a=a, tol=1e-14, **kw, **p), z, q, H0, D0, Hn, al)
        return z, sch, al

    z_rej, sch, al = run(dt=dt, scheme=O.HYB2, implicit_kind=partner, thr=-1.0, dt_imp=dti)
    z_ref, _, al2 = run(dt=dti, scheme=partner)
    assert np.all(sch == 1) and np.array_equal(al, al2) and al.sum() > 0.8 * n
    m = al == 1
    assert (np.abs(z_rej[m] - z_ref[m]) / (np.abs(z_ref[m]) + 1)).max() < 1e-12
    z_acc, sch, _ = run(dt=dt, scheme=O.HYB2, implicit_kind=partner, thr=1e300, dt_imp=dti)
    z_rk4, _, _ = run(dt=dt, scheme=O.RK4)
    assert np.all(sch == 0) and np.array_equal(z_acc, z_rk4)
    thr = 1e-13
    za, _, _ = run(dt=dt, scheme=O.HYB2, implicit_kind=partner, thr=thr, dt_imp=dt)
    zb, _, _ = run(dt=dt, scheme=O.HYB2, implicit_kind=partner, thr=thr, dt_imp=0.0)
    assert np.array_equal(za, zb)


@pytest.mark.parametrize("a", [0.0, 0.9, 0.995])
def test_dg_quotient_closed_form(a):
    """Appendix D quotients in closed form: for a single-variable move the
    value equals the plain difference quotient (H(za) - H(zb)) / dz of the
    Appendix A Hamiltonian at increments where that quotient is accurate
    (|dz| = 1e-3: rounding ~1e-13), and tends to the partial derivative of
    Hamilton's equations (Eqs. p1, p2 with q = 0) at |dz| = 1e-12, where the
    plain quotient has lost all digits; the ph move gives 0."""
    rng = np.random.default_rng(int(a * 1000) + 3)
    H = _H(a)
    for _ in range(20):
        zb = np.array([rng.uniform(1.5 * (1 + math.sqrt(1 - a * a)), 15), rng.uniform(0.3, 2.8), 0.2,
                       rng.normal() * 0.5, rng.normal(), rng.normal() * 3])
        f = O.rhs(1.0, a, zb[None, :], 0.0)[0]
        partial = {0: -f[3], 1: -f[4], 3: f[0], 4: f[1], 5: f[2]}
        for v in (0, 1, 3, 4, 5):
            za = zb.copy(); za[v] += 1e-3 * (1 + abs(zb[v]))
            plain = (H(za) - H(zb)) / (za[v] - zb[v])
            q = O.dg_quot(1.0, a, zb, za, v)
            # the plain quotient's own rounding: a few ulp(H) / |dz|
            assert abs(q - plain) <= 1e-10 * abs(plain) + 4e-16 * max(1.0, abs(H(zb))) / abs(za[v] - zb[v]), \
                (v, q, plain)
            za = zb.copy(); za[v] += 1e-12
            q = O.dg_quot(1.0, a, zb, za, v)
            # O(dz) = 1e-12 from the second derivative
            assert abs(q - partial[v]) <= 1e-10 * abs(partial[v]) + 1e-11, (v, q, partial[v])
        za = zb.copy(); za[2] += 0.3
        assert O.dg_quot(1.0, a, zb, za, 2) == 0.0


def test_dg_converges_from_turning_points():
    """Bound orbits seeded at a th turning point (u_th = 0, where th moves by
    tiny increments): the closed-form quotients let every discrete-gradient
    solve converge to 1e-15 within a few iterations and conserve H to
    rounding."""
    a = 0.9
    z0, bad = O.seed_orbits(1.0, a, I.orbit_candidates(48, seed=12))
    assert bad == 0
    n = z0.shape[0]
    q = np.zeros(n)
    H0, _, D0 = O.hamiltonian(1.0, a, 0.0, z0, q)
    z = z0.copy(); Hn = H0.copy(); al = np.ones(n, np.uint8)
    for _ in range(5):
        nc, sch, its = O.push(O.push_params(a=a, dt=0.15, scheme=O.HAM, tol=1e-15), z, q, H0, D0, Hn, al)
        assert nc == 0 and its.max() <= 12
    assert np.abs(Hn - H0).max() <= 4e-15 * np.abs(H0).max()


# ---- discrete-gradient scheme for charged particles in the Wald field (extension) ----

def _Hc(a, B0, qm):
    """H_c(x, pi) = H(x, u) with u = pi - (q/m) A (Eq. Amu), via the oracle's H."""
    def f(w):
        Ar, Aph = O.wald_A(a, B0, [w[0]], [w[1]])
        z = w.copy(); z[3] -= qm * Ar[0]; z[5] -= qm * Aph[0]
        return O.hamiltonian(1.0, a, B0, z[None, :], np.array([qm]))[0][0]
    return f


@pytest.mark.parametrize("a", [0.0, 0.7, 0.9])
def test_charged_dg_quotient_closed_form(a):
    """Canonical-variable quotients for a charged particle in the Wald field:
    equal to the plain difference quotient of H_c at dz = 1e-3, and at
    dz = 1e-12 to the partial derivatives that the Lorentz-force equations
    (Eqs. p1, p2, O1, O2 with the App. B field) imply, d pi_i / dt = du_i/dt +
    (q/m) dA_i/dt, with the potential derivatives by central differences: this
    ties A_r, A_ph, A_0 of Eq. (Amu) to the field the RHS uses."""
    B0, qm = 1.0, 1.5
    rng = np.random.default_rng(int(a * 100) + 7)
    Hc = _Hc(a, B0, qm)
    for _ in range(12):
        w = np.array([rng.uniform(2.5, 10), rng.uniform(0.4, 2.7), 0.3,
                      rng.normal() * 0.5, rng.normal(), rng.normal() * 3])
        Ar, Aph = O.wald_A(a, B0, [w[0]], [w[1]])
        z = w.copy(); z[3] -= qm * Ar[0]; z[5] -= qm * Aph[0]
        _, _, D, _, _ = O.wald(a, B0, [z[0]], [z[1]])
        Bw = O.wald(a, B0, [z[0]], [z[1]])[0]
        f = O.rhs(1.0, a, z[None, :], qm, D, Bw)[0]
        h = 1e-6
        dA = {}
        for k in (0, 1):
            e = np.zeros(2); e[k] = h
            p1 = O.wald_A(a, B0, [w[0] + e[0]], [w[1] + e[1]])
            m1 = O.wald_A(a, B0, [w[0] - e[0]], [w[1] - e[1]])
            dA[k] = ((p1[0][0] - m1[0][0]) / (2 * h), (p1[1][0] - m1[1][0]) / (2 * h))
        dpir = f[3] + qm * (dA[0][0] * f[0] + dA[1][0] * f[1])
        dpit = f[4]
        partial = {0: None, 1: None, 3: f[0], 4: f[1], 5: f[2]}
        # dH/dr|pi = -dpi_r/dt, dH/dth|pi = -dpi_th/dt
        partial[0] = -dpir
        partial[1] = -dpit
        for v in (0, 1, 3, 4, 5):
            wa = w.copy(); wa[v] += 1e-3 * (1 + abs(w[v]))
            plain = (Hc(wa) - Hc(w)) / (wa[v] - w[v])
            q = O.dg_quot_em(1.0, a, B0, qm, w, wa, v)
            assert abs(q - plain) <= 1e-10 * abs(plain) + 4e-16 * max(1.0, abs(Hc(w))) / abs(wa[v] - w[v]), (v, q, plain)
            wa = w.copy(); wa[v] += 1e-12
            q = O.dg_quot_em(1.0, a, B0, qm, w, wa, v)
            assert abs(q - partial[v]) <= 1e-7 * (abs(partial[v]) + 1.0), (v, q, partial[v])


def _wald_charged_states(a, n, seed):
    rng = np.random.default_rng(seed)
    return np.stack([rng.uniform(4, 9, n), rng.uniform(0.7, 2.4, n), np.zeros(n),
                     rng.normal(size=n) * 0.3, rng.normal(size=n) * 0.5, rng.normal(size=n) * 2], 1)


def test_charged_dg_conserves_H_and_L_and_converges_to_the_lorentz_force():
    """In the exact Wald field the canonical discrete-gradient scheme keeps
    H (Sec. 3.1.3) to rounding and L = u_ph + (q/m) A_ph exactly for any dt,
    and its trajectory converges at second order to the RK4 solution of the
    Lorentz-force equations (Eqs. p1, p2, O1, O2) in the same field."""
    a, B0, qm = 0.9, 1.0, 2.0
    z0 = _wald_charged_states(a, 16, 3)
    n = z0.shape[0]
    q = np.full(n, qm)
    kw = dict(a=a, field_kind=O.FIELD_WALD, B0field=B0, B0pot=B0, tol=1e-15, max_iter=100)
    H0, L0, D0 = O.hamiltonian(1.0, a, B0, z0, q)

    def run(scheme, dt, steps):
        z = z0.copy(); Hn = H0.copy(); al = np.ones(n, np.uint8)
        nc = 0
        for _ in range(steps):
            nc += O.push(O.push_params(dt=dt, scheme=scheme, **kw), z, q, H0, D0, Hn, al)[0]
        return z, Hn, al, nc

    z, Hn, al, nc = run(O.HAM, 0.1, 20)
    assert al.all() and nc == 0
    H1, L1, _ = O.hamiltonian(1.0, a, B0, z, q)
    assert np.abs(H1 - H0).max() <= 1e-14 * np.abs(H0).max()
    assert np.abs(L1 - L0).max() <= 1e-13 * np.abs(L0).max()
    T = 0.8
    ref = run(O.RK4, T / 400, 400)[0]
    errs = [np.abs(run(O.HAM, T / m, m)[0] - ref).max() for m in (20, 40, 80)]
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(abs(r_ - 2) < 0.35 for r_ in rates), (errs, rates)


def _wald_plasma(n, a=0.9, seed=5):
    g = I.wald_grid(64, a)
    d, qm, _ = I.thermal_draws(n, g, 1.02 * I.horizon(1.0, a), 49.0, 0.1, seed=seed, qm=100.0)
    return O.seed_fido(1.0, a, d), qm


def test_imr_newton_blocks_match_finite_differences():
    """The momentum blocks of the IMR Newton matrix (Sec. 2.2.2) are the
    derivatives of the right-hand side (Eqs. p1, p2, O1, O2) with respect
    to u: A = d(dx/dt)/du against central differences of the position rows,
    J against central differences of the momentum rows' field part (the
    right-hand side with the Wald field minus the one without)."""
    a, B0 = 0.9, 1.0
    z, qm = _wald_plasma(64, a)
    B, _, D, _, _ = O.wald(a, B0, z[:, 0], z[:, 1])
    A, J = O.imr_blocks(1.0, a, z, qm, B)
    fdA, fdJ = np.zeros_like(A), np.zeros_like(J)
    for l in range(3):
        h = 1e-5 * (np.abs(z[:, 3 + l]) + 1.0)
        zp, zm = z.copy(), z.copy()
        zp[:, 3 + l] += h
        zm[:, 3 + l] -= h
        fe = O.rhs(1.0, a, zp, qm, D, B) - O.rhs(1.0, a, zm, qm, D, B)
        fg = O.rhs(1.0, a, zp, qm) - O.rhs(1.0, a, zm, qm)
        fdA[:, :, l] = fe[:, :3] / (2 * h)[:, None]
        fdJ[:, :, l] = (fe - fg)[:, 3:] / (2 * h)[:, None]
    assert np.abs(A - fdA).max() < 1e-8 * np.abs(A).max()
    assert np.abs(J - fdJ).max() < 1e-8 * np.abs(J).max()
    # no field: J vanishes, A does not depend on the charge
    A0, J0 = O.imr_blocks(1.0, a, z, qm)
    assert np.array_equal(A0, A) and not J0.any()


@pytest.mark.parametrize("field", ["wald", "grid"])
def test_imr_newton_reaches_the_fixed_point_solution(field):
    """The Newton iteration and the fixed-point update of Eq. (imr2) solve
    the same implicit-midpoint equation: from the same start they stop at
    the same state (to the iteration tolerance), the Newton form in fewer
    iterations for charged particles gyrating in the Wald field."""
    a, B0 = 0.9, 1.0
    z0, qm = _wald_plasma(600, a)
    H0, _, D0 = O.hamiltonian(1.0, a, B0, z0, qm)
    if field == "wald":
        kw, gf = dict(field_kind=O.FIELD_WALD, B0field=B0), {}
    else:
        g = I.wald_grid(64, a)
        kw, gf = dict(field_kind=O.FIELD_GRID), dict(g=g, F=O.wald_on_grid(a, B0, g))
    out = {}
    for newton in (False, True):
        p = O.push_params(a=a, dt=1e-3, scheme=O.IMR, B0pot=B0, tol=1e-14, imr_newton=newton, **kw)
        z = z0.copy()
        Hn, alive = np.zeros(len(z)), np.ones(len(z), np.uint8)
        nc, sch, its = O.push(p, z, qm, H0, D0, Hn, alive, **gf)
        assert nc == 0
        out[newton] = (z, its.astype(float))
    (zf, itf), (zn, itn) = out[False], out[True]
    assert np.abs(zn - zf).max(axis=1).max() < 1e-12 * (np.abs(zf).max() + 1)
    assert itn.mean() < 0.6 * itf.mean() and itn.max() <= 8, (itn.mean(), itf.mean())


def test_imr_newton_keeps_order_and_symmetry():
    """The Newton-solved IMR is the same scheme: second order (global error
    at fixed T with dt halved) and time symmetric (+dt then -dt returns to
    the start) on a Kerr geodesic."""
    a, T = 0.9, 4.0
    z0 = _kerr_orbit_state()
    ref = _ref(a, z0, T)
    errs = []
    for nsteps in (20, 40, 80):
        p = O.push_params(a=a, dt=T / nsteps, scheme=O.IMR, imr_newton=True)
        errs.append(np.abs(_run(p, z0, nsteps)[0][0] - ref).max())
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(abs(q - 2) < 0.35 for q in rates), rates
    p = O.push_params(a=a, dt=0.3, scheme=O.IMR, tol=1e-15, imr_newton=True)
    z1 = _run(p, z0, 1)[0]
    p2 = O.push_params(a=a, dt=-0.3, scheme=O.IMR, tol=1e-15, r_max=1e300, imr_newton=True)
    assert np.abs(_run(p2, z1[0], 1)[0][0] - z0).max() < 1e-12


def test_imr_newton_first_iterates_are_newton_steps():
    """Each Newton iterate of the IMR solve is z - P^-1 R(z) for the residual
    R(z) = z - z^n - dt F((z^n + z)/2) and P = 1 - (dt/2) dF restricted to
    its momentum columns, here built from central differences of the
    right-hand side and solved by numpy: the first two iterates of the
    oracle's solve (max_iter = 1, 2; start z^n) agree with that
    construction far inside the size of the momentum coupling terms."""
    a, B0, dt = 0.9, 1.0, 1e-3
    z0, qm = _wald_plasma(40, a, seed=9)
    H0, _, D0 = O.hamiltonian(1.0, a, B0, z0, qm)

    def F(z):
        B, _, D, _, _ = O.wald(a, B0, z[:, 0], z[:, 1])
        return O.rhs(1.0, a, z, qm, D, B)

    def newton_np(zk):
        y = 0.5 * (z0 + zk)
        R = zk - (z0 + dt * F(y))
        dF = np.zeros((len(y), 6, 3))
        for l in range(3):
            h = 1e-5 * (np.abs(y[:, 3 + l]) + 1.0)
            yp, ym = y.copy(), y.copy()
            yp[:, 3 + l] += h
            ym[:, 3 + l] -= h
            B, _, D, _, _ = O.wald(a, B0, y[:, 0], y[:, 1])   # fields at the midpoint
            fe = O.rhs(1.0, a, yp, qm, D, B) - O.rhs(1.0, a, ym, qm, D, B)
            fg = O.rhs(1.0, a, yp, qm) - O.rhs(1.0, a, ym, qm)
            dF[:, :3, l] = fe[:, :3] / (2 * h)[:, None]
            dF[:, 3:, l] = (fe - fg)[:, 3:] / (2 * h)[:, None]
        P = np.tile(np.eye(6), (len(y), 1, 1))
        P[:, :, 3:] -= 0.5 * dt * dF
        d = np.linalg.solve(P, R[:, :, None])[:, :, 0]
        coup = np.abs(0.5 * dt * np.einsum("nij,nj->ni", dF[:, :3], d[:, 3:]))
        return zk - d, coup, np.abs(d[:, 3:])

    zk = z0.copy()
    for it in (1, 2):
        p = O.push_params(a=a, dt=dt, scheme=O.IMR, B0pot=B0, max_iter=it, imr_newton=True,
                          field_kind=O.FIELD_WALD, B0field=B0)
        z = z0.copy()
        O.push(p, z, qm, H0, D0, np.zeros(len(z)), np.ones(len(z), np.uint8))
        zk, coup, du = newton_np(zk)
        assert (np.abs(z[:, :3] - zk[:, :3]) <= 1e-3 * coup + 1e-15 * (np.abs(zk[:, :3]) + 1)).all(), it
        assert (np.abs(z[:, 3:] - zk[:, 3:]) <= 1e-6 * du + 1e-15 * (np.abs(zk[:, 3:]) + 1)).all(), it


@pytest.mark.parametrize("newton", [False, True])
def test_imr_unconverged_solve_returns_smallest_update_iterate(newton):
    """Reading for a solve stopped by max_iter (the paper gives no policy):
    the result is the iterate whose update max_i |z^[k]_i - z^[k-1]_i| was
    the smallest.  The iterates are rebuilt here from the right-hand side
    and the grid gather (the fixed-point map; for the Newton form only the
    first iterate, which max_iter = 1 returns as is), at a step far too long
    for the map to contract (dt = 0.05, q/m = 100), where the updates grow
    and the first iterate wins over the last."""
    a, B0 = 0.9, 1.0
    g = I.wald_grid(64, a)
    Fo = O.wald_on_grid(a, B0, g)
    z0, qm = _wald_plasma(200, a, seed=13)
    H0, _, D0 = O.hamiltonian(1.0, a, B0, z0, qm)
    dt, m = 0.05, 6

    def push(max_iter):
        p = O.push_params(a=a, dt=dt, scheme=O.IMR, B0pot=B0, max_iter=max_iter, imr_newton=newton,
                          field_kind=O.FIELD_GRID, r_max=1e300)
        z = z0.copy()
        nc, sch, its = O.push(p, z, qm, H0, D0, np.zeros(len(z)), np.ones(len(z), np.uint8), g, Fo)
        return z, nc

    if not newton:
        zk, its, ups = z0.copy(), [], []
        for k in range(m):
            y = 0.5 * (z0 + zk)
            DB = O.gather(g, Fo, y[:, 0], y[:, 1])
            zn = z0 + dt * O.rhs(1.0, a, y, qm, DB[:, :3], DB[:, 3:])
            ups.append(np.abs(zn - zk).max(axis=1))
            its.append(zn)
            zk = zn
        ups, its = np.array(ups), np.array(its)
        pick = np.argmin(ups, axis=0)                 # first minimum on ties
        exp = its[pick, np.arange(len(z0))]
        z, nc = push(m)
        assert nc == len(z0)
        ok = (exp[:, 1] > 0) & (exp[:, 1] < np.pi) & (exp[:, 0] > 1.5)   # no boundary handling applied
        assert ok.mean() > 0.5 and (pick < m - 1).mean() > 0.5
        assert np.abs(z[ok] - exp[ok]).max() <= 1e-12 * (np.abs(exp[ok]).max() + 1)
    # the returned state is one of the iterates, and never one with a larger
    # update than the first: max_iter = 1 (the first iterate) bounds it
    z1, _ = push(1)
    zm, _ = push(m)
    d1 = np.abs(z1 - z0).max(axis=1)
    dm = np.abs(zm - z0).max(axis=1)
    assert np.isfinite(zm).all() and (dm <= 10 * d1 + 1e-12).mean() > 0.9


@pytest.mark.parametrize("newton", [False, True])
def test_imr_successive_update_stop_is_within_tolerance(newton):
    """The IMR iterates to round-off (Sec. 2.2.2): a solve stops when its
    last update is within tol (|z| + 1), in both forms, and the state it
    returns lies within a few tol (|z| + 1) of the solution iterated to the
    end (tol = 0: every iteration until max_iter, the smallest-update
    iterate returned); from z^n the Newton form needs under half the
    iterations of the fixed-point form (4.4 against 10)."""
    a, B0 = 0.9, 1.0
    z0, qm = _wald_plasma(500, a, seed=19)
    H0, _, D0 = O.hamiltonian(1.0, a, B0, z0, qm)

    def solve(tol, max_iter):
        p = O.push_params(a=a, dt=1e-3, scheme=O.IMR, B0pot=B0, tol=tol, max_iter=max_iter, imr_newton=newton,
                          field_kind=O.FIELD_WALD, B0field=B0)
        z = z0.copy()
        nc, sch, its = O.push(p, z, qm, H0, D0, np.zeros(len(z)), np.ones(len(z), np.uint8))
        return z, its.astype(float), nc

    z, its, nc = solve(1e-14, 50)
    zr, _, _ = solve(0.0, 60)
    assert nc == 0
    assert (np.abs(z - zr) / (np.abs(zr) + 1)).max() <= 5e-14
    # the stop is the first iterate whose update passes the test: capped one
    # iteration earlier, every solve is reported unconverged
    _, _, nc1 = solve(1e-14, int(its.min()) - 1)
    assert nc1 == len(z0)
    if newton:
        assert its.mean() < 5.0 and its.max() <= 6, (its.mean(), its.max())
    else:
        assert its.mean() > 8.0


def _axis_particles(n=600, a=0.9, seed=41):
    """Charged particles within 3e-4 rad of a pole moving towards it
    (|u_th| 0.3..3, small u_ph): steps of dt = 1e-3 under-resolve their
    turn at the axis, the IMR solve of many of them does not converge."""
    rng = np.random.default_rng(seed)
    th = np.exp(rng.uniform(np.log(1e-5), np.log(3e-4), n))
    north = rng.random(n) < 0.5
    th = np.where(north, th, np.pi - th)
    uth = rng.uniform(0.3, 3.0, n) * np.where(north, -1.0, 1.0)
    z = np.stack([rng.uniform(1.5, 5.0, n), th, rng.uniform(0, 6, n), rng.normal(size=n) * 0.5, uth,
                  rng.normal(size=n) * 2e-4], 1)
    q = np.where(np.arange(n) % 2 == 0, -100.0, 100.0)
    return np.ascontiguousarray(z), q


@pytest.mark.parametrize("newton", [False, True])
def test_unconverged_imr_step_is_redone_in_substeps(newton):
    """Reading for unconverged IMR solves near the axis: the step is redone
    as 2, 4, ..., 2^K substeps.  Pins, in the analytic Wald field (where the
    exact flow conserves H): (i) with no H condition the result is bitwise
    the composition of m plain IMR steps of dt/m (each a separate oracle
    push with max_iter 16, pole reflection included), m the first level at
    which every substep solve converges; (ii) solves that converge on their own are
    untouched; (iii) the substepped steps keep H far better than the
    smallest-update fallback; (iv) with an H condition of 1e-6 the steps
    redone are the unconverged ones and the converged ones whose end point
    misses it, each taking the first level that meets it (else the finest
    converged one), bitwise as the composition predicts."""
    a, B0, dt, K = 0.9, 1.0, 1e-3, 8
    z, q = _axis_particles(a=a)
    H0, _, D0 = O.hamiltonian(1.0, a, B0, z, q)
    kw = dict(a=a, scheme=O.IMR, B0pot=B0, field_kind=O.FIELD_WALD, B0field=B0, imr_newton=newton)

    def push(dt_, zz, max_iter=50, **extra):
        p = O.push_params(dt=dt_, max_iter=max_iter, **kw, **extra)
        zz = np.ascontiguousarray(zz.copy()); Hn = H0.copy(); al = np.ones(len(zz), np.uint8)
        nc, s, its, ncf = O.push(p, zz, q, H0, D0, Hn, al, flags=True)
        return zz, its, nc, ncf

    z_off, its_off, nc_off, fl_off = push(dt, z)
    fail = fl_off == 1
    assert 50 < fail.sum() < len(q) - 50, fail.sum()
    z_on, its_on, nc_on, _ = push(dt, z, imr_substeps=K)
    assert np.array_equal(z_on[~fail], z_off[~fail]) and np.array_equal(its_on[~fail], its_off[~fail])
    # (i) the composition of m plain pushes of dt/m, level by level
    dH = lambda zz: np.abs(O.hamiltonian(1.0, a, B0, zz, q)[0] - H0) / D0
    levels = []
    for k in range(1, K + 1):
        m = 2 ** k
        zz, ok = z.copy(), np.ones(len(q), bool)
        for _ in range(m):
            zz, it, _, f = push(dt / m, zz, max_iter=16)     # a substep's solve is capped at 16
            ok &= f == 0
        levels.append((zz, ok))

    def expected(tol):
        # the steps redone: unconverged ones, and with an H condition those
        # whose end point is off by more than it (H^n = H0 here)
        trig = fail | ((dH(z_off) > tol) if tol > 0 else False)
        out, left = z_off.copy(), trig.copy()
        finest = z_off.copy()
        for zz, ok in levels:
            finest[trig & ok] = zz[trig & ok]
            take = left & ok & ((dH(zz) <= tol) if tol > 0 else True)
            out[take] = zz[take]
            left &= ~take
        conv = trig & np.any([ok for _, ok in levels], axis=0)
        out[left & conv] = finest[left & conv]
        return out, fail & ~conv

    exp0, never = expected(0.0)
    assert np.array_equal(z_on, exp0)
    assert nc_on == never.sum() < 0.1 * fail.sum()
    # (iii) H of the rescued steps against the fallback's; the H condition
    # takes the first level that meets it, else the finest converged one
    resc = fail & ~never
    assert np.median(dH(z_on)[resc]) < 0.1 * np.median(dH(z_off)[resc])
    z_t, _, _, _ = push(dt, z, imr_substeps=K, substep_tol=1e-6)
    exp_t, _ = expected(1e-6)
    assert np.array_equal(z_t, exp_t)
    assert np.median(dH(z_t)[resc]) <= np.median(dH(z_on)[resc])
    # the H condition also redoes converged steps that miss it: the largest
    # step error over all particles falls
    assert dH(z_t).max() < dH(z_on).max()


def _meridional(a, n, seed):
    """Geodesics with u_ph = 0 (L = 0) heading for a pole: th near 0 or pi,
    u_th towards it."""
    rng = np.random.default_rng(seed)
    north = rng.random(n) < 0.5
    th = rng.uniform(0.02, 0.2, n)
    th = np.where(north, th, np.pi - th)
    uth = rng.uniform(1.0, 3.0, n) * np.where(north, -1.0, 1.0)
    z = np.stack([rng.uniform(6.0, 12.0, n), th, rng.uniform(0, 6, n), rng.normal(size=n) * 0.2, uth,
                  np.zeros(n)], 1)
    return np.ascontiguousarray(z)


def _to_half(zf):
    """A full-theta state in the half-theta coordinates: th taken modulo
    2 pi; th in (pi, 2 pi) is the half plane ph + pi at polar angle
    2 pi - th, with u_th reversed."""
    zh = zf.copy()
    zh[:, 1] = np.mod(zf[:, 1], 2 * np.pi)
    zf = zh.copy()
    low = zf[:, 1] > np.pi
    zh[low, 1] = 2 * np.pi - zf[low, 1]
    zh[low, 4] = -zf[low, 4]
    zh[low, 2] = zf[low, 2] + np.pi
    return zh


def test_full_theta_geodesics_cross_the_poles_as_the_reflection_maps_them():
    """Sec. 2.5: in the full-theta domain particles cross the poles without
    reflection (th continues past pi into the other half plane, and past 0 to
    2 pi, periodically).  Geodesics with u_ph = 0 (regular on the axis) over
    60 RK4 steps that take them over a pole equal, mapped back into the
    half-theta coordinates, the half-theta run with its reflections (1e-12:
    the reflection's ph + pi and 2 pi - th round differently)."""
    a, dt, steps = 0.9, 0.05, 60
    z0 = _meridional(a, 200, 47)
    gf = I.full_theta_grid(16, 32, 1.5, 40.0)
    pf = O.push_params(a=a, dt=dt, scheme=O.RK4, grid=gf)
    ph = O.push_params(a=a, dt=dt, scheme=O.RK4)
    zf, _, _, af = _run(pf, z0, steps)
    zh, _, _, ah = _run(ph, z0, steps)
    assert (af == 1).all() and (ah == 1).all()
    assert ((zf[:, 1] > np.pi) | (zf[:, 1] < z0[:, 1].min())).mean() > 0.3       # crossed
    assert ((zf[:, 1] >= gf.tn[0]) & (zf[:, 1] < gf.tn[0] + 2 * np.pi)).all()
    zm = _to_half(zf)
    dph = np.angle(np.exp(1j * (zm[:, 2] - zh[:, 2])))
    zm[:, 2] = zh[:, 2] + dph
    assert np.abs(zm - zh).max() / (np.abs(zh).max() + 1) < 1e-12


def test_full_theta_particle_boundary_wraps():
    """Particles stepping below tn[0] reappear at th + 2 pi, above tn[0] +
    2 pi at th - 2 pi, with u_th and ph unchanged (no reflection)."""
    a = 0.9
    gf = I.full_theta_grid(8, 16, 1.5, 40.0)
    t0 = gf.tn[0]
    z = np.ascontiguousarray(np.array([[8.0, t0 + 1e-6, 1.0, 0.0, -2.0, 0.0],
                                       [8.0, t0 + 2 * np.pi - 1e-6, 1.0, 0.0, 2.0, 0.0]]))
    pf = O.push_params(a=a, dt=0.01, scheme=O.RK4, grid=gf)
    zf, _, _, af = _run(pf, z, 1)
    assert af.all()
    assert t0 + np.pi < zf[0, 1] < t0 + 2 * np.pi and zf[0, 4] < 0 and zf[0, 2] == pytest.approx(1.0, abs=1e-3)
    assert t0 <= zf[1, 1] < t0 + np.pi and zf[1, 4] > 0 and zf[1, 2] == pytest.approx(1.0, abs=1e-3)


def test_full_theta_gather_is_periodic():
    """The gather on a full-theta grid: a component sampled from a smooth
    2 pi-periodic function (column Nth = column 0) is interpolated at th and
    at th +- 2 pi identically; in the half-node wrap cell (th below th[0])
    it is the linear interpolation between th[Nth-1] - 2 pi and th[0]."""
    gf = I.full_theta_grid(6, 12, 2.0, 20.0)
    ld = gf.ld
    F = []
    for k in range(6):
        roff = k in (0, 4, 5); toff = k in (1, 3, 5)
        X = gf.rh if roff else gf.rn
        Y = gf.th if toff else gf.tn
        f = np.zeros((gf.Nr + 1, ld))
        for i, r in enumerate(X):
            f[i, :len(Y)] = np.log(r) * (1.5 + np.cos(Y + k)) + np.sin(2 * Y)
        if toff:
            f[:, gf.Nth] = f[:, 0]
        else:
            f[:, gf.Nth] = f[:, 0]
        F.append(np.ascontiguousarray(f.ravel()))
    rng = np.random.default_rng(3)
    r = rng.uniform(3.0, 15.0, 400)
    t = rng.uniform(gf.tn[0], gf.tn[0] + 2 * np.pi, 400)
    v0 = O.gather(gf, F, r, t)
    for shift in (2 * np.pi, -2 * np.pi):
        v1 = O.gather(gf, F, r, t + shift)
        assert np.abs(v1 - v0).max() < 1e-13
    # the half-node wrap cell for B^r (k = 3, at (i, j+1/2))
    tw = gf.tn[0] + 0.3 * (gf.th[0] - gf.tn[0])
    rr = np.array([7.0])
    got = O.gather(gf, F, rr, np.array([tw]))[0, 3]
    i = np.searchsorted(gf.rn, 7.0) - 1
    wr = (7.0 - gf.rn[i]) / (gf.rn[i + 1] - gf.rn[i])
    f3 = F[3].reshape(gf.Nr + 1, ld)
    lo, hi = gf.th[-1] - 2 * np.pi, gf.th[0]
    wt = (tw - lo) / (hi - lo)
    col = lambda j: (1 - wr) * f3[i, j] + wr * f3[i + 1, j]
    assert got == pytest.approx((1 - wt) * col(gf.Nth - 1) + wt * col(0), rel=1e-13)


def test_full_theta_continued_lorentz_force_is_the_mirror_half_plane():
    """In the full-theta domain th in (pi, 2 pi) is the other half of the
    meridional plane, described by the same closed forms continued to
    sin th < 0 (a signed sqrt(gamma) in the Lorentz force, the Wald field of
    App. B continued likewise).  Charged particles (q/m = -1, +1) started
    there in the analytic Wald field move exactly as their mirrors
    (2 pi - th, ph + pi, -u_th) in the half-theta domain: 200 RK4 steps,
    1e-10 (the mirror's ph + pi and 2 pi - th round differently)."""
    a, B0, dt, steps, n = 0.9, 1.0, 0.01, 200, 100
    rng = np.random.default_rng(53)
    z = np.stack([rng.uniform(4.0, 9.0, n), rng.uniform(np.pi + 0.4, 2 * np.pi - 0.4, n), rng.uniform(0, 6, n),
                  rng.normal(size=n) * 0.3, rng.normal(size=n) * 0.5, rng.normal(size=n) * 1.5], 1)
    z = np.ascontiguousarray(z)
    q = np.where(np.arange(n) % 2 == 0, -1.0, 1.0)
    gf = I.full_theta_grid(8, 16, 1.5, 40.0)
    zmirror = _to_half(z)
    kw = dict(a=a, dt=dt, scheme=O.RK4, B0pot=B0, field_kind=O.FIELD_WALD, B0field=B0)
    pf = O.push_params(grid=gf, **kw)
    ph = O.push_params(**kw)
    qf = np.ascontiguousarray(q)
    zf = np.ascontiguousarray(z.copy())
    zh = np.ascontiguousarray(zmirror.copy())
    Hf, _, Df = O.hamiltonian(1.0, a, B0, zf, qf)
    Hh, _, Dh = O.hamiltonian(1.0, a, B0, zh, qf)
    assert np.abs(Hf - Hh).max() < 1e-12 * np.abs(Hh).max()       # H is even in the mirror
    af, ah = np.ones(n, np.uint8), np.ones(n, np.uint8)
    Hnf, Hnh = Hf.copy(), Hh.copy()
    for _ in range(steps):
        O.push(pf, zf, qf, Hf, Df, Hnf, af)
        O.push(ph, zh, qf, Hh, Dh, Hnh, ah)
    assert af.all() and ah.all()
    zm = _to_half(zf)
    zm[:, 2] = zh[:, 2] + np.angle(np.exp(1j * (zm[:, 2] - zh[:, 2])))
    assert np.abs(zm - zh).max() / (np.abs(zh).max() + 1) < 1e-10
