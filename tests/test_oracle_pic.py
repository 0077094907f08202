"""Pins of the oracle's deposition and FDTD leapfrog (no GPU)."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import pic as P
from paper_2602_07452_gb300 import inputs as I


def _particles(g, n, seed, a=0.9):
    d, q, w = I.thermal_draws(n, g, g.rn[0], g.rn[-1], 0.3, seed=seed)
    z = O.seed_fido(1.0, a, d)
    w = np.random.default_rng(seed).uniform(0.5, 2.0, n)
    return z, q, w


def test_deposit_weights_partition_unity():
    """Sec. 2.3: the four node shares of a particle are the four subvolumes
    over their sum, so each sub-grid receives exactly the particle's charge
    Q = w q/m (and Q v^i for the currents)."""
    a = 0.9
    g = I.log_grid(12, 10, 1.5, 20.0)
    z, q, w = _particles(g, 300, 1, a)
    rho, jr, jt, jp = P.deposit(1.0, a, g, z, q, w, normalise=False)
    Q = (q * w).sum()
    assert abs(rho.sum() - Q) < 1e-11 * np.abs(q * w).sum()
    m = O.metric(1.0, a, z[:, 0], z[:, 1])
    Ur = m[:, 8] * z[:, 3] + m[:, 9] * z[:, 5]
    Ut = m[:, 10] * z[:, 4]
    Up = m[:, 9] * z[:, 3] + m[:, 11] * z[:, 5]
    G = np.sqrt(1 + z[:, 3] * Ur + z[:, 4] * Ut + z[:, 5] * Up)
    for arr, v in ((jr, Ur / G), (jt, Ut / G), (jp, Up / G)):
        tot = (q * w * v).sum()
        assert abs(arr.sum() - tot) < 1e-11 * np.abs(q * w * v).sum()


def test_deposit_unit_density_is_bilinear():
    """With sqrt(gamma) replaced by 1 the subvolumes are areas and the
    opposite-volume weights reduce to bilinear cloud-in-cell weights."""
    a = 0.9
    g = I.log_grid(6, 5, 2.0, 9.0)
    rng = np.random.default_rng(2)
    for _ in range(20):
        r = rng.uniform(g.rn[0], g.rn[-1]); t = rng.uniform(g.tn[0], g.tn[-1])
        z = np.array([[r, t, 0, 0, 0, 0]])
        rho, _, _, _ = P.deposit(1.0, a, g, z, [1.0], [1.0], unit=True, normalise=False)
        i = np.searchsorted(g.rn, r, side="right") - 1
        j = np.searchsorted(g.tn, t, side="right") - 1
        wr = (r - g.rn[i]) / (g.rn[i + 1] - g.rn[i]); wt = (t - g.tn[j]) / (g.tn[j + 1] - g.tn[j])
        exp = np.zeros(g.size)
        exp[i * g.ld + j] = (1 - wr) * (1 - wt); exp[(i + 1) * g.ld + j] = wr * (1 - wt)
        exp[i * g.ld + j + 1] = (1 - wr) * wt; exp[(i + 1) * g.ld + j + 1] = wr * wt
        assert np.abs(rho - exp).max() < 1e-14


def test_deposit_particle_on_node():
    """A particle on a node puts its whole charge on that node."""
    a = 0.5
    g = I.log_grid(6, 5, 2.0, 9.0)
    z = np.array([[g.rn[3], g.tn[2], 0, 0.1, 0.2, 0.3]])
    rho, _, _, _ = P.deposit(1.0, a, g, z, [2.0], [1.5], normalise=False)
    assert abs(rho[3 * g.ld + 2] - 3.0) < 1e-15 and abs(rho.sum() - 3.0) < 1e-15


def test_deposit_normalisation_conserves_charge():
    """Normalised densities times the 2 pi dual volumes give back the charge,
    and the dual cells tile the domain (their volumes sum to the domain's)."""
    a = 0.9
    g = I.log_grid(16, 12, 1.6, 25.0)
    z, q, w = _particles(g, 500, 3, a)
    rho, jr, jt, jp = P.deposit(1.0, a, g, z, q, w)
    v00, v10, v01 = P.dual_volumes(1.0, a, g)
    assert abs((rho * v00).sum() - (q * w).sum()) < 1e-11 * np.abs(q * w).sum()
    tot = [v00[:].reshape(g.Nr + 1, g.ld)[:, :g.Nth + 1].sum(),
           v10.reshape(g.Nr + 1, g.ld)[:g.Nr, :g.Nth + 1].sum(),
           v01.reshape(g.Nr + 1, g.ld)[:, :g.Nth].sum()]
    assert max(tot) - min(tot) < 1e-3 * max(tot)


def _rand_fields(g, seed):
    rng = np.random.default_rng(seed)
    s = P.FdtdState(g)
    for arrs in (s.B0, s.B1, s.D0, s.D1):
        for x in arrs:
            x[:] = rng.normal(size=g.size)
    s.B0 = [x.copy() for x in s.B1]
    return s


@pytest.mark.parametrize("a", [0.0, 0.9])
def test_fdtd_vacuum_preserves_divergences(a):
    """Sec. 2.1: on the Yee grid the curl updates leave div B unchanged to
    round-off (and div D in vacuum), for arbitrary fields, away from the
    absorbing layer."""
    g = I.log_grid(24, 20, 1.9, 30.0)
    s = _rand_fields(g, 5)
    p = P.FdtdParams(1.0, a, 0.002, 1e4, 5.0, 0.9 * g.rn[-1], g.rn[-1])
    dB0, dD0 = P.div(1.0, a, g, s.B1, s.D1)
    for _ in range(3):
        P.fdtd(p, s, 1)
        P.fdtd(p, s, 2)
        s.swap()
    dB1, dD1 = P.div(1.0, a, g, s.B1, s.D1)
    rm = g.rh < 0.9 * g.rn[-1] * 0.999
    ii = np.arange(g.Nr)[rm[:g.Nr]]
    ii = ii[ii < g.Nr - 2]
    sel = np.zeros((g.Nr + 1, g.ld), bool)
    sel[ii, :g.Nth] = True
    scale = np.abs(dB0).max()
    assert np.abs((dB1 - dB0).reshape(g.Nr + 1, g.ld)[sel]).max() < 1e-12 * scale
    seld = np.zeros((g.Nr + 1, g.ld), bool)
    seld[2:ii.max(), 2:g.Nth - 1] = True
    scale = np.abs(dD0).max()
    assert np.abs((dD1 - dD0).reshape(g.Nr + 1, g.ld)[seld]).max() < 1e-12 * scale


def test_fdtd_gauss_law_with_sources():
    """Ampere's law with sources (sub-step 10): the node divergence of D
    changes by exactly -4 pi dt times the Yee divergence of sqrt(gamma) J."""
    a = 0.9
    g = I.log_grid(20, 16, 1.9, 30.0)
    s = _rand_fields(g, 6)
    rng = np.random.default_rng(7)
    for x in s.j1 + [s.rho1]:
        x[:] = rng.normal(size=g.size)
    for x in s.j0 + [s.rho0]:
        x[:] = 0.0
    p = P.FdtdParams(1.0, a, 0.003, 0.0, 5.0, g.rn[-1], g.rn[-1])
    P.fdtd(p, s, 1)
    D15 = [x.copy() for x in s.D1]
    P.fdtd(p, s, 2)      # D0 <- D^{n+5/2} = D1 + dt (curl H - 4 pi J1)
    _, dA = P.div(1.0, a, g, s.B0, D15)
    _, dB = P.div(1.0, a, g, s.B0, s.D0)
    # J from the same definition as the oracle (alpha j - rho beta) at the Yee points
    m_r = O.metric(1.0, a, np.repeat(g.rh, g.Nth + 1), np.tile(g.tn, g.Nr))
    Jr = np.zeros(g.size); Jt = np.zeros(g.size)
    R = s.rho1.reshape(g.Nr + 1, g.ld)
    for i in range(g.Nr):
        for j in range(g.Nth + 1):
            mm = m_r[i * (g.Nth + 1) + j]
            sa = O.metric(1.0, a, [g.rn[i]], [g.tn[j]])[0, 12]
            sb = O.metric(1.0, a, [g.rn[i + 1]], [g.tn[j]])[0, 12]
            rb = (sa * R[i, j] + sb * R[i + 1, j]) / (2 * mm[12])
            Jr[i * g.ld + j] = mm[2] * s.j1[0][i * g.ld + j] - rb * mm[3]
    mt = O.metric(1.0, a, np.repeat(g.rn, g.Nth), np.tile(g.th, g.Nr + 1))
    for i in range(g.Nr + 1):
        for j in range(g.Nth):
            Jt[i * g.ld + j] = mt[i * g.Nth + j, 2] * s.j1[1][i * g.ld + j]
    _, dJ = P.div(1.0, a, g, s.B0, [Jr, Jt, np.zeros(g.size)])
    sel = np.zeros((g.Nr + 1, g.ld), bool)
    sel[2:g.Nr - 1, 2:g.Nth - 1] = True
    lhs = (dB - dA).reshape(g.Nr + 1, g.ld)[sel]
    rhs = (-4 * math.pi * p.dt * dJ).reshape(g.Nr + 1, g.ld)[sel]
    assert np.abs(lhs - rhs).max() < 1e-10 * np.abs(rhs).max()


def test_fdtd_static_wald_schwarzschild_stays_static():
    """Sec. 3.2 / App. B.1: the a = 0 Wald field (E_i = 0, D = -beta x B /
    alpha) is a static vacuum solution; the leapfrog keeps it static up to
    the truncation error of the grid, which falls with resolution."""
    a = 0.0
    errs = []
    for N in (32, 64):
        g = I.log_grid(N, N, 2.2, 12.0)
        F = O.wald_on_grid(a, 1.0, g)
        s = P.FdtdState(g)
        for k in range(3):
            s.D0[k][:] = F[k]; s.D1[k][:] = F[k]
            s.B0[k][:] = F[3 + k]; s.B1[k][:] = F[3 + k]
        p = P.FdtdParams(1.0, a, 0.2 * (g.rn[1] - g.rn[0]), 0.0, 5.0, 1e9, 2e9)
        nst = int(round(0.5 / p.dt))
        for _ in range(nst):
            P.fdtd(p, s, 1); P.fdtd(p, s, 2); s.swap()
        # a region the boundary perturbations cannot reach in t = 0.5
        ri = (g.rn >= 4.0) & (g.rn <= 8.0)
        tj = (g.th >= 0.5) & (g.th <= math.pi - 0.5)
        Br = s.B1[0].reshape(g.Nr + 1, g.ld)[ri][:, :g.Nth][:, tj]
        Br0 = F[3].reshape(g.Nr + 1, g.ld)[ri][:, :g.Nth][:, tj]
        errs.append(np.abs(Br - Br0).max() / np.abs(Br0).max())
    assert errs[0] < 2e-2 and errs[1] < 0.6 * errs[0], errs


# ---------------------------------------------------------------------------
# Split monopole (Sec. 3.4, App. B.2) and the BZ power diagnostic (Eq. Pbz)
# ---------------------------------------------------------------------------
def _psi(M, B0, zeta0, th):
    return 4.0 * M * M * B0 * (2.0 / np.pi) * np.arctan(zeta0 * (th - np.pi / 2)) * (1.0 - np.cos(th))


def test_split_monopole_flux_function_identity():
    """sqrt(gamma) B^r integrated over th from the pole gives back Psi(th)
    (Schwarzschild sqrt(gamma) = r^2 sin th sqrt(1 + 2M/r), written out here):
    pins the derivative of the flux function, both terms and the sign."""
    M, B0, z0 = 1.0, 1.7, 40.0
    g = I.log_grid(8, 4000, 2.0, 20.0)
    F = P.split_monopole_on_grid(M, 0.0, B0, z0, g)
    Br = F[3].reshape(g.Nr + 1, g.ld)
    for i in (0, 3, 8):
        r = g.rn[i]
        sg = r * r * np.sin(g.th) * np.sqrt(1.0 + 2.0 * M / r)
        f = Br[i, : g.Nth] * sg                       # d_th Psi at the cell centres th_{j+1/2}
        cum = np.concatenate([[0.0], np.cumsum(f * np.diff(g.tn))])   # int from tn[0]
        expect = _psi(M, B0, z0, g.tn) - _psi(M, B0, z0, g.tn[0])
        assert np.abs(cum - expect).max() <= 1e-5 * np.abs(expect).max()
    for k in (0, 1, 2, 4, 5):
        assert not F[k].any()


def test_split_monopole_is_divergence_free():
    """sqrt(gamma) B^r = d_th Psi does not depend on r, so the Yee divergence
    of the field vanishes to rounding (a = 0.9)."""
    a = 0.9
    g = I.log_grid(40, 64, 1.5, 30.0)
    F = P.split_monopole_on_grid(1.0, a, 1.0, 1e3, g)
    dB, _ = P.div(1.0, a, g, F[3:], F[:3])
    scale = (np.abs(F[3]).max() * 30.0 ** 2) / np.diff(g.rn).min()
    assert np.abs(dB).max() <= 1e-12 * scale


@pytest.mark.parametrize("N", [64, 128, 256])
def test_bz_power_quadrature(N):
    """Eq. (Pbz) for E_th = r sin th, H_ph = sin th, E_ph = sin th cos th,
    H_th = cos th on their Yee points: P = (1/2)[r pi/2 - 2/3] on the sphere,
    to the second order of the staggered averages and the midpoint rule."""
    g = I.log_grid(16, N, 2.0, 20.0)
    R = lambda ro: (g.rh if ro else g.rn)
    T = lambda to: (g.th if to else g.tn)
    def field(ro, to, f):
        x = np.zeros((g.Nr + 1, g.ld))
        rr, tt = R(ro), T(to)
        x[: len(rr), : len(tt)] = f(rr[:, None], tt[None, :])
        return x.ravel()
    z = np.zeros(g.size)
    E = [z, field(0, 1, lambda r, t: r * np.sin(t)), field(0, 0, lambda r, t: np.sin(t) * np.cos(t))]
    H = [z, field(1, 0, lambda r, t: np.cos(t) + 0 * r), field(1, 1, lambda r, t: np.sin(t) + 0 * r)]
    i = 7
    got = P.bz_power(g, E, H, i)
    exact = 0.5 * (g.rh[i] * np.pi / 2 - 2.0 / 3.0)
    err = abs(got - exact)
    # staggering in r: E_th is averaged between rn[i] and rn[i+1] (mean
    # cosh(d/2) rh[i] on the log grid, d = ln(rn[i+1] / rn[i])); in th the
    # averages and the midpoint rule are second order
    d = np.log(g.rn[i + 1] / g.rn[i])
    tol_r = 1.5 * g.rh[i] * (np.cosh(d / 2) - 1.0) * np.pi / 4
    assert err < 8.0 / N ** 2 + tol_r, (N, err, tol_r)


def _gauss_residual(a, g, D, rho):
    """Discrete Gauss law at every integer node i = 1 .. Nr-1, j = 0 .. Nth:
    sqrtg-weighted Yee divergence of D (no flux through the poles, dual
    widths reaching the pole) minus 4 pi sqrtg rho, with sqrt(gamma) taken
    from the Appendix A metric."""
    L = g.ld
    sg = lambda r, t: O.metric(1.0, a, [r], [t])[0, 12]
    res = np.zeros((g.Nr + 1, L))
    for i in range(1, g.Nr):
        for j in range(g.Nth + 1):
            o = i * L + j
            wr = g.rh[i] - g.rh[i - 1]
            wt = (g.th[j] if j < g.Nth else math.pi) - (g.th[j - 1] if j > 0 else 0.0)
            flux_r = sg(g.rh[i], g.tn[j]) * D[0][o] - sg(g.rh[i - 1], g.tn[j]) * D[0][o - L]
            flux_t = (sg(g.rn[i], g.th[j]) * D[1][o] if j < g.Nth else 0.0) - \
                     (sg(g.rn[i], g.th[j - 1]) * D[1][o - 1] if j > 0 else 0.0)
            res[i, j] = flux_r / wr + flux_t / wt - 4 * math.pi * sg(g.rn[i], g.tn[j]) * rho[o]
    return res


@pytest.mark.parametrize("a", [0.0, 0.9])
def test_div_clean_restores_gauss_law(a):
    """Sec. 2.4 (Eq. phi): once the Jacobi solve has converged, the corrected
    D satisfies the discrete Gauss law to rounding at every node, the poles
    included, although it violated it at O(1) before."""
    g = I.log_grid(20, 16, 1.9, 30.0)
    rng = np.random.default_rng(11)
    D = [rng.normal(size=g.size) for _ in range(3)]
    rho = rng.normal(size=g.size) * 0.1
    r0 = np.abs(_gauss_residual(a, g, D, rho)).max()
    Dc, phi = P.div_clean(1.0, a, g, D, rho, 20000)
    r1 = np.abs(_gauss_residual(a, g, Dc, rho)).max()
    assert r0 > 1.0
    assert r1 < 1e-12 * r0
    P2 = phi.reshape(g.Nr + 1, g.ld)
    assert np.all(P2[0] == 0.0) and np.all(P2[g.Nr] == 0.0)


def test_div_clean_keeps_covariant_phi_component():
    """The correction is a gradient of an axisymmetric phi: its covariant
    phi component, gamma_rph dD^r + gamma_phph dD^ph at a node (with dD^r
    there the gamma^rr-weighted mean radial slope), vanishes identically."""
    a = 0.9
    g = I.log_grid(16, 12, 1.9, 20.0)
    rng = np.random.default_rng(12)
    D = [rng.normal(size=g.size) for _ in range(3)]
    rho = rng.normal(size=g.size)
    Dc, phi = P.div_clean(1.0, a, g, D, rho, 300)
    P2 = phi.reshape(g.Nr + 1, g.ld)
    dDp = (Dc[2] - D[2]).reshape(g.Nr + 1, g.ld)
    worst, scale = 0.0, 0.0
    for i in range(g.Nr + 1):
        for j in range(g.Nth + 1):
            sl = []
            if i < g.Nr:
                sl.append((P2[i + 1, j] - P2[i, j]) / (g.rn[i + 1] - g.rn[i]))
            if i > 0:
                sl.append((P2[i, j] - P2[i - 1, j]) / (g.rn[i] - g.rn[i - 1]))
            m = O.metric(1.0, a, [g.rn[i]], [g.tn[j]])[0]
            if abs(math.sin(g.tn[j])) < 1e-12:
                continue
            dDr = -m[8] * np.mean(sl)
            worst = max(worst, abs(m[5] * dDr + m[7] * dDp[i, j]))
            scale = max(scale, abs(m[7] * dDp[i, j]))
    assert scale > 1e-3
    assert worst < 1e-12 * scale


def test_div_clean_leaves_solenoidal_field_alone():
    """A D built as the discrete curl of a flux function (zero at both poles)
    has zero Yee divergence, so with rho = 0 the right side vanishes, phi
    stays zero to rounding and D is returned unchanged."""
    a = 0.9
    g = I.log_grid(18, 14, 1.9, 25.0)
    L = g.ld
    # Psi at the (r_{i+1/2}, th_{j+1/2}) corners, zero on the poles
    psi = lambda r, t: math.sin(t) ** 2 * (1.0 + 0.3 * math.cos(t)) * math.log(r)
    sg = lambda r, t: O.metric(1.0, a, [r], [t])[0, 12]
    D = [np.zeros(g.size) for _ in range(3)]
    th_ext = lambda j: 0.0 if j < 0 else (math.pi if j >= g.Nth else g.th[j])
    for i in range(g.Nr):
        for j in range(g.Nth + 1):
            wt = th_ext(j) - th_ext(j - 1)
            D[0][i * L + j] = (psi(g.rh[i], th_ext(j)) - psi(g.rh[i], th_ext(j - 1))) / wt / sg(g.rh[i], g.tn[j])
    for i in range(1, g.Nr):
        for j in range(g.Nth):
            wr = g.rh[i] - g.rh[i - 1]
            D[1][i * L + j] = -(psi(g.rh[i], g.th[j]) - psi(g.rh[i - 1], g.th[j])) / wr / sg(g.rn[i], g.th[j])
    rho = np.zeros(g.size)
    res = _gauss_residual(a, g, D, rho)
    scale = max(np.abs(D[0]).max(), np.abs(D[1]).max())
    assert np.abs(res).max() < 1e-12 * scale * 100
    Dc, phi = P.div_clean(1.0, a, g, D, rho, 500)
    assert np.abs(phi).max() < 1e-12 * scale
    for k in range(3):
        assert np.abs(Dc[k] - D[k]).max() < 1e-12 * scale


# ---- pair injection (Sec. 3.3, 3.4) -------------------------------------------

def _radial_field(g, B0=1.0):
    """B^r = B0 on every B^r point, B^th = 0: at a cell centre the spin-axis
    component is exactly B0 cos th (no averaging error)."""
    return np.full(g.size, B0), np.zeros(g.size)


def _empty_store(cap):
    return np.zeros((cap, 6)), np.zeros(cap), np.zeros(cap), np.zeros(cap, np.uint8)


def _omega_h(a, M=1.0):
    """Horizon angular velocity a / (r_h^2 + a^2)."""
    rh = M + math.sqrt(M * M - a * a)
    return a / (rh * rh + a * a)


def test_inject_weights_follow_the_gj_density():
    """Into an empty region every cell with centre radius in [r_lo, r_hi] gets
    one pair whose two weights give n = n0 n_GJ with n_GJ = |Omega_h B0
    cos th - r B1 sin th| / (4 pi e) for the uniform coordinate components
    B^r = B0, B^th = B1 (exact at the cell centre): w |q/m| x 2 / (n0 e n_GJ)
    equals the proper cell volume, checked against an independent adaptive
    quadrature of sqrt(gamma) (within the 4 x 4 trapezoid's error)."""
    from scipy import integrate
    a = 0.9
    g = I.log_grid(10, 8, 1.5, 12.0)
    Br, Bt = np.full(g.size, 2.0), np.full(g.size, 0.3)
    d = I.injection_draws(g, 0.5, seed=1)
    z, qm, w, al = _empty_store(4 * g.Nr * g.Nth)
    r_lo, r_hi = 2.0, 6.0
    z, qm, w, al, n1, K, fl = P.inject_pairs(1.0, a, g, z, qm, w, al, 0, z.shape[0], Br, Bt, r_lo, r_hi,
                                             3.0, 5.0, 100.0, d)
    F = fl.reshape(g.Nr, g.Nth)
    rows = (g.rh >= r_lo) & (g.rh <= r_hi)
    assert np.array_equal(F.any(axis=1), rows) and np.all(F[rows])
    assert K == F.sum() and n1 == 2 * K
    Om = _omega_h(a)
    sg = lambda t, r: O.metric(1.0, a, [r], [t])[0, 12]
    k = 0
    for i in range(g.Nr):
        for j in range(g.Nth):
            if not F[i, j]:
                continue
            egj = abs(Om * (2.0 * math.cos(g.th[j]) - g.rh[i] * 0.3 * math.sin(g.th[j]))) / (4 * math.pi)
            V = 2 * math.pi * integrate.dblquad(sg, g.rn[i], g.rn[i + 1], g.tn[j], g.tn[j + 1],
                                                epsabs=0, epsrel=1e-11)[0]
            for s in (0, 1):
                Vw = w[k + s] * 100.0 * 2 / (5.0 * egj)
                assert abs(Vw / V - 1) < 2e-3, (i, j, Vw / V)
            assert qm[k] == -100.0 and qm[k + 1] == 100.0 and w[k] == w[k + 1]
            k += 2


def test_inject_stops_at_the_multiplicity():
    """Re-injecting with no particle loss: with n0 = 1.25 and multiplicity 3
    the density climbs 1.25, 2.5, 3.75 n_GJ, so exactly three calls inject
    into each eligible cell and the fourth none; without spin (Omega_h = 0,
    n_GJ = 0) nothing is injected."""
    g = I.log_grid(8, 6, 1.5, 10.0)
    Br, Bt = _radial_field(g)
    d = I.injection_draws(g, 0.5, seed=2)
    cap = 10 * g.Nr * g.Nth
    z, qm, w, al = _empty_store(cap)
    n = 0
    counts = []
    for call in range(4):
        z, qm, w, al, n, K, fl = P.inject_pairs(1.0, 0.7, g, z, qm, w, al, n, cap, Br, Bt, 1.0, 20.0, 3.0, 1.25,
                                                50.0, d)
        counts.append(K)
    C = g.Nr * g.Nth
    assert counts == [C, C, C, 0]
    z0, qm0, w0, al0 = _empty_store(cap)
    _, _, _, _, n0_, K0, _ = P.inject_pairs(1.0, 0.0, g, z0, qm0, w0, al0, 0, cap, Br, Bt, 1.0, 20.0, 3.0, 1.25,
                                            50.0, d)
    assert K0 == 0 and n0_ == 0


def test_inject_pair_kinematics():
    """The two particles of a pair sit at one point inside their cell, carry
    opposite q/m and equal weights, and their covariant momenta have the
    drawn FIDO-frame magnitudes: gamma^ij u_i u_j = |uhat|^2 (Appendix A
    inverse metric)."""
    a = 0.99
    g = I.log_grid(9, 7, 1.3, 8.0)
    Br, Bt = _radial_field(g)
    d = I.injection_draws(g, 0.5, seed=3)
    cap = 2 * g.Nr * g.Nth
    z, qm, w, al, n, K, fl = P.inject_pairs(1.0, a, g, *_empty_store(cap), 0, cap, Br, Bt, 0.0, 1e9, 3.0, 5.0,
                                            100.0, d)
    cells = np.flatnonzero(fl)
    assert n == 2 * cells.size > 0
    for k, c in enumerate(cells):
        i, j = divmod(int(c), g.Nth)
        e, p = z[2 * k], z[2 * k + 1]
        assert np.array_equal(e[:3], p[:3])
        assert g.rn[i] <= e[0] <= g.rn[i + 1] and g.tn[j] <= e[1] <= g.tn[j + 1] and 0 <= e[2] < 2 * math.pi
        m = O.metric(1.0, a, [e[0]], [e[1]])[0]
        for s, zz in ((0, e), (1, p)):
            u = zz[3:]
            norm = m[8] * u[0] ** 2 + 2 * m[9] * u[0] * u[2] + m[10] * u[1] ** 2 + m[11] * u[2] ** 2
            uh = d[c, 3 + 3 * s: 6 + 3 * s]
            assert abs(norm - uh @ uh) < 1e-12 * (1 + uh @ uh)
        assert qm[2 * k] == -qm[2 * k + 1] and w[2 * k] == w[2 * k + 1] and al[2 * k] == al[2 * k + 1] == 1


def test_inject_counts_alive_particles_of_the_cell_only():
    """Existing alive particles fill (saturate) their cell; removed particles
    count for nothing; cells outside [r_lo, r_hi] are never flagged."""
    a = 0.9
    g = I.log_grid(8, 6, 1.5, 10.0)
    Br, Bt = _radial_field(g)
    d = I.injection_draws(g, 0.5, seed=5)
    cap = 4 * g.Nr * g.Nth + 10
    z, qm, w, al = _empty_store(cap)
    # particle 0 alive, huge weight, in cell (3, 2); particle 1 removed, huge weight, in cell (4, 1)
    for p, (i, j), alive in ((0, (3, 2), 1), (1, (4, 1), 0)):
        z[p, 0] = 0.5 * (g.rn[i] + g.rn[i + 1])
        z[p, 1] = 0.5 * (g.tn[j] + g.tn[j + 1])
        qm[p], w[p], al[p] = -10.0, 1e9, alive
    r_lo, r_hi = g.rh[2], g.rh[5]
    _, _, _, _, n, K, fl = P.inject_pairs(1.0, a, g, z, qm, w, al, 2, cap, Br, Bt, r_lo, r_hi, 3.0, 5.0, 100.0, d)
    F = fl.reshape(g.Nr, g.Nth)
    assert not F[3, 2] and F[4, 1]
    assert not F[:2].any() and not F[6:].any()
    assert F[2:6].sum() == 4 * g.Nth - 1 and K == F.sum() and n == 2 + 2 * K


def test_inject_capacity_keeps_cell_order():
    """With room for three pairs only, the pairs of the first three flagged
    cells (cell order) are written, identical to the first three of an
    unlimited call; the return value still counts every wanted pair."""
    a = 0.9
    g = I.log_grid(8, 6, 1.5, 10.0)
    Br, Bt = _radial_field(g)
    d = I.injection_draws(g, 0.5, seed=6)
    big = P.inject_pairs(1.0, a, g, *_empty_store(200), 0, 200, Br, Bt, 0.0, 1e9, 3.0, 5.0, 100.0, d)
    small = P.inject_pairs(1.0, a, g, *_empty_store(200), 0, 7, Br, Bt, 0.0, 1e9, 3.0, 5.0, 100.0, d)
    assert small[4] == 6 and small[5] == big[5] > 3
    assert np.array_equal(small[0][:6], big[0][:6]) and np.array_equal(small[2][:6], big[2][:6])
    assert not small[0][6:].any()


# ---- charge-conserving deposit (extension) -----------------------------------

def _yee_dual(g):
    dr = np.array([(g.rh[i] if i < g.Nr else g.rn[-1]) - (g.rh[i - 1] if i > 0 else g.rn[0])
                   for i in range(g.Nr + 1)])
    dt_ = np.array([(g.th[j] if j < g.Nth else math.pi) - (g.th[j - 1] if j > 0 else 0.0)
                    for j in range(g.Nth + 1)])
    return dr, dt_


def _moves(g, a, n, seed, frac=0.4):
    """States inside the grid and moves of up to frac of a cell (some cross a node)."""
    rng = np.random.default_rng(seed)
    i = rng.integers(1, g.Nr - 1, n); j = rng.integers(1, g.Nth - 1, n)
    r = g.rn[i] + rng.random(n) * (g.rn[i + 1] - g.rn[i])
    t = g.tn[j] + rng.random(n) * (g.tn[j + 1] - g.tn[j])
    z0 = np.stack([r, t, rng.uniform(0, 6, n), rng.normal(size=n), rng.normal(size=n), rng.normal(size=n)], 1)
    z1 = z0.copy()
    z1[:, 0] += frac * rng.uniform(-1, 1, n) * (g.rn[i + 1] - g.rn[i])
    z1[:, 1] += frac * rng.uniform(-1, 1, n) * (g.tn[j + 1] - g.tn[j])
    z1[:, 3:] += 0.1 * rng.normal(size=(n, 3))
    q = np.where(rng.random(n) < 0.5, -1.0, 1.0) * rng.uniform(0.5, 2, n)
    return z0, z1, q, rng.uniform(0.5, 2, n)


@pytest.mark.parametrize("a", [0.0, 0.9])
def test_conserving_deposit_continuity_at_every_node(a):
    """The deposit of a move satisfies the discrete continuity equation
    sqrtg (rho^{n+1} - rho^n) + dt Yee-div(sqrtg J) = 0 at every node (the
    Yee divergence with the Appendix A sqrt(gamma), written here
    independently), and conserves the total charge."""
    g = I.log_grid(12, 10, 1.5, 20.0)
    z0, z1, q, w = _moves(g, a, 400, 3)
    al = np.ones(len(q), np.uint8)
    dt = 0.05
    rho0 = P.deposit_conserving(1.0, a, g, z0, z0, q, w, al, dt)[0]
    rho1, Jr, Jt, Jp, sk = P.deposit_conserving(1.0, a, g, z0, z1, q, w, al, dt)
    assert sk == 0
    L = g.ld
    sg = lambda r, t: O.metric(1.0, a, [r], [t])[0, 12]
    dr, dth = _yee_dual(g)
    worst, scale = 0.0, 0.0
    Qtot = 0.0
    for i in range(g.Nr + 1):
        for j in range(g.Nth + 1):
            o = i * L + j
            fr1 = sg(g.rh[i], g.tn[j]) * Jr[o] if i < g.Nr else 0.0
            fr0 = sg(g.rh[i - 1], g.tn[j]) * Jr[o - L] if i > 0 else 0.0
            ft1 = sg(g.rn[i], g.th[j]) * Jt[o] if j < g.Nth else 0.0
            ft0 = sg(g.rn[i], g.th[j - 1]) * Jt[o - 1] if j > 0 else 0.0
            div = (fr1 - fr0) / dr[i] + (ft1 - ft0) / dth[j]
            lhs = sg(g.rn[i], g.tn[j]) * (rho1[o] - rho0[o])
            worst = max(worst, abs(lhs + dt * div))
            scale = max(scale, abs(lhs))
            Qtot += 2 * math.pi * sg(g.rn[i], g.tn[j]) * dr[i] * dth[j] * rho1[o]
    assert scale > 0 and worst <= 1e-13 * scale
    assert abs(Qtot - (q * w).sum()) <= 1e-12 * np.abs(q * w).sum()


def test_conserving_deposit_particle_on_a_node_and_at_rest():
    """A particle resting on a node puts all its charge there and no
    current; a pure r move makes no th current (and vice versa)."""
    a = 0.9
    g = I.log_grid(8, 8, 1.5, 10.0)
    z = np.array([[g.rn[3], g.tn[4], 0.0, 0.0, 0.0, 0.0]])
    rho, Jr, Jt, Jp, _ = P.deposit_conserving(1.0, a, g, z, z, [2.0], [1.5], [1], 0.1)
    dr, dth = _yee_dual(g)
    o = 3 * g.ld + 4
    V = 2 * math.pi * O.metric(1.0, a, [g.rn[3]], [g.tn[4]])[0, 12] * dr[3] * dth[4]
    assert np.count_nonzero(rho) == 1 and abs(rho[o] * V - 3.0) < 1e-13
    assert not Jr.any() and not Jt.any() and not Jp.any()
    z1 = z.copy(); z1[0, 0] += 0.3 * (g.rn[4] - g.rn[3])
    _, Jr, Jt, _, _ = P.deposit_conserving(1.0, a, g, z, z1, [2.0], [1.5], [1], 0.1)
    assert Jr.any() and not Jt.any()
    z1 = z.copy(); z1[0, 1] -= 0.3 * (g.tn[4] - g.tn[3])
    _, Jr, Jt, _, _ = P.deposit_conserving(1.0, a, g, z, z1, [2.0], [1.5], [1], 0.1)
    assert Jt.any() and not Jr.any()


def test_conserving_pic_loop_keeps_gauss_residual():
    """Sec. 2.1's step with the conserving deposit and the FDTD in its
    conserving mode (no absorbing layer): Yee-div(sqrtg D^{n+1/2}) -
    4 pi sqrtg rho^n stays what it was at the start, at the interior nodes,
    to rounding over 6 steps of a charged plasma (the paper's deposit
    changes it at O(1))."""
    a = 0.9
    g = I.log_grid(24, 20, 1.5, 20.0)
    n = 3000
    rng = np.random.default_rng(4)
    d, q, w = I.thermal_draws(n, g, 3.0, 12.0, 0.3, seed=5, qm=50.0)
    d[:, 1] = rng.uniform(0.5, math.pi - 0.5, n)
    z = O.seed_fido(1.0, a, d)
    Fw = O.wald_on_grid(a, 1.0, g)
    st = P.FdtdState(g)
    for k in range(3):
        st.D0[k][:] = Fw[k]; st.D1[k][:] = Fw[k]; st.B0[k][:] = Fw[3 + k]; st.B1[k][:] = Fw[3 + k]
    dt = 2e-3
    po = P.FdtdParams(1.0, a, dt, 0.0, 5.0, g.rn[-1], g.rn[-1], 1)
    w = np.full(n, 1e-3)
    al = np.ones(n, np.uint8)
    rho, _, _, _, _ = P.deposit_conserving(1.0, a, g, z, z, q, w, al, dt)
    st.rho1 = rho.copy()
    sel = np.zeros((g.Nr + 1, g.ld), bool)
    sel[2:g.Nr - 1, 2:g.Nth - 1] = True
    sg = O.metric(1.0, a, np.repeat(g.rn, g.ld), np.tile(g.tn, g.Nr + 1))[:, 12]

    def resid(D, rho_):
        _, dD = P.div(1.0, a, g, st.B1, D)
        return (dD - 4 * math.pi * sg * rho_).reshape(g.Nr + 1, g.ld)[sel]

    R0 = resid(st.D1, st.rho1)
    H0, _, D0 = O.hamiltonian(1.0, a, 0.0, z, q)
    pp = O.push_params(a=a, dt=dt, scheme=O.RK4, field_kind=O.FIELD_GRID, r_max=g.rn[-1])
    drift = 0.0
    for step in range(6):
        P.fdtd(po, st, 1)
        zold = z.copy()
        O.push(pp, z, q, H0, D0, H0.copy(), al, g, [st.D1[0], st.D1[1], st.D1[2], st.Bh[0], st.Bh[1], st.Bh[2]])
        assert al.all()
        rho, Jr, Jt, Jp, sk = P.deposit_conserving(1.0, a, g, zold, z, q, w, np.ones(n, np.uint8), dt)
        assert sk == 0
        st.j1 = [Jr, Jt, Jp]; st.rho1 = rho
        P.fdtd(po, st, 2)
        st.swap()
        R = resid(st.D1, st.rho0)          # D^{n+5/2} with rho^{n+2} (swapped into slot 0)
        drift = max(drift, np.abs(R - R0).max())
    scale = np.abs(4 * math.pi * sg.reshape(g.Nr + 1, g.ld)[sel] * st.rho0.reshape(g.Nr + 1, g.ld)[sel]).max()
    assert scale > 0 and drift <= 1e-11 * scale, (drift, scale)


# ---------------------------------------------------------------------------
# Full-theta domain (Sec. 2.5: periodic in th), FDTD
# ---------------------------------------------------------------------------
def _images(g, arrs):
    for x in arrs:
        X = x.reshape(g.Nr + 1, g.ld)
        X[:, g.Nth] = X[:, 0]


def _rand_fields_full(g, seed):
    s = _rand_fields(g, seed)
    for arrs in (s.B0, s.B1, s.D0, s.D1):
        _images(g, arrs)
    return s


def _uneven_full_theta_grid(Nr, Nth, r_min, r_max):
    """A full-theta grid whose th spacing varies (nodes displaced by up to
    15 % of a cell, half nodes between them, the period kept): the spacing
    across the seam then differs from its neighbours'."""
    g = I.full_theta_grid(Nr, Nth, r_min, r_max)
    dth = 2.0 * math.pi / Nth
    u = np.arange(Nth + 1) / Nth
    tn = g.tn + 0.15 * dth * np.sin(2.0 * math.pi * u) * np.cos(6.0 * math.pi * u)
    th = 0.5 * (tn[:-1] + tn[1:]) + 0.1 * dth * np.sin(4.0 * math.pi * (u[:-1] + 0.5 / Nth))
    return I.Grid(g.Nr, g.Nth, g.rn, g.rh, tn, th, g.ld, True)


@pytest.mark.parametrize("uneven", [False, True])
@pytest.mark.parametrize("a", [0.0, 0.9])
def test_full_theta_fdtd_preserves_divergences_across_the_seam(a, uneven):
    """Sec. 2.1 / 2.5: on a full-theta grid the curl updates leave div B
    unchanged to round-off in every cell, the one across the seam (j = Nth-1,
    whose upper face is the image column) included, and div D in vacuum at
    every node, j = 0 (whose lower face is half node Nth-1, one period below)
    included; column Nth stays the bitwise image of column 0.  A wrong wrap
    index at the seam breaks these on any grid, a wrong spacing across it on
    the uneven one."""
    g = (_uneven_full_theta_grid if uneven else I.full_theta_grid)(24, 20, 1.9, 30.0)
    s = _rand_fields_full(g, 5)
    p = P.FdtdParams(1.0, a, 0.002, 1e4, 5.0, 0.9 * g.rn[-1], g.rn[-1], 0, 1)
    dB0, dD0 = P.div(1.0, a, g, s.B1, s.D1)
    for _ in range(3):
        P.fdtd(p, s, 1)
        P.fdtd(p, s, 2)
        s.swap()
    dB1, dD1 = P.div(1.0, a, g, s.B1, s.D1)
    for arrs in (s.B0, s.B1, s.D0, s.D1):
        for x in arrs:
            X = x.reshape(g.Nr + 1, g.ld)
            assert np.array_equal(X[:, g.Nth], X[:, 0])
    rm = g.rh < 0.9 * g.rn[-1] * 0.999
    ii = np.arange(g.Nr)[rm[:g.Nr]]
    ii = ii[ii < g.Nr - 2]
    sel = np.zeros((g.Nr + 1, g.ld), bool)
    sel[ii, :g.Nth] = True
    scale = np.abs(dB0).max()
    dB = np.abs((dB1 - dB0).reshape(g.Nr + 1, g.ld))
    assert dB[sel].max() < 1e-12 * scale
    assert dB[ii, g.Nth - 1].max() < 1e-12 * scale
    seld = np.zeros((g.Nr + 1, g.ld), bool)
    seld[2:ii.max(), :g.Nth] = True
    scale = np.abs(dD0).max()
    dD = np.abs((dD1 - dD0).reshape(g.Nr + 1, g.ld))
    assert dD[seld].max() < 1e-12 * scale
    assert dD[2:ii.max(), 0].max() < 1e-12 * scale
    # the seam column carries a divergence of its own (small: sqrt(gamma) ~ sin(dth / 4) there)
    assert np.abs(dD0.reshape(g.Nr + 1, g.ld)[2:ii.max(), 0]).max() > 1e-3 * scale


def test_full_theta_static_wald_stays_static_through_the_axes():
    """The a = 0 Wald field continued to th in (pi, 2 pi) with the signed
    sin th (reading 25) is a static vacuum solution on the full-theta grid:
    the leapfrog keeps it static up to the grid's truncation error, which
    falls at second order, alike in both half planes and in the bands
    around both axes (no axis boundary rows here); a wrong sign of
    sqrt(gamma) beyond th = pi would not be static there."""
    errs = {"north": [], "south": [], "axes": []}
    for N in (32, 64):
        g = I.full_theta_grid(N, 2 * N, 2.2, 12.0)
        F = O.wald_on_grid(0.0, 1.0, g)
        s = P.FdtdState(g)
        for k in range(3):
            s.D0[k][:] = F[k]; s.D1[k][:] = F[k]
            s.B0[k][:] = F[3 + k]; s.B1[k][:] = F[3 + k]
        p = P.FdtdParams(1.0, 0.0, 0.2 * (g.rn[1] - g.rn[0]), 0.0, 5.0, 1e9, 2e9, 0, 1)
        for _ in range(int(round(0.5 / p.dt))):
            P.fdtd(p, s, 1); P.fdtd(p, s, 2); s.swap()
        ri = (g.rn >= 4.0) & (g.rn <= 8.0)
        Br = s.B1[0].reshape(g.Nr + 1, g.ld)[ri][:, :g.Nth]
        Br0 = F[3].reshape(g.Nr + 1, g.ld)[ri][:, :g.Nth]
        for name, tj in (("north", (g.th >= 0.5) & (g.th <= math.pi - 0.5)),
                         ("south", (g.th >= math.pi + 0.5) & (g.th <= 2 * math.pi - 0.5)),
                         ("axes", np.abs(np.sin(g.th)) < 0.3)):
            errs[name].append(np.abs(Br[:, tj] - Br0[:, tj]).max() / np.abs(Br0).max())
    for name, e in errs.items():
        assert e[0] < 1e-4 and e[1] < 0.35 * e[0], (name, e)


def test_full_theta_fdtd_equals_the_half_theta_update_away_from_the_seam():
    """The full-theta mode changes the leapfrog only at the seam: on the same
    node tables, one full step (both stages) of the full and the half mode
    from the same random fields agree bit for bit on every column at least
    six cells from the seam and from the half mode's boundary rows."""
    a = 0.9
    g = I.full_theta_grid(16, 40, 1.9, 30.0)
    outs = []
    for full in (1, 0):
        s = _rand_fields_full(g, 8)
        rng = np.random.default_rng(9)
        for x in s.j0 + s.j1 + [s.rho0, s.rho1]:
            x[:] = rng.normal(size=g.size)
        p = P.FdtdParams(1.0, a, 0.002, 0.0, 5.0, g.rn[-1], g.rn[-1], 0, full)
        P.fdtd(p, s, 1)
        P.fdtd(p, s, 2)
        outs.append([x.reshape(g.Nr + 1, g.ld).copy() for x in s.B0 + s.D0 + s.Bh + s.Dw])
    for X, Y in zip(*outs):
        assert np.array_equal(X[:, 6:g.Nth - 6], Y[:, 6:g.Nth - 6])
    # and they do differ at the seam
    assert any(not np.array_equal(X[:, :2], Y[:, :2]) for X, Y in zip(*outs))
