"""Pins of the oracle's metric, derivatives, Wald field and Hamiltonian
against what the paper and textbook GR fix (no GPU)."""
import math

import numpy as np
import pytest

import oracle as O
from conftest import golden

SPINS = [0.0, 0.5, 0.9, 0.999]


def _pts(n=64, seed=0, rlo=1.3, rhi=40.0):
    rng = np.random.default_rng(seed)
    return rng.uniform(rlo, rhi, n), rng.uniform(0.05, math.pi - 0.05, n)


def _gamma_lower(m):
    g = np.zeros((m.shape[0], 3, 3))
    g[:, 0, 0], g[:, 0, 2], g[:, 2, 0] = m[:, 4], m[:, 5], m[:, 5]
    g[:, 1, 1], g[:, 2, 2] = m[:, 6], m[:, 7]
    return g


def _gamma_upper(m):
    g = np.zeros((m.shape[0], 3, 3))
    g[:, 0, 0], g[:, 0, 2], g[:, 2, 0] = m[:, 8], m[:, 9], m[:, 9]
    g[:, 1, 1], g[:, 2, 2] = m[:, 10], m[:, 11]
    return g


@pytest.mark.parametrize("a", SPINS)
def test_inverse_metric(a):
    """Appendix A: the printed gamma^ij is the inverse of gamma_ij (this pins
    the corrected gamma_{r phi} = -a xi sin^2 th)."""
    r, th = _pts()
    m = O.metric(1.0, a, r, th)
    prod = _gamma_lower(m) @ _gamma_upper(m)
    assert np.abs(prod - np.eye(3)).max() < 1e-13


@pytest.mark.parametrize("a", SPINS)
def test_determinant_and_lapse(a):
    """Eq. (det): gamma = rho^4 xi sin^2 th; alpha^2 xi = 1; beta = (xi-1)/xi."""
    r, th = _pts()
    m = O.metric(1.0, a, r, th)
    det = np.linalg.det(_gamma_lower(m))
    assert np.allclose(m[:, 12] ** 2, det, rtol=1e-12)
    assert np.allclose(m[:, 2] ** 2 * m[:, 1], 1.0, rtol=1e-14)
    rho2 = r ** 2 + a * a * np.cos(th) ** 2
    assert np.allclose(m[:, 0], rho2, rtol=1e-15)


@pytest.mark.parametrize("a", SPINS)
def test_kerr_schild_four_metric(a):
    """Textbook Kerr-Schild: g_tt = -alpha^2 + beta_r beta^r = -(1 - 2Mr/rho^2),
    g_tr = beta_r = 2Mr/rho^2, and g^rr = gamma^rr - beta^2/alpha^2 = Delta/rho^2
    with Delta = r^2 - 2Mr + a^2 (zero on the horizon)."""
    r, th = _pts()
    m = O.metric(1.0, a, r, th)
    rho2 = r ** 2 + a * a * np.cos(th) ** 2
    beta_lo = m[:, 4] * m[:, 3]
    gtt = -m[:, 2] ** 2 + beta_lo * m[:, 3]
    assert np.allclose(gtt, -(1 - 2 * r / rho2), rtol=1e-13, atol=1e-15)
    assert np.allclose(beta_lo, 2 * r / rho2, rtol=1e-13)
    grr_up = m[:, 8] - m[:, 3] ** 2 / m[:, 2] ** 2
    assert np.allclose(grr_up, (r * r - 2 * r + a * a) / rho2, rtol=1e-12, atol=1e-14)
    rh = 1 + math.sqrt(1 - a * a)
    mh = O.metric(1.0, a, np.full(5, rh), np.linspace(0.3, 2.8, 5))
    assert np.abs(mh[:, 8] - mh[:, 3] ** 2 / mh[:, 2] ** 2).max() < 1e-13


def test_schwarzschild_limit():
    """Appendix A: a -> 0 gives the diagonal Schwarzschild metric in KS form."""
    r, th = _pts()
    m = O.metric(1.0, 0.0, r, th)
    assert np.allclose(m[:, 4], 1 + 2 / r, rtol=1e-15)
    assert np.all(m[:, 5] == 0.0) and np.all(m[:, 9] == 0.0)
    assert np.allclose(m[:, 6], r * r, rtol=1e-15)
    assert np.allclose(m[:, 7], r * r * np.sin(th) ** 2, rtol=1e-14)
    assert np.allclose(m[:, 2], 1 / np.sqrt(1 + 2 / r), rtol=1e-15)


@pytest.mark.parametrize("a", SPINS)
def test_derivatives_against_richardson_differences(a):
    """Sec. 2.2: analytic derivatives of alpha, beta, gamma^ij equal the
    Richardson-extrapolated central differences of the metric itself (a
    dropped or mis-signed term would show as an O(1) relative error)."""
    r, th = _pts(24, seed=3)
    d = O.metric_deriv(1.0, a, r, th)
    cols = [2, 3, 8, 9, 10, 11]

    def cdiff(fr, h):
        return (fr(h) - fr(-h)) / (2 * h)

    for axis in range(2):
        def f(h):
            if axis == 0:
                return O.metric(1.0, a, r + h, th)[:, cols]
            return O.metric(1.0, a, r, th + h)[:, cols]
        h = 1e-3
        est = (4 * cdiff(f, h / 2) - cdiff(f, h)) / 3
        got = d[:, axis::2]
        scale = np.abs(est).max(axis=0) + 1e-12
        assert (np.abs(got - est) / scale).max() < 1e-7, axis


def test_table_c1_neutral_energies():
    """Table C.1 (neutral rows): H(x0, u0) = E to the 6 printed digits and
    u_ph = L exactly."""
    for name, (a, E, L, r0, ur, ut, up) in golden("table_c1_neutral.txt"):
        z = np.array([[r0, math.pi / 2, 0.0, ur, ut, up]])
        H, Lc, _ = O.hamiltonian(1.0, a, 0.0, z, 0.0)
        assert abs(H[0] - E) < 5e-7, name
        assert Lc[0] == L


def _A_from_eq_amu(a, B0, r, th):
    """Eq. (Amu) evaluated with the Kerr-Schild four-metric built from the
    oracle's 3+1 quantities: g_00 = -alpha^2 + beta_r beta^r, g_0i = beta_i."""
    m = O.metric(1.0, a, r, th)
    beta_r = m[:, 4] * m[:, 3]
    beta_p = m[:, 5] * m[:, 3]
    g00 = -m[:, 2] ** 2 + beta_r * m[:, 3]
    A0 = 0.5 * B0 * (beta_p + 2 * a * g00)
    Ar = 0.5 * B0 * (m[:, 5] + 2 * a * beta_r)
    Ap = 0.5 * B0 * (m[:, 7] + 2 * a * beta_p)
    return A0, Ar, Ap


@pytest.mark.parametrize("a", [0.0, 0.7, 0.9, 0.999])
def test_wald_potential_matches_eq_amu(a):
    """Sec. 3.1.3's A_0 and A_ph equal Eq. (Amu) (A_0 up to the constant -a B0)."""
    r, th = _pts(32, seed=5)
    _, _, _, A0, Aph = O.wald(a, 1.7, r, th)
    A0e, _, Ape = _A_from_eq_amu(a, 1.7, r, th)
    assert np.allclose(A0 - a * 1.7, A0e, rtol=1e-12, atol=1e-12)
    assert np.allclose(Aph, Ape, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("a", [0.0, 0.7, 0.9, 0.999])
def test_wald_fields_are_curl_and_gradient_of_eq_amu(a):
    """Appendix B.1: B^i = eta^ijk d_j A_k / sqrt(gamma) and E_i = d_i A_0 of
    Eq. (Amu), by central differences (pins the corrected E_th)."""
    B0 = 1.3
    r, th = _pts(32, seed=6)
    B, E, D, _, _ = O.wald(a, B0, r, th)
    h = 1e-5
    A0p, Arp, App = _A_from_eq_amu(a, B0, r + h, th)
    A0m, Arm, Apm = _A_from_eq_amu(a, B0, r - h, th)
    A0u, Aru, Apu = _A_from_eq_amu(a, B0, r, th + h)
    A0d, Ard, Apd = _A_from_eq_amu(a, B0, r, th - h)
    sg = O.metric(1.0, a, r, th)[:, 12]
    Br = (Apu - Apd) / (2 * h) / sg
    Bt = -(App - Apm) / (2 * h) / sg
    Bp = -(Aru - Ard) / (2 * h) / sg
    Er = (A0p - A0m) / (2 * h)
    Et = (A0u - A0d) / (2 * h)
    for got, exp in [(B[:, 0], Br), (B[:, 1], Bt), (B[:, 2], Bp), (E[:, 0], Er), (E[:, 1], Et)]:
        assert np.abs(got - exp).max() < 1e-7 * (np.abs(exp).max() + 1)
    assert np.all(E[:, 2] == 0)


def test_wald_D_satisfies_constitutive_relation():
    """Eq. (Ei): E_i = alpha D_i + sqrt(gamma) eta_ijk beta^j B^k with the
    oracle's D^i lowered by gamma_ij."""
    a = 0.9
    r, th = _pts(32, seed=7)
    B, E, D, _, _ = O.wald(a, 1.0, r, th)
    m = O.metric(1.0, a, r, th)
    Dlo = np.einsum("nij,nj->ni", _gamma_lower(m), D)
    al, be, sg = m[:, 2], m[:, 3], m[:, 12]
    assert np.allclose(E[:, 0], al * Dlo[:, 0], atol=1e-13)
    assert np.allclose(E[:, 1], al * Dlo[:, 1] - sg * be * B[:, 2], atol=1e-13)
    assert np.allclose(E[:, 2], al * Dlo[:, 2] + sg * be * B[:, 1], atol=1e-13)
