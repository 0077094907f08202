"""Seeded synthetic inputs for the GRPIC hot path.

This module holds random draws and grid node tables only -- none of the
method's arithmetic (no metric, no Hamiltonian, no pusher).  Both the CUDA
path (through the library's own initialisation kernels) and the CPU oracle
consume what it produces, so the two sides start from identical numbers.

Workloads (the paper's test-particle and plasma set-ups, Secs. 3.1-3.3):
  * orbit candidates: r ~ U[3, 20] M, th ~ U(0.1, pi - 0.1), E ~ U[0.9, 0.98],
    L ~ U[2.5, 4.5], root sign +-1, K candidates per particle;
  * thermal draws: ln r ~ U[ln r_lo, ln r_hi], th ~ U over the node range,
    ph ~ U[0, 2 pi), FIDO-frame momentum isotropic with |u| drawn from the
    Maxwell-Juettner law of temperature theta_T (tabulated inverse CDF),
    species alternating e-/e+.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class Grid:
    """Node tables of the axisymmetric (r, th) Yee grid.

    Nr, Nth  : number of cells in r and th
    rn, rh   : integer r nodes (Nr + 1) and half nodes r_{i+1/2} (Nr)
    tn, th   : integer th nodes (Nth + 1) and half nodes (Nth)
    ld       : leading dimension of every field array ([i * ld + j])
    full_theta : th spans one full period [tn[0], tn[0] + 2 pi) with
               periodic boundaries (tn[Nth] = tn[0] + 2 pi is the image of
               tn[0]; column Nth of every field array holds the image of
               column 0); False: the half-theta domain between the poles
    """
    Nr: int
    Nth: int
    rn: np.ndarray
    rh: np.ndarray
    tn: np.ndarray
    th: np.ndarray
    ld: int
    full_theta: bool = False

    @property
    def size(self) -> int:
        return (self.Nr + 1) * self.ld


def horizon(M: float, a: float) -> float:
    """Outer horizon radius r_+ = M + sqrt(M^2 - a^2) (grid extent only)."""
    return M + math.sqrt(M * M - a * a)


def log_grid(Nr: int, Nth: int, r_min: float, r_max: float,
             th_min: float | None = None, th_max: float | None = None) -> Grid:
    """Grid uniform in ln r and in th.  Default th range puts both poles half a
    cell outside the end nodes: dth = pi/(Nth+1), th_0 = dth/2, th_N = pi - dth/2."""
    if th_min is None or th_max is None:
        dth = math.pi / (Nth + 1)
        th_min, th_max = 0.5 * dth, math.pi - 0.5 * dth
    lr = np.linspace(math.log(r_min), math.log(r_max), Nr + 1)
    rn = np.exp(lr)
    rh = np.exp(0.5 * (lr[:-1] + lr[1:]))
    tn = np.linspace(th_min, th_max, Nth + 1)
    th = 0.5 * (tn[:-1] + tn[1:])
    return Grid(Nr, Nth, rn, rh, tn, th, Nth + 1)


def full_theta_grid(Nr: int, Nth: int, r_min: float, r_max: float) -> Grid:
    """Full-theta domain (Sec. 2.5): th nodes eps + j dth, j = 0..Nth, with
    dth = 2 pi / Nth and eps = pi / (2 Nth) = dth / 4, half nodes midway;
    both poles (th = pi and th = 0 = 2 pi) then lie midway between a half
    node and a node.  Nth must be even.  Uniform in ln r as log_grid."""
    if Nth % 2:
        raise ValueError("full_theta_grid: Nth must be even")
    lr = np.linspace(math.log(r_min), math.log(r_max), Nr + 1)
    rn = np.exp(lr)
    rh = np.exp(0.5 * (lr[:-1] + lr[1:]))
    dth = 2.0 * math.pi / Nth
    tn = 0.25 * dth + dth * np.arange(Nth + 1)
    th = tn[:-1] + 0.5 * dth
    return Grid(Nr, Nth, rn, rh, tn, th, Nth + 1, True)


def wald_grid(N: int, a: float, M: float = 1.0, r_max: float = 50.0) -> Grid:
    """(ln r, th) grid of the charged test-particle workload:
    r in [0.9 r_+, r_max], th in [0, pi] with the poles between nodes."""
    return log_grid(N, N, 0.9 * horizon(M, a), r_max)


def orbit_candidates(n: int, K: int = 256, seed: int = 1) -> np.ndarray:
    """(n, K, 5) candidates (r, th, E, L, sign) for bound neutral orbits."""
    rng = np.random.default_rng(seed)
    c = np.empty((n, K, 5))
    c[..., 0] = rng.uniform(3.0, 20.0, (n, K))
    c[..., 1] = rng.uniform(0.1, math.pi - 0.1, (n, K))
    c[..., 2] = rng.uniform(0.9, 0.98, (n, K))
    c[..., 3] = rng.uniform(2.5, 4.5, (n, K))
    c[..., 4] = np.where(rng.random((n, K)) < 0.5, -1.0, 1.0)
    return c


def _mj_inverse_cdf(theta: float, m: int = 1 << 16):
    """Tabulated CDF of |u| for f(u) ~ u^2 exp(-sqrt(1+u^2)/theta)."""
    umax = 1.0
    while True:   # extend until the tail weight is negligible
        g = math.sqrt(1.0 + umax * umax)
        if umax * umax * math.exp(-(g - 1.0) / theta) < 1e-18:
            break
        umax *= 1.5
    u = np.linspace(0.0, umax, m)
    pdf = u * u * np.exp(-(np.sqrt(1.0 + u * u) - 1.0) / theta)
    cdf = np.concatenate([[0.0], np.cumsum(0.5 * (pdf[1:] + pdf[:-1]) * np.diff(u))])
    cdf /= cdf[-1]
    return u, cdf


def maxwell_juettner(rng: np.random.Generator, n: int, theta: float) -> np.ndarray:
    """(n, 3) isotropic momenta with |u| ~ Maxwell-Juettner(theta)."""
    u, cdf = _mj_inverse_cdf(theta)
    mag = np.interp(rng.random(n), cdf, u)
    cz = rng.uniform(-1.0, 1.0, n)
    ph = rng.uniform(0.0, 2.0 * math.pi, n)
    sz = np.sqrt(1.0 - cz * cz)
    return np.stack([mag * sz * np.cos(ph), mag * sz * np.sin(ph), mag * cz], axis=1)


def thermal_draws(n: int, g: Grid, r_lo: float, r_hi: float, theta_T: float,
                  seed: int = 2, qm: float = 100.0):
    """Draws for the thermal pair workload.

    Returns (draws (n, 6) = (r, th, ph, uhat_r, uhat_th, uhat_ph), qm (n,),
    w (n,)): species alternate e- (q/m = -qm) and e+ (+qm), unit weight."""
    rng = np.random.default_rng(seed)
    d = np.empty((n, 6))
    d[:, 0] = np.exp(rng.uniform(math.log(r_lo), math.log(r_hi), n))
    d[:, 1] = rng.uniform(g.tn[0], g.tn[-1], n)
    d[:, 2] = rng.uniform(0.0, 2.0 * math.pi, n)
    d[:, 3:] = maxwell_juettner(rng, n, theta_T)
    q = np.where(np.arange(n) % 2 == 0, -qm, qm).astype(np.float64)
    return d, q, np.ones(n)


def cell_fill_draws(g: Grid, ppc: int, theta_T: float, seed: int = 3, qm: float = 100.0,
                    r_lo: float | None = None):
    """Draws for the plasma-filled workload: ppc particles (ppc/2 pairs) in
    every cell with r >= r_lo, uniform in (ln r, th) inside the cell."""
    rng = np.random.default_rng(seed)
    i = np.arange(g.Nr)
    if r_lo is not None:
        i = i[g.rn[1:] > r_lo]
    ii, jj = np.meshgrid(i, np.arange(g.Nth), indexing="ij")
    ii = np.repeat(ii.ravel(), ppc)
    jj = np.repeat(jj.ravel(), ppc)
    n = ii.size
    lr0, lr1 = np.log(g.rn[ii]), np.log(g.rn[ii + 1])
    d = np.empty((n, 6))
    d[:, 0] = np.exp(lr0 + rng.random(n) * (lr1 - lr0))
    if r_lo is not None:
        d[:, 0] = np.maximum(d[:, 0], r_lo)
    d[:, 1] = g.tn[jj] + rng.random(n) * (g.tn[jj + 1] - g.tn[jj])
    d[:, 2] = rng.uniform(0.0, 2.0 * math.pi, n)
    d[:, 3:] = maxwell_juettner(rng, n, theta_T)
    q = np.where(np.arange(n) % 2 == 0, -qm, qm).astype(np.float64)
    return d, q, np.ones(n)


def injection_draws(g: Grid, theta_T: float, seed: int = 4) -> np.ndarray:
    """Random numbers of one pair injection: (Nr Nth, 9) per cell c = i Nth + j
    = (u_r, u_th, u_ph) uniform in [0, 1), then the FIDO-frame momenta of the
    electron and of the positron, each Maxwell-Juttner(theta_T)."""
    rng = np.random.default_rng(seed)
    C = g.Nr * g.Nth
    d = np.empty((C, 9))
    d[:, :3] = rng.random((C, 3))
    d[:, 3:6] = maxwell_juettner(rng, C, theta_T)
    d[:, 6:9] = maxwell_juettner(rng, C, theta_T)
    return d
