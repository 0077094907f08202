"""Oracle wrappers for deposition and the FDTD leapfrog (fpic_oracle_pic.c).
Test infrastructure only."""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _D, _U8, f64, lib, ptr

_I64 = C.c_int64


class FdtdParams(C.Structure):
    _fields_ = [("M", C.c_double), ("a", C.c_double), ("dt", C.c_double), ("chi0", C.c_double),
                ("lam", C.c_double), ("r_abs", C.c_double), ("r_max", C.c_double), ("conserving", C.c_int),
                ("full", C.c_int)]


def _declare(L):
    g = [C.c_int, C.c_int, C.c_int, _D, _D, _D, _D]
    L.or_deposit.argtypes = [C.c_double, C.c_double] + g + [_I64, _D, _D, _D, _U8, _D, _D, _D, _D,
                                                            C.c_int, C.c_int]
    L.or_dual_volumes.argtypes = [C.c_double, C.c_double] + g + [_D, _D, _D]
    P3 = _D * 3
    L.or_fdtd.argtypes = [C.POINTER(FdtdParams)] + g + [C.c_int, P3, P3, P3, P3, P3, _D, P3, _D, P3, P3, P3, P3]
    L.or_div.argtypes = [C.c_double, C.c_double] + g + [P3, P3, _D, _D, C.c_int]
    L.or_split_monopole_on_grid.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double] + g + [_D * 6]
    L.or_bz_power.argtypes = [C.c_int, C.c_int, C.c_int, _D, P3, P3, C.c_int]
    L.or_bz_power.restype = C.c_double
    L.or_div_clean.argtypes = [C.c_double, C.c_double] + g + [P3, _D, C.c_int, _D]
    L.or_inject_pairs.argtypes = [C.c_double, C.c_double] + g + [_D, _D] + [C.c_double] * 5 + [
        _D, _I64, _I64, _D, _D, _D, _U8, _U8, C.POINTER(_I64)]
    L.or_inject_pairs.restype = _I64
    L.or_deposit_conserving.argtypes = [C.c_double, C.c_double] + g + [_I64, _D, _D, _D, _D, _U8, C.c_double,
                                                                       _D, _D, _D, _D]
    L.or_deposit_conserving.restype = _I64


def _g(g):
    return (g.Nr, g.Nth, g.ld, ptr(g.rn), ptr(g.rh), ptr(g.tn), ptr(g.th))


def deposit(M, a, g, z, qm, w, alive=None, unit=False, normalise=True):
    """Sec. 2.3: returns (rho, j^r, j^th, j^ph) on their Yee sub-grids."""
    z = f64(z).reshape(-1, 6)
    n = z.shape[0]
    alive = np.ones(n, np.uint8) if alive is None else np.ascontiguousarray(alive, np.uint8)
    out = [np.zeros(g.size) for _ in range(4)]
    lib().or_deposit(M, a, *_g(g), n, ptr(z), ptr(f64(qm)), ptr(f64(w)), ptr(alive, _U8),
                     ptr(out[0]), ptr(out[1]), ptr(out[2]), ptr(out[3]), int(unit), int(normalise))
    return tuple(out)


def dual_volumes(M, a, g):
    """2 pi x dual-cell volumes of the (i,j), (i+1/2,j), (i,j+1/2) sub-grids."""
    v = [np.zeros(g.size) for _ in range(3)]
    lib().or_dual_volumes(M, a, *_g(g), ptr(v[0]), ptr(v[1]), ptr(v[2]))
    return tuple(v)


def _p3(arrs):
    return (_D * 3)(*[ptr(x) for x in arrs])


class FdtdState:
    """Field storage of the leapfrog: B0, B1, D0, D1 (3 comps each), sources
    (j0, rho0), (j1, rho1) and the work arrays E, H, Bh, Dw."""

    def __init__(self, g):
        z = lambda: [np.zeros(g.size) for _ in range(3)]
        self.g = g
        self.B0, self.B1, self.D0, self.D1 = z(), z(), z(), z()
        self.j0, self.j1 = z(), z()
        self.rho0, self.rho1 = np.zeros(g.size), np.zeros(g.size)
        self.E, self.H, self.Bh, self.Dw = z(), z(), z(), z()

    def swap(self):
        self.B0, self.B1 = self.B1, self.B0
        self.D0, self.D1 = self.D1, self.D0
        self.j0, self.j1 = self.j1, self.j0
        self.rho0, self.rho1 = self.rho1, self.rho0


def fdtd(p: FdtdParams, s: FdtdState, stage: int):
    """Sub-steps 1-4 (stage 1) or 7-10 (stage 2) of Sec. 2.1, in place."""
    lib().or_fdtd(C.byref(p), *_g(s.g), stage, _p3(s.B0), _p3(s.B1), _p3(s.D0), _p3(s.D1), _p3(s.j0),
                  ptr(s.rho0), _p3(s.j1), ptr(s.rho1), _p3(s.E), _p3(s.H), _p3(s.Bh), _p3(s.Dw))


def div(M, a, g, B, D):
    """sqrtg-weighted Yee divergences: div B at cell centres, div D at nodes
    (at j = 0 too, across the seam, on a full-theta grid)."""
    dB, dD = np.zeros(g.size), np.zeros(g.size)
    lib().or_div(M, a, *_g(g), _p3([f64(x) for x in B]), _p3([f64(x) for x in D]), ptr(dB), ptr(dD),
                 int(getattr(g, "full_theta", False)))
    return dB, dD


def split_monopole_on_grid(M, a, B0, zeta0, g):
    """Sec. 3.4 / App. B.2 vacuum split monopole: (D^r, D^th, D^ph, B^r, B^th, B^ph)."""
    F = [np.zeros(g.size) for _ in range(6)]
    lib().or_split_monopole_on_grid(M, a, B0, zeta0, *_g(g), (_D * 6)(*[ptr(x) for x in F]))
    return F


def bz_power(g, E, H, i):
    """Eq. (Pbz) on the sphere r = rh[i] from the auxiliary fields E_i, H_i."""
    return lib().or_bz_power(g.Nr, g.Nth, g.ld, ptr(g.tn), _p3([f64(x) for x in E]), _p3([f64(x) for x in H]), i)


def div_clean(M, a, g, D, rho, n_iter):
    """Sec. 2.4 divergence cleaning of D (list of 3 arrays, returned corrected
    copies) against rho with n_iter Jacobi sweeps; also returns phi."""
    Dc = [f64(x).copy() for x in D]
    phi = np.zeros(g.size)
    lib().or_div_clean(M, a, *_g(g), _p3(Dc), ptr(f64(rho)), int(n_iter), ptr(phi))
    return Dc, phi


def inject_pairs(M, a, g, z, qm, w, alive, n, cap, Br, Bth, r_lo, r_hi, mult, n0, qm_e, draws):
    """Sec. 3.3 / 3.4 pair injection on copies of capacity-sized arrays
    (z: cap x 6, the first n in use).  Returns (z, qm, w, alive, n_new,
    pairs wanted, per-cell flags)."""
    z = np.ascontiguousarray(f64(z).copy()).reshape(-1, 6)
    qm, w = f64(qm).copy(), f64(w).copy()
    alive = np.ascontiguousarray(alive, dtype=np.uint8).copy()
    assert z.shape[0] >= cap and qm.size >= cap and w.size >= cap and alive.size >= cap
    flags = np.zeros(g.Nr * g.Nth, np.uint8)
    d = np.ascontiguousarray(f64(draws))
    assert d.size >= 9 * g.Nr * g.Nth
    n_out = C.c_int64(0)
    K = lib().or_inject_pairs(M, a, *_g(g), ptr(f64(Br)), ptr(f64(Bth)), r_lo, r_hi, mult, n0, qm_e, ptr(d),
                              int(n), int(cap), ptr(z), ptr(qm), ptr(w),
                              ptr(alive, _U8), ptr(flags, _U8), C.byref(n_out))
    return z, qm, w, alive, int(n_out.value), int(K), flags


def deposit_conserving(M, a, g, z0, z1, qm, w, alive, dt):
    """Charge-conserving deposit of the moves z0 -> z1: (rho at z1 in the Yee
    node volume, coordinate currents J^r, J^th, J^ph, moves skipped)."""
    z0 = np.ascontiguousarray(f64(z0)).reshape(-1, 6)
    z1 = np.ascontiguousarray(f64(z1)).reshape(-1, 6)
    n = z0.shape[0]
    alive = np.ascontiguousarray(alive, np.uint8)
    out = [np.zeros(g.size) for _ in range(4)]
    sk = lib().or_deposit_conserving(M, a, *_g(g), n, ptr(z0), ptr(z1), ptr(f64(qm)), ptr(f64(w)),
                                     ptr(alive, _U8), float(dt), *[ptr(x) for x in out])
    return out[0], out[1], out[2], out[3], int(sk)
