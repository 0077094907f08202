"""FPIC oracle: the plain serial FP64 CPU restatement of the GRPIC particle
path (arXiv 2602.07452), used ONLY as test infrastructure.

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library: the arithmetic lives in ``fpic_oracle.c`` (and ``fpic_oracle_pic.c``
for deposition and the field solver), compiled here with gcc at
``-O2 -ffp-contract=off`` and called through ctypes.

Parity status of each function is stated in its docstring; every function is
pinned by a ``-m "not gpu"`` test under ``tests/`` against a property the
paper or the mathematics fixes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SRCS = ["fpic_oracle.c", "fpic_oracle_pic.c", "fpic_oracle_mlp.c"]
_LIB = None
_LOCK = threading.Lock()

RK4, IMR, HAM, HYB1, HYB2 = 0, 1, 2, 3, 4
FIELD_NONE, FIELD_GRID, FIELD_WALD = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2 -ffp-contract=off)."""
    os.makedirs(_BUILD, exist_ok=True)
    out = os.path.join(_BUILD, "libfpic_oracle.so")
    srcs = [os.path.join(_HERE, s) for s in _SRCS if os.path.exists(os.path.join(_HERE, s))]
    if (not force and os.path.exists(out)
            and all(os.path.getmtime(out) >= os.path.getmtime(s) for s in srcs)):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-D_GNU_SOURCE",
           "-fPIC", "-shared", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            _LIB = C.CDLL(build())
            _declare(_LIB)
    return _LIB


class PushParams(C.Structure):
    """Mirror of ``or_push_params`` in fpic_oracle.c."""
    _fields_ = [("M", C.c_double), ("a", C.c_double), ("B0pot", C.c_double),
                ("field_kind", C.c_int), ("B0field", C.c_double), ("dt", C.c_double),
                ("scheme", C.c_int), ("implicit_kind", C.c_int), ("thr", C.c_double),
                ("tol", C.c_double), ("max_iter", C.c_int), ("r_h", C.c_double),
                ("r_max", C.c_double), ("dg_eps", C.c_double), ("dt_imp", C.c_double),
                ("imr_newton", C.c_int), ("imr_substeps", C.c_int), ("substep_tol", C.c_double),
                ("theta_full", C.c_int), ("theta_lo", C.c_double), ("theta_period", C.c_double)]


_D = C.POINTER(C.c_double)
_U8 = C.POINTER(C.c_uint8)
_U32 = C.POINTER(C.c_uint32)
_I64 = C.c_int64


def _declare(L):
    L.or_metric.argtypes = [C.c_double, C.c_double, _I64, _D, _D, _D]
    L.or_metric_deriv.argtypes = [C.c_double, C.c_double, _I64, _D, _D, _D]
    L.or_wald.argtypes = [C.c_double, C.c_double, _I64, _D, _D, _D, _D, _D, _D, _D]
    L.or_hamiltonian.argtypes = [C.c_double, C.c_double, C.c_double, _I64, _D, _D, _D, _D, _D]
    L.or_rhs.argtypes = [C.c_double, C.c_double, _I64, _D, _D, _D, _D, _D]
    L.or_imr_blocks.argtypes = [C.c_double, C.c_double, _I64, _D, _D, _D, _D, _D]
    L.or_gather.argtypes = [C.c_int, C.c_int, C.c_int, _D, _D, _D, _D, C.POINTER(_D), _I64, _D, _D, _D, C.c_int]
    L.or_cell_index.argtypes = [C.c_int, C.c_int, _D, _D, _I64, _D, _D, _U32]
    L.or_dg_grad.argtypes = [C.c_double, C.c_double, _D, _D, C.c_double, _D]
    L.or_dg_quot.argtypes = [C.c_double, C.c_double, _D, _D, C.c_int, _D]
    L.or_dg_quot_em.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double, _D, _D, C.c_int, _D]
    L.or_wald_A.argtypes = [C.c_double, C.c_double, _I64, _D, _D, _D, _D]
    L.or_push.argtypes = [C.POINTER(PushParams), C.c_int, C.c_int, C.c_int, _D, _D, _D, _D,
                          C.POINTER(_D), _I64, _D, _D, _D, _D, _D, _U8, _U8, _U8, _U8]
    L.or_push.restype = _I64
    L.or_wald_on_grid.argtypes = [C.c_double, C.c_double, C.c_int, C.c_int, C.c_int, _D, _D, _D, _D,
                                  C.POINTER(_D)]
    L.or_seed_orbits.argtypes = [C.c_double, C.c_double, _I64, C.c_int, _D, _D]
    L.or_seed_orbits.restype = _I64
    L.or_seed_fido.argtypes = [C.c_double, C.c_double, _I64, _D, _D]
    if hasattr(L, "or_deposit"):
        from . import pic as _pic  # noqa: F401  (declares its own symbols)
        _pic._declare(L)
    if hasattr(L, "or_mlp_forward"):
        from . import mlp as _mlp
        _mlp._declare(L)


def f64(x):
    return np.ascontiguousarray(x, dtype=np.float64)


def ptr(a: np.ndarray, t=_D):
    return a.ctypes.data_as(t)


def _fields_ptrs(F):
    arr = (_D * 6)(*[ptr(f) for f in F])
    return arr


# ---------------------------------------------------------------------------
# Metric, fields, Hamiltonian (Appendix A, Appendix B.1, Eq. Ham)
# ---------------------------------------------------------------------------

def metric(M, a, r, th):
    """Appendix A.  Columns: rho2, xi, alpha, beta, g_rr, g_rp, g_tt, g_pp,
    g^rr, g^rp, g^tt, g^pp, sqrt(gamma)."""
    r, th = f64(np.atleast_1d(r)), f64(np.atleast_1d(th))
    out = np.empty((r.size, 13))
    lib().or_metric(M, a, r.size, ptr(r), ptr(th), ptr(out))
    return out


def metric_deriv(M, a, r, th):
    """(d_r, d_th) of alpha, beta, g^rr, g^rp, g^tt, g^pp (Sec. 2.2)."""
    r, th = f64(np.atleast_1d(r)), f64(np.atleast_1d(th))
    out = np.empty((r.size, 12))
    lib().or_metric_deriv(M, a, r.size, ptr(r), ptr(th), ptr(out))
    return out


def wald(a, B0, r, th):
    """Appendix B.1 (M = 1): returns B^i, E_i, D^i, A_0, A_phi."""
    r, th = f64(np.atleast_1d(r)), f64(np.atleast_1d(th))
    n = r.size
    B, E, D = np.empty((n, 3)), np.empty((n, 3)), np.empty((n, 3))
    A0, Aph = np.empty(n), np.empty(n)
    lib().or_wald(a, B0, n, ptr(r), ptr(th), ptr(B), ptr(E), ptr(D), ptr(A0), ptr(Aph))
    return B, E, D, A0, Aph


def hamiltonian(M, a, B0pot, z, qm):
    """H (Eq. Ham with the Wald A_0), L and the error normaliser D_0."""
    z = f64(z).reshape(-1, 6)
    qm = f64(np.broadcast_to(qm, (z.shape[0],)))
    n = z.shape[0]
    H, L, Dn = np.empty(n), np.empty(n), np.empty(n)
    lib().or_hamiltonian(M, a, B0pot, n, ptr(z), ptr(qm), ptr(H), ptr(L), ptr(Dn))
    return H, L, Dn


def rhs(M, a, z, qm, D=None, B=None):
    """Eqs. (p1), (p2), (O1), (O2)."""
    z = f64(z).reshape(-1, 6)
    n = z.shape[0]
    qm = f64(np.broadcast_to(qm, (n,)))
    f = np.empty((n, 6))
    Dp = Bp = None
    if D is not None:
        Dk, Bk = f64(D).reshape(n, 3), f64(B).reshape(n, 3)
        Dp, Bp = ptr(Dk), ptr(Bk)
    lib().or_rhs(M, a, n, ptr(z), ptr(qm), Dp, Bp, ptr(f))
    return f


def imr_blocks(M, a, z, qm, B=None):
    """Momentum blocks (A, J), each (n, 3, 3), of the IMR Newton matrix (Sec. 2.2.2)."""
    z = f64(z).reshape(-1, 6)
    n = z.shape[0]
    qm = f64(np.broadcast_to(qm, (n,)))
    A, J = np.empty((n, 3, 3)), np.empty((n, 3, 3))
    Bp = None if B is None else ptr(f64(B).reshape(n, 3))
    lib().or_imr_blocks(M, a, n, ptr(z), ptr(qm), Bp, ptr(A), ptr(J))
    return A, J


def dg_quot(M, a, zb, za, v):
    """Closed-form quotient (H(za) - H(zb)) / (za_v - zb_v) of a single-variable move."""
    out = np.zeros(1)
    lib().or_dg_quot(M, a, ptr(f64(zb)), ptr(f64(za)), int(v), ptr(out))
    return float(out[0])


def dg_quot_em(M, a, B0, qm, wb, wa, v):
    """Charged closed-form quotient in canonical variables (Wald field)."""
    out = np.zeros(1)
    lib().or_dg_quot_em(M, a, B0, qm, ptr(f64(wb)), ptr(f64(wa)), int(v), ptr(out))
    return float(out[0])


def wald_A(a, B0, r, th):
    """A_r and A_ph of Eq. (Amu) (M = 1)."""
    r, th = f64(np.atleast_1d(r)), f64(np.atleast_1d(th))
    Ar, Aph = np.empty(r.size), np.empty(r.size)
    lib().or_wald_A(a, B0, r.size, ptr(r), ptr(th), ptr(Ar), ptr(Aph))
    return Ar, Aph


def dg_grad(M, a, z0, z1, eps=1e-10):
    """Symmetrised coordinate-increment discrete gradient (Sec. 2.2.3)."""
    z0, z1 = f64(z0), f64(z1)
    G = np.empty(6)
    lib().or_dg_grad(M, a, ptr(z0), ptr(z1), eps, ptr(G))
    return G


# ---------------------------------------------------------------------------
# Grid-based pieces
# ---------------------------------------------------------------------------

def _grid_args(g):
    return (g.Nr, g.Nth, g.ld, ptr(g.rn), ptr(g.rh), ptr(g.tn), ptr(g.th))


def gather(g, F, r, t):
    """Bilinear (r, th) gather of the six Yee components at points."""
    r, t = f64(np.atleast_1d(r)), f64(np.atleast_1d(t))
    F = [f64(f) for f in F]
    out = np.empty((r.size, 6))
    lib().or_gather(*_grid_args(g), _fields_ptrs(F), r.size, ptr(r), ptr(t), ptr(out),
                    int(getattr(g, "full_theta", False)))
    return out


def cell_index(g, r, t):
    r, t = f64(np.atleast_1d(r)), f64(np.atleast_1d(t))
    out = np.empty(r.size, dtype=np.uint32)
    lib().or_cell_index(g.Nr, g.Nth, ptr(g.rn), ptr(g.tn), r.size, ptr(r), ptr(t), ptr(out, _U32))
    return out


def wald_on_grid(a, B0, g):
    """Appendix B.1 sampled at every Yee point; returns [D^r, D^th, D^ph, B^r, B^th, B^ph].
    Full-theta grid: column Nth of every component is the periodic image of
    column 0 (copied, so the two are equal bit for bit)."""
    F = [np.zeros((g.Nr + 1) * g.ld) for _ in range(6)]
    arr = (_D * 6)(*[ptr(f) for f in F])
    lib().or_wald_on_grid(a, B0, *_grid_args(g), arr)
    if getattr(g, "full_theta", False):
        for f in F:
            v = f.reshape(g.Nr + 1, g.ld)
            v[:, g.Nth] = v[:, 0]
    return F


def push_params(M=1.0, a=0.9, B0pot=0.0, field_kind=FIELD_NONE, B0field=0.0, dt=0.01,
                scheme=RK4, implicit_kind=IMR, thr=1e-12, tol=1e-14, max_iter=50,
                r_h=None, r_max=1e300, dg_eps=1e-10, dt_imp=0.0, imr_newton=False, imr_substeps=0,
                substep_tol=0.0, grid=None):
    """grid: with a full-theta grid (inputs.full_theta_grid) the particles'
    th boundary is periodic over its period; otherwise the half-theta
    reflection at the poles."""
    if r_h is None:
        r_h = M + np.sqrt(M * M - a * a)
    full = grid is not None and getattr(grid, "full_theta", False)
    lo, per = (float(grid.tn[0]), float(grid.tn[-1] - grid.tn[0])) if full else (0.0, 0.0)
    return PushParams(M, a, B0pot, field_kind, B0field, dt, scheme, implicit_kind, thr, tol,
                      max_iter, r_h, r_max, dg_eps, dt_imp, int(bool(imr_newton)), int(imr_substeps),
                      float(substep_tol), int(full), lo, per)


def push(p: PushParams, z, qm, H0, D0, Hn, alive, g=None, F=None, flags=False):
    """One step of all particles, in place on z (n x 6), Hn and alive.
    Returns (n_not_converged, scheme[n], iters[n]), and with flags=True also
    the per-particle not-converged flags."""
    n = z.shape[0]
    assert z.dtype == np.float64 and z.flags.c_contiguous
    sch = np.zeros(n, np.uint8)
    its = np.zeros(n, np.uint8)
    if g is not None:
        Fk = [f64(f) for f in F]
        gargs = _grid_args(g)
        Fp = _fields_ptrs(Fk)
    else:
        e = np.zeros(2)
        gargs = (1, 1, 2, ptr(e), ptr(e), ptr(e), ptr(e))
        Fp = None
    ncf = np.zeros(n, np.uint8)
    nc = lib().or_push(C.byref(p), *gargs, Fp, n, ptr(z), ptr(f64(qm)), ptr(f64(H0)),
                       ptr(f64(D0)), ptr(Hn), ptr(alive, _U8), ptr(sch, _U8), ptr(its, _U8), ptr(ncf, _U8))
    return (nc, sch, its, ncf) if flags else (nc, sch, its)


def seed_orbits(M, a, cand):
    """Bound-orbit initial states from candidates (n, K, 5)."""
    cand = f64(cand)
    n, K, _ = cand.shape
    z = np.empty((n, 6))
    bad = lib().or_seed_orbits(M, a, n, K, ptr(cand), ptr(z))
    return z, bad


def seed_fido(M, a, draws):
    """Thermal initial states from FIDO-frame draws (n, 6)."""
    draws = f64(draws)
    z = np.empty((draws.shape[0], 6))
    lib().or_seed_fido(M, a, draws.shape[0], ptr(draws), ptr(z))
    return z
