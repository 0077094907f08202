"""Thin ctypes binding of libfpic.so: the C ABI of include/fpic.h, same names.

Argument marshalling only -- every step runs in the library's CUDA kernels.
PyTorch supplies device memory and streams.  Importing this module does not
load the library; the first call does, and it raises if libfpic.so is
missing (build it with ``paper_2602_07452_gb300.build.build()``).
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from dataclasses import dataclass

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libfpic.so")

FPIC_OK, FPIC_EINVAL, FPIC_ECUDA, FPIC_ENOMEM, FPIC_ETIMEOUT = 0, -1, -2, -3, -4
FPIC_ENOTCONVERGED = 1
FPIC_RK4, FPIC_IMR, FPIC_HAM, FPIC_HYB1, FPIC_HYB2 = 0, 1, 2, 3, 4
FPIC_SEED_ORBIT, FPIC_SEED_FIDO = 0, 1

_lib = None
_lock = threading.Lock()


class FpicError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"fpic error {code}: {msg}")
        self.code = code


_D = C.POINTER(C.c_double)
_U8 = C.POINTER(C.c_uint8)
_U32 = C.POINTER(C.c_uint32)


class fpic_particles(C.Structure):
    _fields_ = [("n", C.c_int64), ("r", _D), ("th", _D), ("ph", _D), ("ur", _D), ("uth", _D),
                ("uph", _D), ("qm", _D), ("w", _D), ("H0", _D), ("D0", _D), ("Hn", _D),
                ("alive", _U8), ("scheme", _U8), ("iters", _U8), ("cell", _U32)]


class fpic_push_params(C.Structure):
    _fields_ = [("dt", C.c_double), ("scheme", C.c_int), ("implicit", C.c_int), ("thr", C.c_double),
                ("tol", C.c_double), ("max_iter", C.c_int), ("r_max", C.c_double),
                ("dg_eps", C.c_double), ("B0pot", C.c_double), ("guess", C.c_void_p),
                ("events", C.c_void_p), ("dt_implicit", C.c_double), ("t", C.c_void_p), ("B0field", C.c_double),
                ("imr_newton", C.c_int), ("imr_substeps", C.c_int), ("substep_tol", C.c_double),
                ("before", C.POINTER(fpic_particles))]


class fpic_push_stats(C.Structure):
    _fields_ = [("n_alive_before", C.c_int64), ("n_implicit", C.c_int64), ("n_iter_total", C.c_int64),
                ("n_notconv", C.c_int64), ("n_removed", C.c_int64), ("n_rhs_evals", C.c_int64),
                ("n_slope_reused", C.c_int64), ("n_tiles_staged", C.c_int64)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


_P3 = _D * 3


class fpic_inject_params(C.Structure):
    _fields_ = [("r_lo", C.c_double), ("r_hi", C.c_double), ("multiplicity", C.c_double), ("n0", C.c_double),
                ("qm_e", C.c_double), ("B0pot", C.c_double)]


class fpic_fields(C.Structure):
    _fields_ = [("B0", _P3), ("B1", _P3), ("D0", _P3), ("D1", _P3), ("j0", _P3), ("rho0", _D),
                ("j1", _P3), ("rho1", _D), ("E", _P3), ("H", _P3), ("Bh", _P3), ("Dw", _P3)]


class fpic_fdtd_params(C.Structure):
    _fields_ = [("dt", C.c_double), ("chi0", C.c_double), ("lam", C.c_double), ("r_abs", C.c_double),
                ("r_max", C.c_double), ("conserving", C.c_int)]


class fpic_run(C.Structure):
    _fields_ = [("ctx", C.c_void_p), ("fields", _D * 6), ("begin", C.c_int64), ("end", C.c_int64),
                ("r_max", C.c_double), ("B0pot", C.c_double)]


class fpic_learned_cfg(C.Structure):
    _fields_ = [("feat_mean", C.c_float * 16), ("feat_std", C.c_float * 16), ("inc_scale", C.c_double * 6),
                ("p_skip", C.c_float),
                ("mode", C.c_int),
                ("restart_after", C.c_int)]


FPIC_LEARN_SKIP, FPIC_LEARN_CORRECT = 0, 1
FPIC_TUNE_IMR_BLOCKS_PER_SM, FPIC_TUNE_DEP_THREADS, FPIC_TUNE_STATIC_FIELDS, FPIC_TUNE_REUSE_SLOPE = 0, 1, 2, 3
FPIC_TUNE_STAGE_FIELDS = 4
FPIC_TUNE_DEP_LATTICE = 5
FPIC_TUNE_ASYNC = 6
FPIC_TUNE_HOST_STAGING = 7
FPIC_THETA_HALF, FPIC_THETA_FULL = 0, 1


# name -> (restype, argtypes)
_SIGS = {
    "fpic_push_batched": (C.c_int, [C.POINTER(fpic_run), C.c_int, C.POINTER(fpic_particles),
                                    C.POINTER(fpic_push_params), C.POINTER(fpic_push_stats), C.c_void_p]),
    "fpic_push_batched_learned": (C.c_int, [C.POINTER(fpic_run), C.c_int, C.c_void_p, C.POINTER(fpic_particles),
                                            C.POINTER(fpic_push_params), C.POINTER(fpic_learned_cfg),
                                            C.POINTER(fpic_push_stats), C.c_void_p]),
    "fpic_features": (C.c_int, [C.c_void_p, C.POINTER(fpic_particles), C.POINTER(_D), C.c_double,
                                C.POINTER(fpic_learned_cfg), C.c_void_p, C.c_void_p]),
    "fpic_learn_sample": (C.c_int, [C.c_void_p, C.POINTER(fpic_particles), C.POINTER(_D), C.POINTER(fpic_push_params),
                                    C.POINTER(fpic_learned_cfg), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "fpic_push_learned": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(fpic_particles), C.POINTER(_D),
                                    C.POINTER(fpic_push_params), C.POINTER(fpic_learned_cfg),
                                    C.POINTER(fpic_push_stats), C.c_void_p]),
    "fpic_mma_bf16": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_int, C.c_int,
                                C.c_int, C.c_int, C.c_void_p, C.c_void_p]),
    "fpic_mlp_create": (C.c_int, [C.POINTER(C.c_void_p)]),
    "fpic_mlp_destroy": (None, [C.c_void_p]),
    "fpic_mlp_nparams": (C.c_longlong, []),
    "fpic_mlp_set_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "fpic_mlp_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_longlong, C.c_void_p]),
    "fpic_mlp_status": (C.c_int, [C.c_void_p, C.POINTER(C.c_int)]),
    "fpic_mlp_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_float), C.c_longlong,
                                C.c_void_p, C.POINTER(C.c_float), C.c_void_p]),
    "fpic_mlp_train_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_void_p, C.POINTER(C.c_float), C.c_longlong, C.c_int, C.c_float, C.c_float,
                                      C.c_float, C.c_float, C.POINTER(C.c_float), C.c_void_p]),
    "fpic_sort": (C.c_int, [C.c_void_p, C.POINTER(fpic_particles), C.c_void_p]),
    "fpic_deposit": (C.c_int, [C.c_void_p, C.POINTER(fpic_particles), _D, _D, _D, _D, C.c_void_p]),
    "fpic_fdtd_step": (C.c_int, [C.c_void_p, C.POINTER(fpic_fields), C.POINTER(fpic_fdtd_params), C.c_int,
                                 C.c_void_p]),
    "fpic_init_metric": (C.c_int, [C.POINTER(C.c_void_p), C.c_double, C.c_double]),
    "fpic_destroy": (None, [C.c_void_p]),
    "fpic_last_error": (C.c_char_p, []),
    "fpic_set_grid": (C.c_int, [C.c_void_p, C.c_int, C.c_int, _D, _D, _D, _D]),
    "fpic_set_theta_mode": (C.c_int, [C.c_void_p, C.c_int]),
    "fpic_init_wald": (C.c_int, [C.c_void_p, C.POINTER(_D), C.c_double, C.c_void_p]),
    "fpic_init_particles": (C.c_int, [C.c_void_p, C.POINTER(fpic_particles), C.c_int, _D, C.c_int,
                                      C.c_double, C.c_void_p]),
    "fpic_push": (C.c_int, [C.c_void_p, C.POINTER(fpic_particles), C.POINTER(_D),
                            C.POINTER(fpic_push_params), C.POINTER(fpic_push_stats), C.c_void_p]),
    "fpic_push_host": (C.c_int, [C.c_void_p, C.POINTER(fpic_particles), C.POINTER(_D),
                                 C.POINTER(fpic_push_params), C.POINTER(fpic_push_stats), C.c_void_p]),
    "fpic_probe_fp64": (C.c_int, [C.POINTER(C.c_double), C.c_int]),
    "fpic_probe_math": (C.c_int, [C.c_int, C.c_void_p, C.c_void_p, C.c_longlong, C.c_void_p]),
    "fpic_set_tuning": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    "fpic_init_split_monopole": (C.c_int, [C.c_void_p, C.POINTER(_D), C.c_double, C.c_double, C.c_void_p]),
    "fpic_bz_power": (C.c_int, [C.c_void_p, C.POINTER(fpic_fields), C.c_int, C.c_void_p, C.c_void_p]),
    "fpic_div_clean": (C.c_int, [C.c_void_p, C.POINTER(_D), C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "fpic_deposit_conserving": (C.c_int, [C.c_void_p, C.POINTER(fpic_particles), C.POINTER(fpic_particles),
                                          C.c_double, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                          C.POINTER(C.c_longlong), C.c_void_p]),
    "fpic_inject_pairs": (C.c_int, [C.c_void_p, C.POINTER(fpic_particles), C.c_longlong, C.c_void_p, C.c_void_p,
                                    C.POINTER(fpic_inject_params), C.c_void_p, C.c_void_p,
                                    C.POINTER(C.c_longlong), C.POINTER(C.c_longlong), C.c_void_p]),
    "fpic_get_tuning": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int)]),
    "fpic_push_noalloc": (C.c_int, [C.c_double, C.c_double, C.POINTER(fpic_particles),
                                    C.POINTER(fpic_push_params), C.POINTER(fpic_push_stats), C.c_void_p]),
    "fpic_hamiltonian": (C.c_int, [C.c_void_p, C.POINTER(fpic_particles), C.c_double, _D, _D, C.c_void_p]),
    "fpic_cell_index": (C.c_int, [C.c_void_p, C.POINTER(fpic_particles), C.c_void_p]),
}


def declared_symbols():
    """Every entry point the binding declares (include/fpic.h)."""
    return sorted(_SIGS)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise FpicError(FPIC_EINVAL, f"libfpic.so not built ({LIB_PATH}); run build()")
            L = C.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _check(rc, allow_notconv=True):
    if rc == FPIC_OK or (allow_notconv and rc == FPIC_ENOTCONVERGED):
        return rc
    raise FpicError(rc, lib().fpic_last_error().decode())


def _dp(t):
    """Device pointer of a tensor as a typed ctypes pointer (None for None)."""
    if t is None:
        return None
    return C.cast(C.c_void_p(t.data_ptr()), _D)


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


@dataclass
class Particles:
    """SoA particle set in device memory (torch tensors)."""
    r: torch.Tensor
    th: torch.Tensor
    ph: torch.Tensor
    ur: torch.Tensor
    uth: torch.Tensor
    uph: torch.Tensor
    qm: torch.Tensor
    w: torch.Tensor
    H0: torch.Tensor
    D0: torch.Tensor
    Hn: torch.Tensor
    alive: torch.Tensor
    scheme: torch.Tensor
    iters: torch.Tensor
    cell: torch.Tensor

    @staticmethod
    def empty(n, device="cuda"):
        f = lambda: torch.zeros(n, dtype=torch.float64, device=device)
        u = lambda: torch.zeros(n, dtype=torch.uint8, device=device)
        return Particles(f(), f(), f(), f(), f(), f(), f(), f(), f(), f(), f(), u(), u(), u(),
                         torch.zeros(n, dtype=torch.int32, device=device))

    @property
    def n(self):
        return self.r.numel()

    def head(self, n):
        """The first n particles (views of the same storage)."""
        return Particles(*[getattr(self, f)[:n] for f in self.__dataclass_fields__])

    def state(self):
        return torch.stack([self.r, self.th, self.ph, self.ur, self.uth, self.uph], dim=1)

    def set_state(self, z):
        for k, name in enumerate(("r", "th", "ph", "ur", "uth", "uph")):
            getattr(self, name).copy_(z[:, k])

    def struct(self):
        # the ctypes struct is rebuilt only when an array was replaced
        arrs = (self.r, self.th, self.ph, self.ur, self.uth, self.uph, self.qm, self.w, self.H0, self.D0, self.Hn,
                self.alive, self.scheme, self.iters, self.cell)
        key = (self.n,) + tuple(t.data_ptr() for t in arrs)
        if getattr(self, "_skey", None) != key:
            self._s = fpic_particles(self.n, *[_dp(t) for t in arrs[:11]],
                                     *[C.cast(C.c_void_p(t.data_ptr()), _U8) for t in arrs[11:14]],
                                     C.cast(C.c_void_p(arrs[14].data_ptr()), _U32))
            self._skey = key
        return self._s


class Ctx:
    """Owns an fpic_ctx handle."""

    def __init__(self, handle):
        self.handle = handle

    def __del__(self):
        h, self.handle = getattr(self, "handle", None), None
        if h and _lib is not None:
            _lib.fpic_destroy(h)


def fpic_init_metric(M: float, a: float) -> Ctx:
    h = C.c_void_p()
    _check(lib().fpic_init_metric(C.byref(h), M, a))
    return Ctx(h)


def fpic_set_grid(ctx: Ctx, grid) -> None:
    """The grid's node tables; a full-theta grid (inputs.full_theta_grid)
    also switches the context to FPIC_THETA_FULL."""
    import numpy as np
    arrs = [np.ascontiguousarray(x, dtype=np.float64) for x in (grid.rn, grid.rh, grid.tn, grid.th)]
    _check(lib().fpic_set_grid(ctx.handle, grid.Nr, grid.Nth, *[a.ctypes.data_as(_D) for a in arrs]))
    ctx.cells = grid.Nr * grid.Nth
    ctx.cells_size = (grid.Nr + 1) * (grid.Nth + 1)
    if getattr(grid, "full_theta", False):
        fpic_set_theta_mode(ctx, FPIC_THETA_FULL)


def fpic_set_theta_mode(ctx: Ctx, mode: int) -> None:
    _check(lib().fpic_set_theta_mode(ctx.handle, int(mode)))


_FIELDS_CACHE = {}


def _fields_arg(fields):
    if fields is None:
        return None
    assert len(fields) == 6
    for f in fields:
        assert f.dtype == torch.float64 and f.is_cuda and f.is_contiguous()
    key = tuple(f.data_ptr() for f in fields)
    arg = _FIELDS_CACHE.get(key)
    if arg is None:
        if len(_FIELDS_CACHE) > 64:
            _FIELDS_CACHE.clear()
        arg = _FIELDS_CACHE[key] = (_D * 6)(*[_dp(f) for f in fields])
    return arg


def fpic_init_wald(ctx: Ctx, fields, B0: float, stream=None) -> None:
    _check(lib().fpic_init_wald(ctx.handle, _fields_arg(fields), B0, _stream(stream)))


def fpic_init_particles(ctx: Ctx, p: Particles, kind: int, draws: torch.Tensor, K: int = 1,
                        B0pot: float = 0.0, stream=None) -> None:
    s = p.struct()
    _check(lib().fpic_init_particles(ctx.handle, C.byref(s), kind, _dp(draws.contiguous()), K, B0pot,
                                     _stream(stream)))


def push_params(dt, scheme=FPIC_RK4, implicit=FPIC_IMR, thr=1e-12, tol=1e-14, max_iter=50,
                r_max=1e300, dg_eps=1e-10, B0pot=0.0, guess=None, events=None, dt_implicit=0.0, t=None,
                B0field=0.0, imr_newton=False, imr_substeps=0, substep_tol=0.0):
    """events: optional list of 4 torch.cuda.Event(enable_timing=True);
    dt_implicit: step of the hybrid's implicit partner (0 = dt); t: optional
    per-particle time tensor (float64, device) advanced by each step;
    B0field: analytic Wald field (fields must be None); imr_newton: solve
    the IMR by the Newton iteration instead of the fixed-point update;
    imr_substeps, substep_tol: unconverged IMR solves redone in up to
    2^imr_substeps substeps (see fpic.h)."""
    prm = fpic_push_params(dt, scheme, implicit, thr, tol, max_iter, r_max, dg_eps, B0pot,
                           None if guess is None else guess.data_ptr(), None, dt_implicit,
                           None if t is None else t.data_ptr(), B0field, int(bool(imr_newton)),
                           int(imr_substeps), float(substep_tol))
    if events is not None:
        arr = (C.c_void_p * 4)(*[C.c_void_p(e.cuda_event) for e in events])
        prm._events_keepalive = arr
        prm.events = C.cast(arr, C.c_void_p)
    return prm


def set_push_before(prm: fpic_push_params, before) -> None:
    """Point prm.before at a Particles set (or None): the push then writes
    each particle's r, th, ur, uth, uph and alive at the start of its step
    into before's arrays (see fpic.h)."""
    if before is None:
        prm.before = None
        prm._before_keepalive = None
    else:
        s = before.struct()
        prm._before_keepalive = (before, s)
        prm.before = C.pointer(s)


def _stats_ptr(stats_out):
    """A page-locked int64 tensor of at least 8 elements as fpic_push_stats*
    (FPIC_TUNE_ASYNC: the library copies the stats there asynchronously)."""
    if stats_out.dtype != torch.int64 or stats_out.numel() < 8 or not stats_out.is_pinned():
        raise ValueError("stats_out must be a pinned int64 tensor of >= 8 elements")
    return C.cast(C.c_void_p(stats_out.data_ptr()), C.POINTER(fpic_push_stats))


def stats_dict(stats_out) -> dict:
    """The fpic_push_stats fields of an int64 tensor filled through stats_out."""
    v = stats_out.tolist()
    return {k: int(v[i]) for i, (k, _) in enumerate(fpic_push_stats._fields_)}


def fpic_push(ctx: Ctx, p: Particles, fields, prm: fpic_push_params, stats: bool = False, stream=None,
              stats_out=None):
    """One push of every alive particle; returns the stats dict if asked.
    stats_out (a pinned int64 tensor) receives the stats instead, without
    synchronising when the context has FPIC_TUNE_ASYNC set."""
    s = p.struct()
    st = fpic_push_stats() if stats and stats_out is None else None
    sp = _stats_ptr(stats_out) if stats_out is not None else (C.byref(st) if st is not None else None)
    rc = lib().fpic_push(ctx.handle, C.byref(s), _fields_arg(fields), C.byref(prm), sp, _stream(stream))
    _check(rc)
    return st.as_dict() if st is not None else None


def fpic_hamiltonian(ctx: Ctx, p: Particles, B0pot: float = 0.0, stream=None):
    H = torch.empty(p.n, dtype=torch.float64, device=p.r.device)
    L = torch.empty_like(H)
    s = p.struct()
    _check(lib().fpic_hamiltonian(ctx.handle, C.byref(s), B0pot, _dp(H), _dp(L), _stream(stream)))
    return H, L


def fpic_cell_index(ctx: Ctx, p: Particles, stream=None) -> torch.Tensor:
    s = p.struct()
    _check(lib().fpic_cell_index(ctx.handle, C.byref(s), _stream(stream)))
    return p.cell


class HostParticles:
    """Particle set in pinned host memory (numpy views of pinned tensors)."""

    FIELDS_D = ("r", "th", "ph", "ur", "uth", "uph", "qm", "w", "H0", "D0", "Hn")
    FIELDS_B = ("alive", "scheme", "iters")

    def __init__(self, n):
        self.n = n
        for f in self.FIELDS_D:
            setattr(self, f, torch.zeros(n, dtype=torch.float64).pin_memory())
        for f in self.FIELDS_B:
            setattr(self, f, torch.zeros(n, dtype=torch.uint8).pin_memory())
        self.cell = torch.zeros(n, dtype=torch.int32).pin_memory()

    def struct(self):
        # the ctypes struct is rebuilt only when an array was replaced
        arrs = [getattr(self, f) for f in self.FIELDS_D + self.FIELDS_B] + [self.cell]
        key = (self.n,) + tuple(t.data_ptr() for t in arrs)
        if getattr(self, "_skey", None) != key:
            hp = lambda t, ty: C.cast(C.c_void_p(t.data_ptr()), ty)
            self._s = fpic_particles(self.n, *[hp(t, _D) for t in arrs[:11]],
                                     *[hp(t, _U8) for t in arrs[11:14]], hp(arrs[14], _U32))
            self._skey = key
        return self._s

    def bytes_in(self):
        # every double array but w (not read by the push), plus alive
        return self.n * (8 * (len(self.FIELDS_D) - 1) + 1)

    def bytes_out(self):
        return self.n * (8 * 7 + 3 + 4)


def fpic_push_host(ctx: Ctx, hp: HostParticles, fields, prm: fpic_push_params, stats: bool = False,
                   stream=None, stats_out=None):
    """fpic_push on host arrays; stats_out as in fpic_push (with
    FPIC_TUNE_ASYNC the call on pinned arrays only enqueues the push)."""
    s = hp.struct()
    st = fpic_push_stats() if stats and stats_out is None else None
    sp = _stats_ptr(stats_out) if stats_out is not None else (C.byref(st) if st is not None else None)
    rc = lib().fpic_push_host(ctx.handle, C.byref(s), _fields_arg(fields), C.byref(prm), sp, _stream(stream))
    _check(rc)
    return st.as_dict() if st is not None else None


def fpic_init_split_monopole(ctx: Ctx, fields, B0: float, zeta0: float = 1e3, stream=None) -> None:
    _check(lib().fpic_init_split_monopole(ctx.handle, _fields_arg(fields), B0, zeta0, _stream(stream)))


def fpic_bz_power(ctx: Ctx, f: "Fields", i: int, stream=None) -> torch.Tensor:
    """Eq. (Pbz) through the sphere r = rh[i]; a one-element device tensor."""
    out = torch.empty(1, dtype=torch.float64, device=f.E[0].device)
    s = f.struct()
    _check(lib().fpic_bz_power(ctx.handle, C.byref(s), i, out.data_ptr(), _stream(stream)))
    return out


def fpic_inject_pairs(ctx: Ctx, store: "Particles", n: int, Br: torch.Tensor, Bth: torch.Tensor,
                      prm: fpic_inject_params, draws: torch.Tensor, want_flags: bool = False, stream=None):
    """Sec. 3.3 / 3.4 pair injection into a capacity-sized particle store whose
    first n entries are in use.  Returns (n_new, pairs wanted, flags or None);
    store.head(n_new) is the particle set afterwards."""
    st = fpic_particles.from_buffer_copy(store.struct())
    st.n = int(n)
    flags = torch.zeros(ctx.cells, dtype=torch.uint8, device=Br.device) if want_flags else None
    wanted, n_new = C.c_longlong(0), C.c_longlong(0)
    _check(lib().fpic_inject_pairs(ctx.handle, C.byref(st), store.n, Br.data_ptr(), Bth.data_ptr(), C.byref(prm),
                                   draws.data_ptr(), flags.data_ptr() if flags is not None else None,
                                   C.byref(wanted), C.byref(n_new), _stream(stream)))
    return int(n_new.value), int(wanted.value), flags


def fpic_div_clean(ctx: Ctx, D, rho: torch.Tensor, n_iter: int = 500, want_phi: bool = False, stream=None):
    """Sec. 2.4 divergence cleaning of D (3 device tensors, corrected in place)."""
    arr = (_D * 3)(*[_dp(d) for d in D])
    phi = torch.zeros_like(rho) if want_phi else None
    _check(lib().fpic_div_clean(ctx.handle, arr, rho.data_ptr(), n_iter,
                                phi.data_ptr() if phi is not None else None, _stream(stream)))
    return phi


def fpic_set_tuning(ctx: Ctx, key: int, value: int) -> None:
    _check(lib().fpic_set_tuning(ctx.handle, key, value))


def fpic_get_tuning(ctx: Ctx, key: int) -> int:
    v = C.c_int()
    _check(lib().fpic_get_tuning(ctx.handle, key, C.byref(v)))
    return v.value


def fpic_probe_math(fn: int, x: torch.Tensor) -> torch.Tensor:
    """The library's elementary routine `fn` (0 reciprocal, 1 square root,
    2 small-step sin / cos - 1, 3 paired-FP32 square root, 4 paired-FP32
    small-step sin / cos - 1, 5 reciprocal square root, 6 paired-FP32
    reciprocal, 7 the integer compares of non-negative doubles beside the
    FP64 ones on the pairs (x[2i], x[2i+1]): rows of six) applied to the
    device tensor x."""
    x = x.contiguous()
    if fn == 7:
        shape = (x.numel() // 2, 6)
    else:
        shape = (x.numel(), 2) if fn in (2, 4) else (x.numel(),)
    y = torch.empty(shape, dtype=torch.float64, device=x.device)
    _check(lib().fpic_probe_math(fn, x.data_ptr(), y.data_ptr(), x.numel(), _stream(None)))
    return y


def fpic_probe_fp64(reps: int = 2000) -> float:
    out = C.c_double()
    _check(lib().fpic_probe_fp64(C.byref(out), reps))
    return out.value


FPIC_NOALLOC_MAX_PARTICLES = 65536


def fpic_push_noalloc(M: float, a: float, p: Particles, prm: fpic_push_params, stats: bool = False,
                      stream=None):
    """Allocation-free geodesic push (no context; fixed scratch capacity)."""
    s = p.struct()
    st = fpic_push_stats() if stats else None
    rc = lib().fpic_push_noalloc(M, a, C.byref(s), C.byref(prm), C.byref(st) if st is not None else None,
                                 _stream(stream))
    _check(rc)
    return st.as_dict() if st is not None else None


def fpic_sort(ctx: Ctx, p: Particles, stream=None) -> None:
    s = p.struct()
    _check(lib().fpic_sort(ctx.handle, C.byref(s), _stream(stream)))


def fpic_deposit(ctx: Ctx, p: Particles, size: int, out=None, stream=None):
    """Returns (rho, j^r, j^th, j^ph) device arrays of the grid size."""
    if out is None:
        out = tuple(torch.zeros(size, dtype=torch.float64, device=p.r.device) for _ in range(4))
    s = p.struct()
    _check(lib().fpic_deposit(ctx.handle, C.byref(s), *[_dp(t) for t in out], _stream(stream)))
    return out


def fpic_deposit_conserving(ctx: Ctx, before: Particles, after: Particles, dt: float, out=None,
                            want_skipped: bool = False, stream=None):
    """Charge-conserving deposit of the moves before -> after; returns
    (rho, J^r, J^th, J^ph) (and the number of skipped moves if asked)."""
    if out is None:
        out = tuple(torch.zeros(ctx.cells_size, dtype=torch.float64, device=after.r.device) for _ in range(4))
    sk = C.c_longlong(0)
    _check(lib().fpic_deposit_conserving(ctx.handle, C.byref(before.struct()), C.byref(after.struct()), float(dt),
                                         *[_dp(t) for t in out], C.byref(sk) if want_skipped else None,
                                         _stream(stream)))
    return (out, int(sk.value)) if want_skipped else out


class Fields:
    """Leapfrog field storage (device tensors) mirroring fpic_fields."""

    NAMES3 = ("B0", "B1", "D0", "D1", "j0", "j1", "E", "H", "Bh", "Dw")

    # the four source arrays of one level (rho, J^r, J^th, J^ph) are
    # consecutive slices of one buffer, each starting on a 256-byte boundary,
    # so a multi-rank step sums them with a single collective
    SRC_ALIGN = 32

    def __init__(self, size, device="cuda"):
        z = lambda: [torch.zeros(size, dtype=torch.float64, device=device) for _ in range(3)]
        for nm in self.NAMES3:
            if nm not in ("j0", "j1"):
                setattr(self, nm, z())
        slot = -(-size // self.SRC_ALIGN) * self.SRC_ALIGN
        for lvl in (0, 1):
            buf = torch.zeros(4 * slot, dtype=torch.float64, device=device)
            setattr(self, "rho%d" % lvl, buf[:size])
            setattr(self, "j%d" % lvl, [buf[(k + 1) * slot:(k + 1) * slot + size] for k in range(3)])

    def struct(self):
        p3 = lambda arrs: _P3(*[_dp(t) for t in arrs])
        return fpic_fields(p3(self.B0), p3(self.B1), p3(self.D0), p3(self.D1), p3(self.j0), _dp(self.rho0),
                           p3(self.j1), _dp(self.rho1), p3(self.E), p3(self.H), p3(self.Bh), p3(self.Dw))

    def swap(self):
        self.B0, self.B1 = self.B1, self.B0
        self.D0, self.D1 = self.D1, self.D0
        self.j0, self.j1 = self.j1, self.j0
        self.rho0, self.rho1 = self.rho1, self.rho0

    def push_fields(self):
        """D^{n+3/2}, B^{n+3/2}: the fields of the push after stage 1."""
        return [self.D1[0], self.D1[1], self.D1[2], self.Bh[0], self.Bh[1], self.Bh[2]]


def fdtd_params(dt, chi0=0.0, lam=5.0, r_abs=0.0, r_max=1.0, conserving=False):
    return fpic_fdtd_params(dt, chi0, lam, r_abs, r_max, int(bool(conserving)))


def fpic_fdtd_step(ctx: Ctx, f: Fields, prm: fpic_fdtd_params, stage: int, stream=None) -> None:
    s = f.struct()
    _check(lib().fpic_fdtd_step(ctx.handle, C.byref(s), C.byref(prm), stage, _stream(stream)))


def fpic_mma_bf16(A, B, C=None, accumulate=False, stream=None):
    """C (+)= A @ B.T on the tensor cores; A [M,K], B [N,K] bf16 (cuda)."""
    M, K = A.shape
    N = B.shape[0]
    if C is None:
        C = torch.zeros(M, N, dtype=torch.float32, device=A.device)
    err = torch.zeros(1, dtype=torch.int32, device=A.device)
    _check(lib().fpic_mma_bf16(A.data_ptr(), A.stride(0), B.data_ptr(),
                               B.stride(0), C.data_ptr(), C.stride(0), M, N, K, int(accumulate), err.data_ptr(),
                               _stream(stream)))
    return C, err


class MLP:
    """Handle of the learned-guess network (fpic_mlp)."""

    def __init__(self):
        h = C.c_void_p()
        _check(lib().fpic_mlp_create(C.byref(h)))
        self.handle = h

    def __del__(self):
        h, self.handle = getattr(self, "handle", None), None
        if h and _lib is not None:
            _lib.fpic_mlp_destroy(h)

    @staticmethod
    def nparams():
        return int(lib().fpic_mlp_nparams())

    def set_params(self, P, stream=None):
        assert P.dtype == torch.float32 and P.is_cuda and P.numel() == self.nparams()
        _check(lib().fpic_mlp_set_params(self.handle, P.data_ptr(), _stream(stream)))

    def forward(self, X, Y=None, stream=None):
        B = X.shape[0]
        assert X.dtype == torch.float32 and X.shape[1] == 16 and X.is_contiguous()
        if Y is None:
            Y = torch.empty(B, 16, dtype=torch.float32, device=X.device)
        _check(lib().fpic_mlp_forward(self.handle, X.data_ptr(), Y.data_ptr(), B, _stream(stream)))
        return Y

    def grad(self, X, T, S, lossw, stream=None):
        """(loss, grad) of a batch; all tensors float32 cuda."""
        B = X.shape[0]
        g = torch.empty(self.nparams(), dtype=torch.float32, device=X.device)
        lw = (C.c_float * 9)(*[float(v) for v in lossw])
        L = C.c_float()
        _check(lib().fpic_mlp_grad(self.handle, X.data_ptr(), T.data_ptr(), S.data_ptr(), lw, B, g.data_ptr(),
                                   C.byref(L), _stream(stream)))
        return L.value, g

    def train_step(self, P, mom, vel, X, T, S, lossw, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8, want_loss=False,
                   stream=None):
        B = X.shape[0]
        lw = (C.c_float * 9)(*[float(v) for v in lossw])
        L = C.c_float()
        _check(lib().fpic_mlp_train_step(self.handle, P.data_ptr(), mom.data_ptr(), vel.data_ptr(), X.data_ptr(),
                                         T.data_ptr(), S.data_ptr(), lw, B, step, lr, b1, b2, eps,
                                         C.byref(L) if want_loss else None, _stream(stream)))
        return L.value if want_loss else None

    def status(self):
        st = C.c_int()
        rc = lib().fpic_mlp_status(self.handle, C.byref(st))
        if rc != 0:
            raise FpicError(rc, lib().fpic_last_error().decode())
        return st.value


def learned_cfg(feat_mean=None, feat_std=None, inc_scale=None, p_skip=0.5, mode=FPIC_LEARN_SKIP,
                restart_after=0):
    cfg = fpic_learned_cfg()
    for i in range(16):
        cfg.feat_mean[i] = 0.0 if feat_mean is None or i >= len(feat_mean) else float(feat_mean[i])
        cfg.feat_std[i] = 1.0 if feat_std is None or i >= len(feat_std) else float(feat_std[i])
    for i in range(6):
        cfg.inc_scale[i] = 1.0 if inc_scale is None else float(inc_scale[i])
    cfg.p_skip = p_skip
    cfg.mode = mode
    cfg.restart_after = restart_after
    return cfg


def fpic_features(ctx: Ctx, p: Particles, fields, dt, cfg=None, stream=None):
    X = torch.empty(p.n, 16, dtype=torch.float32, device=p.r.device)
    s = p.struct()
    _check(lib().fpic_features(ctx.handle, C.byref(s), _fields_arg(fields), dt,
                               C.byref(cfg) if cfg is not None else None, X.data_ptr(), _stream(stream)))
    return X


def fpic_learn_sample(ctx: Ctx, p: Particles, fields, prm, cfg=None, stream=None):
    """(X, T, S) training samples from the plain method; particles unchanged."""
    X = torch.empty(p.n, 16, dtype=torch.float32, device=p.r.device)
    T = torch.zeros(p.n, 16, dtype=torch.float32, device=p.r.device)
    S = torch.empty(p.n, dtype=torch.float32, device=p.r.device)
    s = p.struct()
    _check(lib().fpic_learn_sample(ctx.handle, C.byref(s), _fields_arg(fields), C.byref(prm),
                                   C.byref(cfg) if cfg is not None else None, X.data_ptr(), T.data_ptr(),
                                   S.data_ptr(), _stream(stream)))
    return X, T, S


def fpic_push_learned(ctx: Ctx, net: "MLP", p: Particles, fields, prm, cfg, stats=False, stream=None):
    s = p.struct()
    st = fpic_push_stats() if stats else None
    rc = lib().fpic_push_learned(ctx.handle, net.handle, C.byref(s), _fields_arg(fields), C.byref(prm),
                                 C.byref(cfg), C.byref(st) if st is not None else None, _stream(stream))
    _check(rc)
    return st.as_dict() if st is not None else None


def fpic_push_batched_learned(runs, net: "MLP", p: Particles, prm, cfg, stats=False, stream=None):
    """fpic_push_batched with the learned corrector (cfg.mode = FPIC_LEARN_CORRECT)."""
    s = p.struct()
    st = fpic_push_stats() if stats else None
    rc = lib().fpic_push_batched_learned(runs, len(runs), net.handle, C.byref(s), C.byref(prm), C.byref(cfg),
                                         C.byref(st) if st is not None else None, _stream(stream))
    _check(rc)
    return st.as_dict() if st is not None else None


def make_runs(specs):
    """specs: list of (ctx, fields or None, begin, end, r_max, B0pot) -> ctypes array."""
    arr = (fpic_run * len(specs))()
    for i, (ctx, fields, b, e, r_max, B0pot) in enumerate(specs):
        arr[i].ctx = ctx.handle
        for k in range(6):
            arr[i].fields[k] = _dp(fields[k]) if fields is not None else None
        arr[i].begin, arr[i].end, arr[i].r_max, arr[i].B0pot = b, e, r_max, B0pot
    return arr


def fpic_push_batched(runs, p: Particles, prm, stats=False, stream=None):
    """runs: result of make_runs (keep the field tensors alive)."""
    s = p.struct()
    st = fpic_push_stats() if stats else None
    rc = lib().fpic_push_batched(runs, len(runs), C.byref(s), C.byref(prm),
                                 C.byref(st) if st is not None else None, _stream(stream))
    _check(rc)
    return st.as_dict() if st is not None else None
