"""Oracle wrappers of the learned-guess MLP (fpic_oracle_mlp.c).  Test
infrastructure only."""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _D, f64, lib, ptr

N_IN, N_H, N_OUT = 14, 128, 9
_F = C.POINTER(C.c_float)
_I64 = C.c_int64


def _declare(L):
    L.or_mlp_nparams.restype = _I64
    L.or_mlp_forward.argtypes = [_D, _I64, _D, C.c_int, _D, _D, _D]
    L.or_mlp_loss_grad.argtypes = [_D, _I64, _D, _D, _D, _D, C.c_int, _D]
    L.or_mlp_loss_grad.restype = C.c_double
    L.or_mlp_adam.argtypes = [_F, _F, _F, _F, _I64, C.c_int, C.c_float, C.c_float, C.c_float, C.c_float]
    L.or_bf16_round.argtypes = [_I64, _F, _F]


DIMS = (14, 128, 128, 128, 9)


def nparams():
    return int(lib().or_mlp_nparams())


def unpack(P):
    """Split the flat parameter vector into [(W1, b1), ..., (W4, b4)]."""
    out, o = [], 0
    for l in range(4):
        ni, no = DIMS[l], DIMS[l + 1]
        W = P[o:o + ni * no].reshape(no, ni); o += ni * no
        b = P[o:o + no]; o += no
        out.append((W, b))
    return out


def init_params(seed=0):
    rng = np.random.default_rng(seed)
    parts = []
    for l in range(4):
        ni, no = DIMS[l], DIMS[l + 1]
        parts.append(rng.normal(0, np.sqrt(2.0 / ni), (no, ni)).ravel())
        parts.append(rng.normal(0, 0.01, no))
    return np.concatenate(parts)


def forward(P, x, mode=0, keep=False):
    P, x = f64(P), f64(x).reshape(-1, 14)
    B = x.shape[0]
    y = np.empty((B, 9))
    act = np.empty((B, 3, 128)) if keep else None
    pre = np.empty((B, 3, 128)) if keep else None
    lib().or_mlp_forward(ptr(P), B, ptr(x), mode, ptr(y), ptr(act) if keep else None,
                         ptr(pre) if keep else None)
    return (y, act, pre) if keep else y


def loss_grad(P, x, t, s, m, mode=0, grad=True):
    P, x, t, s, m = f64(P), f64(x).reshape(-1, 14), f64(t).reshape(-1, 9), f64(s), f64(m)
    g = np.empty(P.size) if grad else None
    L = lib().or_mlp_loss_grad(ptr(P), x.shape[0], ptr(x), ptr(t), ptr(s), ptr(m), mode,
                               ptr(g) if grad else None)
    return (L, g) if grad else L


def adam(P, mom, vel, g, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """In place on float32 arrays."""
    for a in (P, mom, vel, g):
        assert a.dtype == np.float32 and a.flags.c_contiguous
    lib().or_mlp_adam(P.ctypes.data_as(_F), mom.ctypes.data_as(_F), vel.ctypes.data_as(_F),
                      g.ctypes.data_as(_F), P.size, t, lr, b1, b2, eps)


def bf16_round(x):
    x = np.ascontiguousarray(x, dtype=np.float32)
    out = np.empty_like(x)
    lib().or_bf16_round(x.size, x.ctypes.data_as(_F), out.ctypes.data_as(_F))
    return out
