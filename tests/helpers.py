"""Shared helpers of the GPU parity tests (host-side marshalling only)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2602_07452_gb300 import inputs as I

torch = pytest.importorskip("torch")


def cuda_or_skip():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def fpic():
    from paper_2602_07452_gb300 import fpic as F
    return F


def dev(x, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def make_particles(z, qm, H0=None, D0=None, Hn=None, alive=None, w=None):
    F = fpic()
    n = z.shape[0]
    p = F.Particles.empty(n)
    if n:
        p.set_state(dev(z))
        p.qm.copy_(dev(qm))
        p.w.copy_(dev(np.ones(n) if w is None else w))
        if H0 is not None:
            p.H0.copy_(dev(H0)); p.D0.copy_(dev(D0)); p.Hn.copy_(dev(Hn))
        p.alive.copy_(dev(np.ones(n, np.uint8) if alive is None else alive, torch.uint8))
    return p


def to_np(p):
    return (p.state().cpu().numpy(), p.Hn.cpu().numpy(), p.alive.cpu().numpy(),
            p.scheme.cpu().numpy(), p.iters.cpu().numpy(), p.cell.cpu().numpy().view(np.uint32))


def fields_dev(F):
    return [dev(f) for f in F]


def thermal_state(n, g, a=0.9, theta=0.1, seed=2, qm=100.0, r_lo=None, r_hi=None):
    r_lo = r_lo or 1.02 * I.horizon(1.0, a)
    r_hi = r_hi or g.rn[-1] * 0.98
    d, q, w = I.thermal_draws(n, g, r_lo, r_hi, theta, seed=seed, qm=qm)
    z = O.seed_fido(1.0, a, d)
    return d, z, q


def assert_state_close(zg, zo, tol=1e-12, mask=None):
    err = np.abs(zg - zo) / (np.abs(zo) + 1.0)
    if mask is not None:
        err = err[mask]
    assert err.size == 0 or err.max() <= tol, f"max rel err {err.max():.3e}"
    return err.max() if err.size else 0.0
