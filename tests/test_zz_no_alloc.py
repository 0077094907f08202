"""The allocation-free push (fpic_push_noalloc) against the regular
fpic_push, through the C ABI, on two calls in a row.

fpic_push_noalloc serves callers that may not allocate device memory (their
device memory is owned by a host framework or allocator, or allocation is
forbidden in their loop); it keeps its scratch in a fixed file-scope device
array instead of the context.  Cases: neutral geodesics, charged particles
in the analytic Wald field, and a set of exactly the capacity.  This file is
collected last on purpose."""
import numpy as np
import pytest

import oracle as O
from paper_2602_07452_gb300 import inputs as I
from helpers import cuda_or_skip, fpic, make_particles, to_np

pytestmark = pytest.mark.gpu
TOL = 1e-12


def _pair(n, a, seed):
    cand = I.orbit_candidates(n, seed=seed)
    z, bad = O.seed_orbits(1.0, a, cand)
    assert bad == 0
    q = np.zeros(n)
    H0 = O.hamiltonian(1.0, a, 0.0, z, q)[0]
    mk = lambda: make_particles(z, q, H0, H0, H0.copy())
    return mk(), mk()


@pytest.mark.parametrize("scheme,implicit,newton", [("HYB2", "IMR", False), ("HYB2", "IMR", True),
                                                   ("HYB1", "HAM", False), ("RK4", "IMR", False)])
def test_noalloc_matches_regular_push_two_calls(scheme, implicit, newton):
    cuda_or_skip()
    F = fpic()
    a, dt, n = 0.9, 0.5, 3001
    p_ref, p_na = _pair(n, a, seed=21)
    ctx = F.fpic_init_metric(1.0, a)
    thr = 1e-10 if scheme == "HYB2" else 1e-11
    prm = F.push_params(dt, scheme=getattr(F, "FPIC_" + scheme), implicit=getattr(F, "FPIC_" + implicit),
                        thr=thr, tol=1e-14, imr_newton=newton)
    for _ in range(2):                     # two calls in a row
        st_ref = F.fpic_push(ctx, p_ref, None, prm, stats=True)
        st_na = F.fpic_push_noalloc(1.0, a, p_na, prm, stats=True)
        zr, Hr, ar, sr, ir, _ = to_np(p_ref)
        zn, Hn, an, sn, iN, _ = to_np(p_na)
        err = (np.abs(zn - zr) / (np.abs(zr) + 1.0)).max()
        assert err <= TOL, err
        assert np.abs(Hn - Hr).max() <= TOL * np.abs(Hr).max()
        assert np.array_equal(an, ar) and np.array_equal(sn, sr) and np.array_equal(iN, ir)
        assert st_na == st_ref
    if scheme != "RK4":
        assert 0 < st_ref["n_implicit"] < n


def test_noalloc_rejects_more_than_capacity():
    cuda_or_skip()
    F = fpic()
    n = F.FPIC_NOALLOC_MAX_PARTICLES + 1
    p = make_particles(np.tile([[8.0, 1.0, 0.0, 0.0, 0.0, 3.0]], (n, 1)), np.zeros(n))
    with pytest.raises(F.FpicError, match="capacity"):
        F.fpic_push_noalloc(1.0, 0.9, p, F.push_params(0.1))


def _charged_pair(n, a, B0, seed):
    rng = np.random.default_rng(seed)
    z = np.stack([rng.uniform(4, 9, n), rng.uniform(0.7, 2.4, n), rng.uniform(0, 6, n),
                  rng.normal(size=n) * 0.3, rng.normal(size=n) * 0.5, rng.normal(size=n) * 2], 1)
    q = np.choose(np.arange(n) % 3, [np.full(n, -100.0), np.full(n, 100.0), np.zeros(n)])
    H0, _, D0 = O.hamiltonian(1.0, a, B0, z, q)
    mk = lambda: make_particles(z, q, H0, D0, H0.copy())
    return z, q, H0, D0, mk(), mk()


@pytest.mark.parametrize("scheme,implicit,newton", [("HYB2", "IMR", True), ("HYB1", "HAM", False)])
def test_noalloc_charged_wald_matches_regular_push_two_calls(scheme, implicit, newton):
    """Charged particles (q/m = -100, +100, 0) in the analytic Wald field
    (B0field = B0pot = 1, M = 1, no grid), dt = 1e-3: the allocation-free
    push equals fpic_push on two calls in a row, with the IMR (Newton form)
    or the charged discrete-gradient partner taking the rejected trials."""
    cuda_or_skip()
    F = fpic()
    a, B0, dt, n = 0.9, 1.0, 1e-3, 3001
    z, q, H0, D0, p_ref, p_na = _charged_pair(n, a, B0, seed=27)
    pr = O.push_params(a=a, dt=dt, scheme=O.RK4, field_kind=O.FIELD_WALD, B0field=B0, B0pot=B0)
    zr = np.ascontiguousarray(z.copy()); Hr = H0.copy()
    O.push(pr, zr, q, H0, D0, Hr, np.ones(n, np.uint8))
    Ht = np.abs(Hr - H0) / D0
    thr = float(np.median(Ht) if scheme == "HYB2" else np.median(Ht) / dt)
    ctx = F.fpic_init_metric(1.0, a)
    prm = F.push_params(dt, scheme=getattr(F, "FPIC_" + scheme), implicit=getattr(F, "FPIC_" + implicit),
                        thr=thr, tol=1e-14, max_iter=100, B0pot=B0, B0field=B0, imr_newton=newton)
    for _ in range(2):
        st_ref = F.fpic_push(ctx, p_ref, None, prm, stats=True)
        st_na = F.fpic_push_noalloc(1.0, a, p_na, prm, stats=True)
        zr, Hr, ar, sr, ir, _ = to_np(p_ref)
        zn, Hn, an, sn, iN, _ = to_np(p_na)
        err = (np.abs(zn - zr) / (np.abs(zr) + 1.0)).max()
        assert err <= TOL, err
        assert np.abs(Hn - Hr).max() <= TOL * np.abs(Hr).max()
        assert np.array_equal(an, ar) and np.array_equal(sn, sr) and np.array_equal(iN, ir)
        assert st_na == st_ref
    assert 0 < st_ref["n_implicit"] < n


def test_noalloc_at_exactly_the_capacity():
    """n = FPIC_NOALLOC_MAX_PARTICLES, the largest set the fixed array holds:
    a Hyb2 RK4 <-> IMR step equals fpic_push's."""
    cuda_or_skip()
    F = fpic()
    a, n = 0.9, F.FPIC_NOALLOC_MAX_PARTICLES
    p_ref, p_na = _pair(n, a, seed=29)
    ctx = F.fpic_init_metric(1.0, a)
    prm = F.push_params(0.5, scheme=F.FPIC_HYB2, implicit=F.FPIC_IMR, thr=1e-10, tol=1e-14)
    st_ref = F.fpic_push(ctx, p_ref, None, prm, stats=True)
    st_na = F.fpic_push_noalloc(1.0, a, p_na, prm, stats=True)
    zr, Hr, ar, sr, ir, _ = to_np(p_ref)
    zn, Hn, an, sn, iN, _ = to_np(p_na)
    assert (np.abs(zn - zr) / (np.abs(zr) + 1.0)).max() <= TOL
    assert np.array_equal(an, ar) and np.array_equal(sn, sr) and np.array_equal(iN, ir)
    assert st_na == st_ref and 0 < st_ref["n_implicit"] < n
