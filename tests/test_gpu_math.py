"""The library's own FP64 elementary routines against correctly rounded
references (numpy's reciprocal and square root are IEEE correctly rounded;
sin / cos - 1 are checked against libm in extended form)."""
import numpy as np
import pytest

from helpers import cuda_or_skip, dev, fpic

pytestmark = pytest.mark.gpu

ULP = 2.0 ** -52


@pytest.fixture(scope="module")
def F():
    cuda_or_skip()
    return fpic()


def _samples(lo, hi, n, seed):
    rng = np.random.default_rng(seed)
    return np.exp(rng.uniform(np.log(lo), np.log(hi), n))


def test_reciprocal_within_two_ulp(F):
    """1/x from the hardware estimate and one third-order step, over 60
    decades of either sign, within two ulp of the correctly rounded value."""
    x = _samples(1e-30, 1e30, 1 << 20, 1)
    x[: 1 << 19] *= -1.0
    got = F.fpic_probe_math(0, dev(x)).cpu().numpy()
    rel = np.abs(got * x - 1.0)
    assert rel.max() <= 2 * ULP, rel.max()


def test_reciprocal_sqrt_within_two_ulp(F):
    """1/sqrt(x) from the hardware estimate and the second-order binomial
    correction (the push's lapse and 1/Gamma), over 60 decades, within two
    ulp of an extended-precision reference (the first omitted term, of order
    e^3, is far below double rounding)."""
    x = _samples(1e-30, 1e30, 1 << 20, 5)
    x[:4] = [1.0, 4.0, 2.0, 1.0 + 2.0 ** -52]    # exact squares and the next double above 1
    got = F.fpic_probe_math(5, dev(x)).cpu().numpy()
    ref = 1.0 / np.sqrt(x.astype(np.longdouble))
    if np.finfo(np.longdouble).nmant < 60:
        pytest.skip("no extended precision on this host")
    rel = np.abs((got.astype(np.longdouble) - ref) / ref).astype(np.float64)
    print("rsqrt max rel err", rel.max(), "= 2^%.1f" % np.log2(rel.max() + 1e-300))
    assert rel.max() <= 2 * ULP, rel.max()


def test_deposit_sqrt_error_bound(F):
    """One Goldschmidt step on the hardware estimate: relative error far
    below the deposit's 1e-10 tolerance (bound 2^-38; 2^-39.6 measured) over the radicands of
    sqrt(gamma) on a grid r in [1, 1e4] (x ~ r^4)."""
    x = _samples(0.5, 1e17, 1 << 20, 2)
    got = F.fpic_probe_math(1, dev(x)).cpu().numpy()
    ref = np.sqrt(x)
    rel = np.abs(got - ref) / ref
    print("sqrt_dep max rel err", rel.max(), "= 2^%.1f" % np.log2(rel.max() + 1e-300))
    assert rel.max() <= 2.0 ** -38, rel.max()


def test_paired_sqrt_error_bound(F):
    """The deposit's paired-FP32 square root (the FP32 estimate, one Newton
    step for the root with the exact square error): relative error below
    2^-43 over the same radicands (3 e^2 / 2 of the estimate's 2-ulp error
    e, at most about 2^-43.4, plus roundings; 2^-44.5 measured), an order of
    magnitude inside the FP64 form's 2^-39.6."""
    x = _samples(0.5, 1e17, 1 << 20, 4)
    got = F.fpic_probe_math(3, dev(x)).cpu().numpy()
    ref = np.sqrt(x)
    rel = np.abs(got - ref) / ref
    print("paired sqrt max rel err", rel.max(), "= 2^%.1f" % np.log2(rel.max() + 1e-300))
    assert rel.max() <= 2.0 ** -43, rel.max()


def test_paired_reciprocal_error_bound(F):
    """The deposit's paired-FP32 1/x (FP32 estimate, the exact product
    errors, a second-order series) over 30 decades (where the input's and
    the result's low floats are normal: the deposit's subvolume sums):
    relative error below 2^-44 against an extended-precision reference
    (about 2^-46 expected)."""
    x = _samples(1e-15, 1e15, 1 << 20, 6)
    if np.finfo(np.longdouble).nmant < 60:
        pytest.skip("no extended precision on this host")
    ref = 1.0 / x.astype(np.longdouble)
    got = F.fpic_probe_math(6, dev(x)).cpu().numpy().astype(np.longdouble)
    rel = np.abs((got - ref) / ref).astype(np.float64)
    print("paired rcp max rel err", rel.max(), "= 2^%.1f" % np.log2(rel.max() + 1e-300))
    assert rel.max() <= 2.0 ** -44, rel.max()


def test_integer_compares_of_nonnegative_doubles(F):
    """The IMR stopping tests' integer compares of bit patterns (le_nonneg,
    lt_nonneg, fmax_nonneg) give exactly the FP64 results on non-negative
    doubles, zeros, subnormals, infinity and NaN on either side (a NaN
    compares false; the running maximum ignores a NaN), against the GPU's
    own FP64 compares and numpy's."""
    rng = np.random.default_rng(8)
    special = np.array([0.0, 5e-324, 1e-310, 2.2250738585072014e-308, 1e-300, 1e-16, 1.0,
                        1.0 + 2.0 ** -52, 1e300, np.inf, np.nan])
    a = np.concatenate([np.repeat(special, special.size), np.abs(rng.normal(size=4096)) * 10.0 ** rng.integers(-20, 20, 4096)])
    b = np.concatenate([np.tile(special, special.size), np.abs(rng.normal(size=4096)) * 10.0 ** rng.integers(-20, 20, 4096)])
    b[-2048:] = a[-2048:] * (1.0 + (rng.integers(0, 3, 2048) - 1) * 2.0 ** -52)   # neighbours and ties
    x = np.empty(2 * a.size); x[0::2] = a; x[1::2] = b
    got = F.fpic_probe_math(7, dev(x)).cpu().numpy()
    with np.errstate(invalid="ignore"):
        le, lt, mx = (a <= b).astype(float), (a < b).astype(float), np.fmax(a, b)
    assert np.array_equal(got[:, 0], got[:, 1]) and np.array_equal(got[:, 0], le)
    assert np.array_equal(got[:, 2], got[:, 3]) and np.array_equal(got[:, 2], lt)
    ok_a = ~np.isnan(a)     # the running maximum a is never a NaN
    assert np.array_equal(got[ok_a, 4].view(np.int64), got[ok_a, 5].view(np.int64))
    assert np.array_equal(got[ok_a, 4], mx[ok_a])


def test_paired_small_step_sin_cos(F):
    """The deposit's paired-FP32 sin h, cos h - 1 of a lattice step: the
    series branch (|h| < 2^-7) to 2^-45 of sin h and 2^-54 absolute on
    cos h - 1 (2^-38 of itself), the FP64 branch above within the same
    relative bounds (the split into two floats); against sin h and
    -2 sin^2(h/2)."""
    rng = np.random.default_rng(5)
    h = np.concatenate([rng.uniform(0.0, 0.0078, 1 << 18), rng.uniform(0.0, 1e-4, 1 << 14),
                        [0.0, 1e-12, 0.0078124], rng.uniform(0.0079, 0.3, 1 << 12)])
    got = F.fpic_probe_math(4, dev(h)).cpu().numpy()
    s_ref = np.sin(h)
    cm_ref = -2.0 * np.sin(0.5 * h) ** 2
    es = np.abs(got[:, 0] - s_ref) / np.maximum(s_ref, 1e-300)
    ec = np.abs(got[:, 1] - cm_ref)
    print("paired sin rel %.3e, cos-1 abs %.3e, cos-1 rel %.3e" % (es.max(), ec.max(),
          (ec / np.maximum(np.abs(cm_ref), 1e-300)).max()))
    assert es.max() <= 2.0 ** -45
    assert ec[h < 0.0078125].max() <= 2.0 ** -54
    assert np.all(ec <= 2.0 ** -38 * np.abs(cm_ref) + 1e-300)


def test_small_step_sin_cos(F):
    """Series branches (|h| < 2^-10: through h^5 / h^6; |h| < 2^-7: through
    h^7 / h^8): sin h and cos h - 1 to a few ulp of their own magnitude,
    against cos h - 1 = -2 sin^2(h/2); libm branch (larger steps): to a few
    ulp of 1."""
    rng = np.random.default_rng(3)
    hs = np.concatenate([rng.uniform(-0.0078, 0.0078, 1 << 18), rng.uniform(-0.00098, 0.00098, 1 << 18),
                         [0.0, 1e-300, -1e-9, 0.0009765, -0.0009766]])
    hl = rng.uniform(-0.5, 0.5, 1 << 12)
    hl = hl[np.abs(hl) >= 0.0078125]
    for h, series in ((hs, True), (hl, False)):
        got = F.fpic_probe_math(2, dev(h)).cpu().numpy()
        s_ref = np.sin(h)
        cm_ref = -2.0 * np.sin(0.5 * h) ** 2
        if series:
            assert np.all(np.abs(got[:, 0] - s_ref) <= 8 * ULP * np.abs(s_ref))
            assert np.all(np.abs(got[:, 1] - cm_ref) <= 8 * ULP * np.abs(cm_ref))
        else:
            assert np.abs(got[:, 0] - s_ref).max() <= 4 * ULP
            assert np.abs(got[:, 1] - cm_ref).max() <= 4 * ULP
