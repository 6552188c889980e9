"""CPU pin of the compensated dot product (Dot2, Ogita, Rump and Oishi 2005) that
the persistent many-problem kernel and the batched path use in place of FP64
products: the device helper's steps are emulated in float32 (a fused
multiply-add is emulated through the exact FP64 product of two floats, which has
at most 48 significant bits) and the result, lanes added in FP64 as on the
device, is compared with the exact rational dot product.  The bound is the
paper's (Ogita et al.): with the final sum in FP64, |res - x'y| <= gamma_m^2 |x|'|y|
plus FP64 rounding, m the length of one lane's chain.  Plain FP32 accumulation
and Dot2 without the product's error term both fail it (the test's power)."""
from fractions import Fraction

import numpy as np
import pytest

F32 = np.float32
U = 2.0 ** -24


def _fma32(a, b, c):
    # a*b exact in FP64 (two 24-bit significands), + c then one rounding to FP32;
    # the FP64 add can round only below 2^-53 relative, far under FP32's step
    return F32(np.float64(a) * np.float64(b) + np.float64(c))


def _dot2_lane(x, hi, lo, drop_product_error=False):
    s, c = F32(0), F32(0)
    for xi, h, l in zip(x, hi, lo):
        p = F32(xi * h)                               # __fmul_rn
        e = _fma32(xi, h, -p)                         # fmaf(x, hi, -p): the exact error of p
        if drop_product_error:
            e = F32(0)
        t = F32(s + p)                                # __fadd_rn
        z = F32(t - s)
        q = F32(F32(s - F32(t - z)) + F32(p - z))     # TwoSum: s + p = t + q exactly
        s = t
        c = _fma32(xi, l, F32(c + F32(q + e)))        # fmaf(x, lo, c + (q + e))
    return np.float64(s) + np.float64(c)


def dot2_device_order(x, y, lanes=32, **kw):
    """The device's order: lane l takes elements l, l + lanes, ...; the lane
    results are added in FP64."""
    hi = y.astype(F32)
    lo = (y - hi.astype(np.float64)).astype(F32)
    return float(sum(_dot2_lane(x[l::lanes], hi[l::lanes], lo[l::lanes], **kw) for l in range(lanes)))


def exact_dot(x, y):
    return sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(x, y))


def _bound(x, y, lanes=32):
    m = -(-len(x) // lanes) + 2
    gam = m * U / (1 - m * U)
    return gam * gam * float(np.abs(x.astype(np.float64)) @ np.abs(y)) + 4 * 2.0 ** -53 * float(
        np.abs(x.astype(np.float64)) @ np.abs(y))


@pytest.mark.parametrize("n,scale", [(100, 1.0), (2000, 1.0), (2048, 1e3), (1999, 1e-4)])
def test_dot2_meets_the_twice_precision_bound(n, scale):
    rng = np.random.default_rng(n)
    x = (rng.standard_normal(n) * scale).astype(F32)
    y = rng.standard_normal(n) + 0.3                  # FP64 residual-like values
    ex = exact_dot(x, y)
    got = dot2_device_order(x, y)
    err = abs(Fraction(got) - ex)
    assert float(err) <= _bound(x, y), (float(err), _bound(x, y))


def test_dot2_on_a_cancelling_sum():
    # x'y near zero against |x|'|y| large: the regime of sum x r - c sum r
    rng = np.random.default_rng(7)
    n = 2000
    x = rng.standard_normal(n).astype(F32)
    y = rng.standard_normal(n)
    y -= float(exact_dot(x, y)) / float(np.float64(x) @ np.float64(x)) * x.astype(np.float64)
    ex = exact_dot(x, y)
    got = dot2_device_order(x, y)
    assert float(abs(Fraction(got) - ex)) <= _bound(x, y)


def test_the_bound_has_power():
    rng = np.random.default_rng(11)
    n = 2000
    x = rng.standard_normal(n).astype(F32)
    y = rng.standard_normal(n)
    ex = exact_dot(x, y)
    b = _bound(x, y)
    # plain FP32 accumulation per lane (FP64 lane sum)
    naive = float(sum(np.float64(np.sum((x[l::32] * y[l::32].astype(F32)).astype(F32), dtype=F32))
                      for l in range(32)))
    assert float(abs(Fraction(naive) - ex)) > 10 * b
    # Dot2 without the products' rounding errors
    broken = dot2_device_order(x, y, drop_product_error=True)
    assert float(abs(Fraction(broken) - ex)) > 10 * b
