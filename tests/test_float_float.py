"""The float-float accumulation of the global statistics (per thread an
unevaluated sum hi + lo of FP32 values kept by Knuth's error-free two-sum and
a renormalisation), emulated in numpy FP32 and checked against exact
rational sums: about 44 significant bits, against 24 for a plain FP32 sum of
the same values.  The variance pass's difference (x - m, m = mh + ml) and
square (with an FMA for the exact error of q*q) are checked the same way."""
from fractions import Fraction

import numpy as np

f32 = np.float32


def two_sum(a, b):
    s = f32(a + b)
    bb = f32(s - a)
    e = f32(f32(a - f32(s - bb)) + f32(b - bb))
    return s, e


def ff_add(hi, lo, v, ve):
    s, e = two_sum(hi, v)
    e = f32(e + f32(lo + ve))
    nhi = f32(s + e)
    nlo = f32(e - f32(nhi - s))
    return nhi, nlo


def fma32(a, b, c):
    """FP32 fma: the exact a*b + c rounded once (exact in float64 for FP32 inputs
    up to a final double rounding, far below the tolerances here)."""
    return f32(float(Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c))))


def test_float_float_sum_keeps_about_44_bits():
    rng = np.random.default_rng(0)
    for scale, shift in ((1.0, 0.0), (3.0, 1e3), (1e-3, 5.0)):
        x = (rng.normal(shift, scale, 3000)).astype(np.float32)
        hi, lo = f32(0), f32(0)
        plain = f32(0)
        for v in x:
            hi, lo = ff_add(hi, lo, v, f32(0))
            plain = f32(plain + v)
        exact = sum(Fraction(float(v)) for v in x)
        ff = Fraction(float(hi)) + Fraction(float(lo))
        mag = sum(abs(Fraction(float(v))) for v in x)
        assert abs(ff - exact) <= mag * Fraction(1, 2 ** 42)
        # the plain FP32 sum is much worse (the test would catch dropping lo)
        assert abs(Fraction(float(plain)) - exact) > 100 * abs(ff - exact)


def test_float_float_squared_differences():
    rng = np.random.default_rng(1)
    x = rng.normal(1e3, 2.0, 2000).astype(np.float32)
    m = float(np.mean(x.astype(np.float64)))
    mh = f32(m)
    ml = f32(m - float(mh))
    hi, lo = f32(0), f32(0)
    for v in x:
        q, qe = two_sum(v, f32(-mh))
        qe = f32(qe - ml)
        p = f32(q * q)
        pe = fma32(q, q, -p)
        pe = fma32(f32(q + q), qe, pe)
        hi, lo = ff_add(hi, lo, p, pe)
    mq = Fraction(m)
    exact = sum((Fraction(float(v)) - mq) ** 2 for v in x)
    got = Fraction(float(hi)) + Fraction(float(lo))
    assert abs(got - exact) <= exact * Fraction(1, 2 ** 36)
