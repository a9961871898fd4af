"""Error bounds of the double-word square root and quotient that the FP32 line search uses
(Dekker 1971, sqrt2 / div2), written out step by step in IEEE FP32 as the kernels evaluate
them (numpy float32 operations round to nearest like the device's __f*_rn intrinsics;
TwoProduct's fused multiply-add is the exact FP64 product of two FP32 numbers), against
extended-precision references.  Relative error within 2^-45 over many binades, as long as
the low word stays a normal FP32 number (results above about 2^-100; smaller terms lose their
low word, which changes a sum of such terms by less than 2^-120 of its largest term)."""

import numpy as np
import pytest

f32 = np.float32


def two_sum(a, b):
    s = f32(a + b)
    bb = f32(s - a)
    return s, f32(f32(a - f32(s - bb)) + f32(b - bb))


def fast_two_sum(a, b):
    s = f32(a + b)
    return s, f32(b - f32(s - a))


def two_prod(a, b):
    p = f32(a * b)
    return p, f32(np.float64(a) * np.float64(b) - np.float64(p))   # exact: fma(a, b, -p)


def ff_sqrt(vh, vl):
    s = f32(np.sqrt(vh))
    if s == 0:
        return f32(0), f32(0)
    s2h, s2l = two_prod(s, s)
    e = f32(f32(f32(vh - s2h) - s2l) + vl)
    return fast_two_sum(s, f32(e * f32(f32(0.5) * f32(f32(1) / s))))


def ff_div(ah, al, bh, bl):
    r = f32(f32(1) / bh)
    c = f32(ah * r)
    uh, ul = two_prod(c, bh)
    cc = f32(f32(f32(f32(f32(ah - uh) - ul) + al) - f32(c * bl)) * r)
    return fast_two_sum(c, cc)


def split(x):
    """A float-float pair of a longdouble value."""
    hi = f32(x)
    lo = f32(np.longdouble(x) - np.longdouble(hi))
    return hi, lo


def value(p):
    return np.longdouble(p[0]) + np.longdouble(p[1])


@pytest.mark.skipif(np.finfo(np.longdouble).nmant < 60, reason="needs an extended-precision long double")
def test_sqrt_and_quotient_relative_error():
    rng = np.random.default_rng(7)
    worst_s = worst_d = 0.0
    for _ in range(20000):
        v = np.longdouble(rng.uniform(1, 2)) * np.longdouble(2.0) ** int(rng.integers(-100, 100))
        vh, vl = split(v)
        vv = value((vh, vl))
        s = value(ff_sqrt(vh, vl))
        ref = np.sqrt(vv)
        worst_s = max(worst_s, float(abs(s - ref) / ref))
        a = np.longdouble(rng.uniform(-2, 2)) * np.longdouble(2.0) ** int(rng.integers(-40, 40))
        b = np.longdouble(rng.uniform(1, 2)) * np.longdouble(2.0) ** int(rng.integers(-40, 40)) * (1 if rng.uniform() < 0.5 else -1)
        ap, bp = split(a), split(b)
        q = value(ff_div(ap[0], ap[1], bp[0], bp[1]))
        qref = value(ap) / value(bp)
        if qref != 0:
            worst_d = max(worst_d, float(abs(q - qref) / abs(qref)))
    assert worst_s <= 2.0 ** -45, worst_s
    assert worst_d <= 2.0 ** -45, worst_d


def test_sqrt_of_zero_and_exact_squares():
    assert ff_sqrt(f32(0), f32(0)) == (0, 0)
    for k in range(1, 50):
        s = ff_sqrt(f32(k * k), f32(0))
        assert float(s[0]) + float(s[1]) == k
