"""The square root and reciprocal of the binary64 kernels (`sqrt_nonneg`,
`recip_pos` in csrc/eig3_f64.cuh) take a binary32 seed and correct it with a
truncated binomial series in binary64.  Emulated here with exactly rounded
binary64 operations (every FMA rounded once, through fractions) for seeds at
the worst relative error the seed instructions allow, the corrected results
must be faithful: within one unit in the last place of the exact value (the
kernels' claim is 0.75 ulp for the square roots, 0.5 ulp for the reciprocal).

  sqrt(c x'), x' in [1, 4), c = 1 or 3:  g = x' (c y0),  h = (1 - g y0)/2,
      s = g + (g h)(1 + 1.5 h)          (y0 ~ (c x')^-1/2, 22 bits for c = 3)
  1/x', x' in [1, 2):  e = 1 - x' c0,  c = c0 + c0 (e + e e)
"""
import math
import random
from fractions import Fraction as Fr

import numpy as np
import pytest


def fma(a, b, c):
    return float(Fr(a) * Fr(b) + Fr(c))


def f32(x):
    return float(np.float32(x))


def trunc24(x):  # the seed's truncating binary64 -> binary32 conversion
    m, e = math.frexp(x)
    return math.ldexp(math.floor(m * 2 ** 24) / 2 ** 24, e)


def trunc22(y):  # mantissa cut to 22 significant bits (c = 3 seeds)
    b = np.float32(y).view(np.int32) & ~3
    return float(np.int32(b).view(np.float32))


def ulp_error(got, exact_sq=None, exact=None):
    if exact_sq is not None:   # |got - sqrt(exact_sq)| in ulps, without taking a square root
        ref = math.sqrt(float(exact_sq))
        return float(abs(Fr(got) ** 2 - exact_sq) / (Fr(got) + Fr(ref)) / Fr(math.ulp(ref)))
    return float(abs(Fr(got) - exact) / Fr(math.ulp(float(exact))))


@pytest.mark.parametrize("c", [1, 3])
def test_sqrt_series_is_faithful(c):
    rng = random.Random(20 + c)
    worst = 0.0
    xs_list = [1.0, 4.0 - 2 ** -50, 2.0, 3.0] + [rng.uniform(1.0, 4.0) for _ in range(4000)]
    for xs in xs_list:
        y = 1.0 / math.sqrt(f32(c * trunc24(xs)))
        for rel in (-2 ** -22, 2 ** -22, rng.uniform(-2 ** -22, 2 ** -22)):
            y0 = f32(y * (1.0 + rel))
            if c == 3:
                y0 = trunc22(y0)
            cy0 = f32(c * y0)
            assert cy0 == c * y0                    # exact in binary32
            g = xs * cy0
            h = fma(-g, f32(0.5 * y0), 0.5)
            s = fma(g * h, fma(1.5, h, 1.0), g)
            worst = max(worst, ulp_error(s, exact_sq=c * Fr(xs)))
    print(f"sqrt({c} x) worst {worst:.3f} ulp")
    assert worst < 0.76


def test_reciprocal_series_is_faithful():
    rng = random.Random(30)
    worst = 0.0
    for xs in [1.0, 2.0 - 2 ** -51, 1.5] + [rng.uniform(1.0, 2.0) for _ in range(4000)]:
        c_exact = 1.0 / f32(trunc24(xs))
        for rel in (-2 ** -22, 2 ** -22, rng.uniform(-2 ** -22, 2 ** -22)):
            c0 = f32(c_exact * (1.0 + rel))
            e = fma(-xs, c0, 1.0)
            cc = fma(c0, fma(e, e, e), c0)
            worst = max(worst, ulp_error(cc, exact=1 / Fr(xs)))
    print(f"1/x worst {worst:.3f} ulp")
    assert worst < 0.51


def test_reciprocal_of_three_x_series_is_faithful():
    """recip3_pos: 1/(3 x') from a seed of 1/(3 x') cut to 22 bits (its
    triple exact in binary32), e = 1 - x' (3 c0), the same series."""
    rng = random.Random(31)
    worst = 0.0
    for xs in [1.0, 2.0 - 2 ** -51, 1.5, 4.0 / 3.0] + [rng.uniform(1.0, 2.0) for _ in range(4000)]:
        c_exact = 1.0 / f32(trunc24(xs))
        for rel in (-2 ** -22, 2 ** -22, rng.uniform(-2 ** -22, 2 ** -22)):
            cf = trunc22(f32(f32(c_exact * (1.0 + rel)) * f32(1.0 / 3.0)))
            c3 = f32(3.0 * cf)
            assert c3 == 3.0 * cf                    # exact in binary32
            e = fma(-xs, c3, 1.0)
            cc = fma(cf, fma(e, e, e), cf)
            worst = max(worst, ulp_error(cc, exact=1 / (3 * Fr(xs))))
    print(f"1/(3x) worst {worst:.3f} ulp")
    assert worst < 0.51


def test_truncating_the_series_earlier_is_not_faithful():
    """The t^2 term of the square root matters: without it the error is far
    above one ulp for seeds at the allowed error (the check can fail)."""
    xs = 2.7
    y0 = f32(1.0 / math.sqrt(f32(trunc24(xs))) * (1.0 + 2 ** -22))
    g = xs * y0
    h = fma(-g, f32(0.5 * y0), 0.5)
    s = fma(g, h, g)                                 # 1 + t/2 only
    assert ulp_error(s, exact_sq=Fr(xs)) > 100
