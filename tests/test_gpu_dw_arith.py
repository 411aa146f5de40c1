"""Pins of the double-word arithmetic of precision 48 (FP32 pairs), against
exact rational references (fractions.Fraction) of the same split inputs.

Error bounds, u = 2^-24.  Joldes, Muller and Popescu (ACM TOMS 44(2), 2017)
prove 3u^2 for the accurate sum and 5u^2 for the product of normalised
double words (|l| <= ulp(h)/2).  The inputs here come from the kernels'
truncating split, |l| < ulp(h) <= 2u |h|, which doubles the low-order terms
of the product: x_l y_l (4u^2), the rounding of x_h y_l (2u^2), of the fma
adding x_l y_h (4u^2) and of the sum of the corrections (5u^2), 15u^2 in all.
  split            |z - x| <= 2^-47 |x|
  accurate sum     4u^2 |a + b|
  sloppy sum       4u^2 |a + b| for operands of one sign, 4u^2 (|a| + |b|) else
  product          15u^2 |a b| (also before renormalisation)
  1/x, 1/sqrt(x)   2^-45 relative (FP32 approximation + one second-order correction)
  8-term dot2      16u^2 sum |a_j b_j|
"""
import math
from decimal import Decimal, getcontext
from fractions import Fraction

import numpy as np
import pytest

from paper_2102_12933_gb300 import fdu

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

U2 = 2.0 ** -48
N = 4096


def _values(rng, n, positive=False):
    mag = 10.0 ** rng.uniform(-8, 5, n)
    x = mag * rng.uniform(0.5, 2.0, n)
    if not positive:
        x *= rng.choice([-1.0, 1.0], n)
    return x


@pytest.fixture(scope="module")
def data():
    rng = np.random.default_rng(2024)
    x, y = _values(rng, N), _values(rng, N)
    # close pairs: cancellation in sums and differences
    y[: N // 4] = -x[: N // 4] * (1.0 + rng.uniform(-1e-6, 1e-6, N // 4))
    a = fdu.check_dw("split", x)
    b = fdu.check_dw("split", y)
    return x, y, a, b


def _rel(z, exact):
    return abs(Fraction(z) - exact) / abs(exact)


def test_split(data):
    x, y, a, b = data
    assert np.all(np.abs(a - x) <= 2.0 ** -47 * np.abs(x))
    # the split values are what every other op receives
    assert np.array_equal(fdu.check_dw("split", a), a)


@pytest.mark.parametrize("op", ["add", "add_sloppy"])
def test_sums(data, op):
    x, y, a, b = data
    z = fdu.check_dw(op, a, b)
    worst = 0.0
    for zi, ai, bi in zip(z, a, b):
        exact = Fraction(ai) + Fraction(bi)
        err = abs(Fraction(zi) - exact)
        if op == "add" or (ai > 0) == (bi > 0):
            scale = abs(exact)
        else:
            scale = abs(Fraction(ai)) + abs(Fraction(bi))
        if scale == 0:
            assert zi == 0.0
            continue
        worst = max(worst, float(err / scale))
    assert worst <= 4 * U2, worst


@pytest.mark.parametrize("op", ["mul", "mul_unnormalised"])
def test_products(data, op):
    x, y, a, b = data
    z = fdu.check_dw(op, a, b)
    worst = max(float(_rel(zi, Fraction(ai) * Fraction(bi))) for zi, ai, bi in zip(z, a, b))
    assert worst <= 15 * U2, worst


def test_reciprocal_and_rsqrt():
    rng = np.random.default_rng(7)
    x = fdu.check_dw("split", _values(rng, N, positive=True))
    r = fdu.check_dw("recip", x)
    worst = max(float(_rel(ri, 1 / Fraction(xi))) for ri, xi in zip(r, x))
    assert worst <= 2.0 ** -45, worst
    getcontext().prec = 60
    s = fdu.check_dw("rsqrt", x)
    worst = 0.0
    for si, xi in zip(s, x):
        exact = Decimal(1) / Decimal(xi).sqrt()
        worst = max(worst, float(abs(Decimal(si) - exact) / exact))
    assert worst <= 2.0 ** -45, worst


def test_compensated_dot_product(data):
    x, y, a, b = data
    z = fdu.check_dw("dot8", a, b)
    assert z.size == N // 8
    for i, zi in enumerate(z):
        terms = [Fraction(a[8 * i + j]) * Fraction(b[8 * i + j]) for j in range(8)]
        exact = sum(terms)
        bound = 16 * U2 * float(sum(abs(t) for t in terms))
        assert abs(float(Fraction(zi) - exact)) <= bound


def test_bad_arguments():
    with pytest.raises(fdu.FduError):
        fdu.check_dw("dot8", np.ones(12), np.ones(12))  # not a multiple of 8
    assert math.isfinite(fdu.check_dw("split", np.array([1.0]))[0])
