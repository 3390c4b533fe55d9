"""The arithmetic behind the digit-slice FP64 form, checked with exact integers on
the CPU (no GPU, no library code): the representation of a column in 7 balanced
base-256 digits, the error of a product that keeps the digit pairs t + u <= 8,
and the exactness of the FP32 level sums over 128-row blocks.  These are the
facts the GPU tolerances of tests/test_gpu_ozaki.py rest on.

For |x| < 2^E:  A = floor(|x| 2^(55 - E)) < 2^55,  A = sum_{t=1..7} d_t 256^(7-t)
with d_1 in [0, 128] and d_2..d_7 in [-128, 127], so
x = sign(x) 2^(E+1) sum_t d_t 2^(-8t) up to the truncation |x| - A 2^(E-55) < 2^(E-55).
"""
import math
import random
from fractions import Fraction

import pytest


def exact(x: float) -> Fraction:
    return Fraction(x)


def fixed_point(x: float, E: int) -> int:
    """A = floor(|x| 2^(55 - E)), exactly."""
    v = abs(exact(x)) * (Fraction(2) ** (55 - E))
    return v.numerator // v.denominator


def balanced_digits(A: int):
    """7 balanced base-256 digits of A < 2^55 (top digit absorbs the carries)."""
    d = []
    rest = A
    for _ in range(6):
        low = rest % 256
        if low >= 128:
            low -= 256
        d.append(low)
        rest = (rest - low) // 256
    d.append(rest)
    return d[::-1]  # d_1 .. d_7


def column_exponent(xs) -> int:
    """Smallest E with max |x| < 2^E (frexp: |x| = f 2^e, 0.5 <= f < 1, so |x| < 2^e)."""
    m = max(abs(x) for x in xs)
    return math.frexp(m)[1] if m > 0 else -1022


def random_double(rng, lo=-60, hi=60):
    return math.ldexp(rng.uniform(-1.0, 1.0), rng.randint(lo, hi))


@pytest.mark.parametrize("seed", range(5))
def test_digits_reconstruct_and_ranges(seed):
    rng = random.Random(seed)
    for _ in range(2000):
        x = random_double(rng)
        E = math.frexp(x)[1] + rng.randint(0, 4) if x != 0 else 0
        A = fixed_point(x, E)
        assert 0 <= A < 2 ** 55
        d = balanced_digits(A)
        assert sum(dt * 256 ** (6 - t) for t, dt in enumerate(d)) == A
        assert 0 <= d[0] <= 128 and all(-128 <= dt <= 127 for dt in d[1:])
        # x = sign 2^(E+1) sum d_t 2^(-8t) up to the truncation below 2^(E-55)
        rep = Fraction(2) ** (E + 1) * sum(Fraction(dt, 256 ** (t + 1)) for t, dt in enumerate(d))
        err = abs(exact(x)) - rep
        assert 0 <= err < Fraction(2) ** (E - 55)


def kept_product(di, dj, Ei, Ej) -> Fraction:
    """2^(Ei+Ej+2) sum_{t+u<=8} d_t d_u 2^(-8(t+u)) (digits of |x_i|, |x_j|)."""
    s = Fraction(0)
    for t in range(1, 8):
        for u in range(1, 8):
            if t + u <= 8:
                s += Fraction(di[t - 1] * dj[u - 1], 256 ** (t + u))
    return Fraction(2) ** (Ei + Ej + 2) * s


@pytest.mark.parametrize("seed", range(5))
def test_product_error_within_bound(seed):
    """|x_i x_j - sign kept_product| < 1.26 * 2^(Ei + Ej - 53) per row."""
    rng = random.Random(100 + seed)
    worst = 0.0
    for _ in range(1500):
        xi, xj = random_double(rng, -20, 20), random_double(rng, -20, 20)
        Ei = math.frexp(xi)[1] + rng.randint(0, 2)
        Ej = math.frexp(xj)[1] + rng.randint(0, 2)
        di, dj = balanced_digits(fixed_point(xi, Ei)), balanced_digits(fixed_point(xj, Ej))
        sgn = (1 if xi >= 0 else -1) * (1 if xj >= 0 else -1)
        err = abs(exact(xi) * exact(xj) - sgn * kept_product(di, dj, Ei, Ej))
        ratio = float(err / (Fraction(2) ** (Ei + Ej - 53)))
        worst = max(worst, ratio)
        assert ratio < 1.26
    assert worst > 0.01  # the bound is not vacuous on random data


def test_product_error_worst_case_reaches_the_dropped_level_term():
    """Digits d_2..d_7 = -128 on both sides: the dropped level-9 pairs alone give
    6 * 2^14 * 2^-72 of 2^(Ei+Ej+2) = 6 * 2^(Ei+Ej-56); the total stays below the
    stated 1.26 * 2^(Ei+Ej-53) and above 0.7 of it."""
    d = [128] + [-128] * 6
    A = sum(dt * 256 ** (6 - t) for t, dt in enumerate(d))
    assert balanced_digits(A) == d
    E = 0
    x = float(Fraction(A, 2 ** 55))  # A = 2^7 * (odd part < 2^48): exact in FP64
    assert exact(x) == Fraction(A, 2 ** 55) and fixed_point(x, E) == A
    err = abs(exact(x) * exact(x) - kept_product(d, d, E, E))
    ratio = float(err / Fraction(2) ** (2 * E - 53))
    assert 0.7 < ratio < 1.26, ratio


def test_level_sums_fit_fp32_exactly_over_128_rows():
    """Level s = t + u holds s - 1 pairs (at most 7); over 128 rows a level sum is an
    integer of magnitude <= 7 * 128 * 2^14 = 7 * 2^21 < 2^24, so every partial sum of
    the FP32 tensor-core accumulation is an exactly representable integer."""
    bound = max(s - 1 for s in range(2, 9)) * 128 * (128 * 128)
    assert bound == 7 * 2 ** 21 < 2 ** 24
    # the extreme digits realise products of 2^14 exactly
    assert 128 * 128 == (-128) * (-128) == 2 ** 14


def test_column_exponent_bounds_every_entry():
    rng = random.Random(7)
    for _ in range(200):
        xs = [random_double(rng, -30, 30) for _ in range(16)]
        E = column_exponent(xs)
        assert all(abs(x) < 2.0 ** E for x in xs)
        assert max(abs(x) for x in xs) >= 2.0 ** (E - 1)
