"""CPU checks of the emit pass's snap tiers (the kernels' FP32 arithmetic emulated
operation by operation with correctly rounded FP32 results, from exact rationals).

A child's dependent field is rint(y), y = q_f + sum_m q_t,m G64_m -+ H the residual at
the child centre in snap steps (canonization, Sec. 3.2).  The kernels decide it

* in double-float (``snap_df_words``): y as hi + lo from the coefficient's FP32 part
  G and remainder G_lo = fl32(G64 - G), exact products by FMA and Knuth's two-sum; it
  decides only when y is more than 2^-36 M + 2^-20 from a rounding tie, M the
  record's magnitudes.  Checked: every decision equals rint of the exact y and rint
  of an FP64 evaluation, on random records and on records placed 0 to 2^-20 steps
  from a tie.
* in FP32 at a tie, when every coefficient and the shift are FP32-exact multiples of
  2^e and M < 2^(24 + e): then the FMA chain is exact and adding 1.5 * 2^23 rounds
  half to even, as rint does.  Checked on dyadic records with many exact ties.
"""
import math
import random
from fractions import Fraction

import numpy as np
import pytest

MAGIC = Fraction(3 * 2 ** 22)          # 1.5 * 2^23 (32-bit fields)
MAGIC16 = MAGIC + 2 ** 15              # the same biased by 2^15 (16-bit fields)


def f32(x) -> Fraction:
    """x rounded to the nearest FP32 value, ties to even (normal and subnormal range)."""
    x = Fraction(x)
    if x == 0:
        return Fraction(0)
    s = -1 if x < 0 else 1
    a = abs(x)
    e = math.floor(math.log2(a.numerator) - math.log2(a.denominator))
    while Fraction(2) ** e > a:
        e -= 1
    while Fraction(2) ** (e + 1) <= a:
        e += 1
    q = Fraction(2) ** (max(e, -126) - 23)      # the ulp
    n = a / q
    f = math.floor(n)
    r = n - f
    if r > Fraction(1, 2) or (r == Fraction(1, 2) and f % 2 == 1):
        f += 1
    return s * f * q


def fma(a, b, c):
    return f32(Fraction(a) * Fraction(b) + Fraction(c))


def add(a, b):
    return f32(Fraction(a) + Fraction(b))


def sub(a, b):
    return f32(Fraction(a) - Fraction(b))


def mul(a, b):
    return f32(Fraction(a) * Fraction(b))


def rint(x: Fraction) -> int:
    f = math.floor(x)
    r = x - f
    if r > Fraction(1, 2) or (r == Fraction(1, 2) and f % 2 == 1):
        f += 1
    return int(f)


def split_int(q: int):
    hi = f32(q)
    lo = f32(q - int(hi))
    assert hi + lo == q
    return hi, lo


def two_sum(a, b):
    s = add(a, b)
    bb = sub(s, a)
    err = add(sub(a, sub(s, bb)), sub(b, bb))
    assert s + err == Fraction(a) + Fraction(b)        # Knuth: exact
    return s, err


def df_snap(qf, qt, G64, hs64):
    """The kernel's double-float snap: (q, decided)."""
    hi, lo = split_int(qf)
    for q, g in zip(qt, G64):
        th, tl = split_int(q)
        gh = f32(g)
        gl = f32(Fraction(g) - gh)
        p = mul(th, gh)
        e = fma(th, gh, -p)
        assert p + e == th * gh
        hi, err = two_sum(hi, p)
        lo = add(lo, add(err, fma(tl, gl, fma(th, gl, fma(tl, gh, e)))))
    h = f32(hs64)
    hl = f32(Fraction(hs64) - h)
    hi, err = two_sum(hi, h)
    lo = add(lo, add(err, hl))
    r = Fraction(rint(hi))
    w = add(hi - r, lo)                 # hi - r is exact
    assert hi - r == sub(hi, r)
    k = rint(w)
    fr = w - k
    M = abs(qf) + sum(abs(q) * abs(g) for q, g in zip(qt, G64)) + abs(hs64)
    bd = Fraction(2) ** -36 * Fraction(M) + Fraction(2) ** -20
    return int(r) + k, Fraction(1, 2) - abs(fr) > bd


def y_exact(qf, qt, G64, hs64) -> Fraction:
    return Fraction(qf) + sum(Fraction(q) * Fraction(g) for q, g in zip(qt, G64)) + Fraction(hs64)


def y_fp64(qf, qt, G64, hs64) -> float:
    v = float(qf)
    for q, g in zip(qt, G64):
        v = v + float(q) * g
    return v + hs64


def random_record(rng, le, mag):
    qf = int(rng.integers(-2 ** mag, 2 ** mag))
    qt = [int(rng.integers(-2 ** min(mag, 30), 2 ** min(mag, 30))) for _ in range(le)]
    G64 = [float(rng.uniform(-1, 1) * 2.0 ** int(rng.integers(-12, 3))) for _ in range(le)]
    hs64 = float(rng.uniform(0, 64))
    return qf, qt, G64, hs64


@pytest.mark.parametrize("le", [1, 2, 3, 11])
def test_double_float_snap_agrees_with_exact_and_fp64(le):
    rng = np.random.default_rng(2107 + le)
    decided = 0
    for it in range(300):
        mag = int(rng.integers(4, 31))
        qf, qt, G64, hs64 = random_record(rng, le, mag)
        if it % 3 == 0:
            # move the residual to 0 .. 2^-20 steps from a tie through the shift
            y = y_exact(qf, qt, G64, 0.0)
            frac = y - math.floor(y)
            d = [0.0, 2.0 ** -40, -2.0 ** -40, 2.0 ** -26, -2.0 ** -22, 2.0 ** -20][it % 6]
            hs64 = float(Fraction(1, 2) - frac) + d + 8.0
        q, ok = df_snap(qf, qt, G64, hs64)
        if ok:
            decided += 1
            assert q == rint(y_exact(qf, qt, G64, hs64))
            assert q == int(np.rint(y_fp64(qf, qt, G64, hs64)))
    assert decided >= 150                      # the tier decides the ordinary cases


def test_exact_ties_round_to_even_in_fp32():
    rng = random.Random(5)
    ties = 0
    for _ in range(2000):
        e = -rng.randint(0, 6)                 # coefficients multiples of 2^e
        le = rng.randint(1, 4)
        G = [Fraction(rng.choice([-1, 1]) * rng.randint(1, 2 ** 10), 2 ** -e) for _ in range(le)]
        hs = Fraction(rng.randint(0, 2 ** 8), 2 ** -e)
        qt = [rng.randint(-2 ** 12, 2 ** 12) for _ in range(le)]
        qf = rng.randint(-2 ** 12, 2 ** 12)
        M = abs(qf) + sum(abs(q) * abs(g) for q, g in zip(qt, G)) + hs
        if not M < Fraction(2) ** (24 + e):
            continue
        for g in G + [hs]:                     # FP32-exact multiples of 2^e
            assert f32(g) == g and (g * Fraction(2) ** -e).denominator == 1
        v = f32(qf)
        for q, g in zip(qt, G):
            v = fma(q, g, v)                   # partial32: one FMA per essential parameter
        for sgn in (1, -1):
            y = add(v, sgn * hs)
            ye = Fraction(qf) + sum(Fraction(q) * g for q, g in zip(qt, G)) + sgn * hs
            assert y == ye                     # the FP32 residual is exact
            if abs(ye) < 4.0e6:                # the kernel's rounding (beyond: the FP64 snap)
                assert int(add(y, MAGIC) - MAGIC) == rint(ye)
            if abs(ye) < 32767:
                assert int(add(y, MAGIC16) - MAGIC16) == rint(ye)
                ties += (ye - math.floor(ye)) == Fraction(1, 2)
    assert ties > 50
