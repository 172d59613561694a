"""Host restatements of three pieces of integer/FP arithmetic the CUDA path
uses in place of plain FP64 operations, checked against exact arithmetic
(Python integers and fractions).  They mirror the device code step by step;
the GPU suite checks the device code itself (tests/test_gpu_fast_math.py,
and every parity test runs the other two).

- the panel exchange's fixed-point sums (fx_q / fx_x): partials bounded by
  2^(E-1), truncated to units of 2^(E-56), added as int64 in four copies,
  within P 2^(E-56) plus one rounding of the exact sum, and no overflow for
  P <= 256;
- ll_scaled: an int64 times 2^es rounded once to nearest-even, built from
  the integer's bits, equal to float(u) * 2^es;
- rcp_nr / sqrt_gm: Newton-Raphson reciprocal and Goldschmidt square root
  with a Newton correction, from a seed within 2^-22, within one ulp of the
  correctly rounded result.
"""
import math
import random
import struct
from fractions import Fraction

import numpy as np


def fma(a, b, c):
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def d2b(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def b2d(b):
    return struct.unpack("<d", struct.pack("<Q", b & (2 ** 64 - 1)))[0]


def f2b(x):
    return struct.unpack("<I", struct.pack("<f", x))[0]


def b2f(b):
    return struct.unpack("<f", struct.pack("<I", b))[0]


# ---------------------------------------------------------------- fixed point
def fx_q(x, E):
    return int(math.ldexp(x, 56 - E))  # truncation toward zero, as __double2ll_rz


def fx_x(q, E):
    return math.ldexp(float(q), E - 56)


def wrap64(v):
    v &= 2 ** 64 - 1
    return v - 2 ** 64 if v >= 2 ** 63 else v


def test_fixed_point_exchange_bound_and_no_overflow():
    rng = random.Random(7)
    for _ in range(3000):
        P = rng.randint(1, 256)
        E = rng.randint(-200, 200)
        spread = 2.0 ** rng.randint(-60, 0)
        xs = [rng.uniform(-1, 1) * spread * 2.0 ** (E - 1) for _ in range(P)]
        if rng.random() < 0.1:
            xs = [math.copysign(2.0 ** (E - 1), rng.uniform(-1, 1)) for _ in range(P)]  # at the bound
        copies = [0, 0, 0, 0]
        for r, x in enumerate(xs):
            q = fx_q(x, E)
            assert abs(q) <= 2 ** 55
            copies[r % 4] = wrap64(copies[r % 4] + q)
        total = 0
        for c in copies:
            assert abs(c) < 2 ** 63
            total = wrap64(total + c)
        exact = sum(Fraction(x) for x in xs)
        got = fx_x(total, E)
        err = abs(Fraction(got) - exact)
        bound = P * Fraction(2) ** (E - 56) + Fraction(math.ulp(abs(float(exact)) or 1e-300))
        assert err <= bound, (P, E, float(err), float(bound))


# ---------------------------------------------------------------- ll_scaled
def ll_scaled(u, es):
    if u == 0:
        return 0.0
    neg = u < 0
    a = -u if neg else u
    lz = 64 - a.bit_length()
    e = 63 - lz + es + 1023
    if e < 1 or e > 2045:
        return math.ldexp(float(u), es)  # the FP64 route
    a <<= lz
    m = a >> 11
    rem = a & 0x7FF
    if rem > 0x400 or (rem == 0x400 and (m & 1)):
        m += 1
    if m >> 53:
        m >>= 1
        e += 1
    return b2d((1 << 63 if neg else 0) | (e << 52) | (m & (2 ** 52 - 1)))


def test_ll_scaled_is_the_rounded_conversion():
    rng = random.Random(3)
    cases = [(1, 0), (-1, 0), (2 ** 53 + 1, 0), (2 ** 53 + 3, -7), (2 ** 63 - 1, 5), (-(2 ** 63), -3),
             ((2 ** 54 - 1) << 5, 0), (0x400 | (1 << 62), -60)]
    for _ in range(100000):
        cases.append((rng.getrandbits(rng.randint(1, 63)) * rng.choice([1, -1]), rng.randint(-300, 300)))
    for u, es in cases:
        assert ll_scaled(u, es) == math.ldexp(float(u), es), (u, es)


# ---------------------------------------------------------------- rcp / sqrt
def seed(v, rng):
    """A single-precision approximation within 2^-22, like rcp/rsqrt.approx."""
    return np.float32(v * (1.0 + rng.uniform(-(2.0 ** -22), 2.0 ** -22)))


def rcp_nr(d, rng):
    b = d2b(d)
    E = ((b >> 52) & 0x7FF) - 1023
    if E < -1000 or E > 1000:
        return 1.0 / d
    mf = b2f(0x3F800000 | ((b >> 29) & 0x7FFFFF))
    rb = f2b(float(seed(1.0 / float(mf), rng)))
    ye = ((rb >> 23) & 0xFF) - 127 - E + 1023
    y = b2d((b & (1 << 63)) | (ye << 52) | ((rb & 0x7FFFFF) << 29))
    e = fma(-d, y, 1.0)
    y = fma(y, e, y)
    e = fma(-d, y, 1.0)
    return fma(y, e, y)


def sqrt_gm(s, rng):
    b = d2b(s)
    E = ((b >> 52) & 0x7FF) - 1023
    if not s > 0.0 or E < -1000 or E > 1000:
        return math.sqrt(s)
    k = E >> 1
    fe = E - 2 * k
    mf = b2f(((127 + fe) << 23) | ((b >> 29) & 0x7FFFFF))
    rb = f2b(float(seed(1.0 / math.sqrt(float(mf)), rng)))
    ye = ((rb >> 23) & 0xFF) - 127 - k + 1023
    y = b2d((ye << 52) | ((rb & 0x7FFFFF) << 29))
    hy = b2d(((ye - 1) << 52) | ((rb & 0x7FFFFF) << 29))
    g = s * y
    r1 = fma(-g, hy, 0.5)
    g = fma(g, r1, g)
    h = fma(hy, r1, hy)
    dr = fma(-g, g, s)
    return fma(dr, h, g)


def test_newton_reciprocal_and_goldschmidt_sqrt_within_one_ulp():
    rng = random.Random(5)
    for _ in range(20000):
        x = math.ldexp(rng.uniform(1.0, 2.0), rng.randint(-990, 990)) * rng.choice([1.0, -1.0])
        r = rcp_nr(x, rng)
        assert abs(r - 1.0 / x) <= math.ulp(1.0 / x)
        a = abs(x)
        q = sqrt_gm(a, rng)
        assert abs(q - math.sqrt(a)) <= math.ulp(math.sqrt(a))
