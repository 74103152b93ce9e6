"""CPU restatement of the FP64-grade arithmetic of the mixed-precision Arnoldi
(the f53 basis and the FP32 three-word expansions), checked against exact
rational arithmetic.

The GPU stores every FP64 basis value x as an FP32 head (x with its fraction
truncated to 23 bits) and a 29-bit integer tail (the low fraction bits), and sums
products c x (c an FP32 coefficient) or u x (u another FP64 value) in three-word
FP32 expansions: products split exactly by FMA (TwoProd), TwoSum at the two
upper levels, a plain FP32 sum at the third, and a renormalisation every four
terms.  This file restates those steps with NumPy FP32 operations (IEEE round to
nearest; the fused multiply-add is evaluated exactly and rounded once) and checks
  - the codec: head + tail pieces reproduce x exactly, for every exponent in range;
  - the error of a sum of j products against the exact rational sum: below
    2^-60 sum |terms| (an FP64 evaluation of the same sum is allowed j 2^-53);
  - that the same sum in double-float (two words, the previous design) does not
    meet that bound, so the test would catch the third word being dropped.
It shares no code with the kernels (which are CUDA); it checks the design.
"""
from fractions import Fraction

import numpy as np
import pytest

F32 = np.float32


def rn32(q: Fraction) -> np.float32:
    """q rounded to the nearest FP32 value (ties to even), no double rounding."""
    if q == 0:
        return F32(0.0)
    s = -1 if q < 0 else 1
    q = abs(q)
    e = q.numerator.bit_length() - q.denominator.bit_length()
    if Fraction(2) ** e > q:
        e -= 1
    e = max(e, -126)                       # subnormal range: fixed quantum 2^-149
    m = q / Fraction(2) ** (e - 23)        # in [2^23, 2^24) for normal values
    n, r = divmod(m.numerator, m.denominator)
    if 2 * r > m.denominator or (2 * r == m.denominator and n % 2 == 1):
        n += 1
    return F32(s * float(Fraction(n) * Fraction(2) ** (e - 23)))


def fma32(a, b, c) -> np.float32:
    return rn32(Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c)))


def two_sum(a, b):
    s = F32(a + b)
    bb = F32(s - a)
    e = F32(F32(a - F32(s - bb)) + F32(b - bb))
    return s, e


def two_diff(a, b):
    # s - en = a - b exactly
    s = F32(a - b)
    bb = F32(s - a)
    en = F32(F32(F32(s - bb) - a) + F32(b + bb))
    return s, en


# ---- the f53 codec (integer operations on the FP64 and FP32 words)
def f53_encode(x: float):
    b = np.array([x], dtype=np.float64).view(np.uint64)[0]
    H, L = int(b >> np.uint64(32)), int(b & np.uint64(0xFFFFFFFF))
    a, sg = H & 0x7FFFFFFF, H & 0x80000000
    hb = ((((a - (896 << 20)) << 3) | (L >> 29)) & 0xFFFFFFFF) | sg
    t = L & 0x1FFFFFFF
    if a < (926 << 20):
        hb, t = sg, 0
    if a >= (1151 << 20):
        hb, t = 0x7FC00000, 0
    return np.array([hb], dtype=np.uint32).view(np.float32)[0], t


def f53_low(head, tail):
    hb = int(np.array([head], dtype=np.float32).view(np.uint32)[0])
    F1 = ((hb & 0xFF800000) - (23 << 23)) & 0xFFFFFFFF
    F2 = (F1 - (6 << 23)) & 0xFFFFFFFF
    asf = lambda u: np.array([u & 0xFFFFFFFF], dtype=np.uint32).view(np.float32)[0]
    v1 = F32(asf(F1 | (tail >> 6)) - asf(F1))
    v2 = F32(asf(F2 | (tail & 63)) - asf(F2))
    return v1, v2


def f53_double(head, tail):
    hb = int(np.array([head], dtype=np.float32).view(np.uint32)[0])
    a = hb & 0x7FFFFFFF
    H = (hb & 0x80000000) | ((a >> 3) + (896 << 20))
    if a < 0x00800000:
        H = hb & 0x80000000
    if a >= 0x7F800000:
        H = 0x7FF80000
    L = ((hb << 29) & 0xFFFFFFFF) | tail
    return float(np.array([(H << 32) | L], dtype=np.uint64).view(np.float64)[0])


def test_f53_codec_is_exact():
    rng = np.random.default_rng(7)
    xs = list(rng.standard_normal(2000) * np.exp2(rng.integers(-90, 120, 2000)))
    xs += [0.0, -0.0, 1.0, -1.0, 2.0 ** -96, -(2.0 ** 127) * 1.5, float(np.nextafter(1.0, 2.0))]
    for x in xs:
        h, t = f53_encode(x)
        assert f53_double(h, t) == x
        v1, v2 = f53_low(h, t)
        assert Fraction(float(h)) + Fraction(float(v1)) + Fraction(float(v2)) == Fraction(x)
        # the pieces are ordered: |v1| < 2^-23 |head|, |v2| < 2^-46 |head|
        if x != 0.0:
            assert abs(float(v1)) < 2.0 ** -22 * abs(float(h)) and abs(float(v2)) < 2.0 ** -45 * abs(float(h))
    # below the range: a signed zero; above it: NaN
    assert f53_encode(2.0 ** -100)[0] == 0.0 and f53_encode(2.0 ** -100)[1] == 0
    assert np.isnan(f53_encode(2.0 ** 129)[0]) and np.isnan(f53_encode(float("inf"))[0])


# ---- three-word expansion accumulators
class TF:
    def __init__(self):
        self.s = [F32(0.0), F32(0.0), F32(0.0)]

    def add0(self, x):
        self.s[0], t = two_sum(self.s[0], x)
        self.s[1], t2 = two_sum(self.s[1], t)
        self.s[2] = F32(self.s[2] + t2)

    def add1(self, x):
        self.s[1], t = two_sum(self.s[1], x)
        self.s[2] = F32(self.s[2] + t)

    def sub1(self, x):
        self.s[1], en = two_diff(self.s[1], x)
        self.s[2] = F32(self.s[2] - en)

    def renorm(self):
        self.s[0], t = two_sum(self.s[0], self.s[1])
        self.s[1], self.s[2] = two_sum(t, self.s[2])

    def value(self):
        return sum(Fraction(float(v)) for v in self.s)


def mac24(A: TF, c, x):
    """A += c x, c an FP32 value, x an FP64 value (f53 pieces)."""
    h, t = f53_encode(x)
    v1, v2 = f53_low(h, t)
    nc = F32(-c)
    p0 = F32(c * h); e0n = fma32(nc, h, p0)
    p1 = F32(c * v1); e1n = fma32(nc, v1, p1)
    A.add0(p0)
    A.add1(p1)
    A.sub1(e0n)
    A.s[2] = F32(fma32(c, v2, A.s[2]) - e1n)


def mac53(A: TF, u, x):
    """A += u x for two FP64 values (both as f53 pieces)."""
    uh, ut = f53_encode(u)
    u1, u2 = f53_low(uh, ut)
    h, t = f53_encode(x)
    v1, v2 = f53_low(h, t)
    p0 = F32(uh * h); e0n = fma32(F32(-uh), h, p0)
    p1 = F32(uh * v1); e1n = fma32(F32(-uh), v1, p1)
    p2 = F32(u1 * h); e2n = fma32(F32(-u1), h, p2)
    A.add0(p0)
    A.add1(p1)
    A.add1(p2)
    A.sub1(e0n)
    l2 = fma32(uh, v2, A.s[2])
    l2 = fma32(u1, v1, l2)
    l2 = fma32(u2, h, l2)
    A.s[2] = F32(F32(l2 - e1n) - e2n)


def df_mac24(S, c, x):
    """The same sum in double-float: (sh, sl) += c (head + v1), TwoSum on the head only."""
    h, t = f53_encode(x)
    v1, _ = f53_low(h, t)
    p = F32(c * h)
    en = fma32(F32(-c), h, p)
    en = fma32(F32(-c), v1, en)
    s, tt = two_sum(S[0], p)
    S[0], S[1] = s, F32(S[1] + F32(tt - en))


def _cancelling_terms(rng, j):
    """j coefficient/value pairs whose sum cancels to about 2^-20 of sum |terms|
    (the regime of a Gram-Schmidt projection)."""
    x = rng.standard_normal(j) * np.exp2(rng.integers(-6, 6, j))
    c = rng.standard_normal(j).astype(np.float32)
    exact = sum(Fraction(float(ci)) * Fraction(float(xi)) for ci, xi in zip(c, x))
    # make the last term cancel the rest up to a small remainder
    target = float(-(exact - Fraction(float(c[-1])) * Fraction(float(x[-1]))))
    x[-1] = target / float(c[-1]) * (1 + 2.0 ** -20)
    return c, x


@pytest.mark.parametrize("j", [4, 37, 200])
def test_three_word_sum_of_fp32_times_fp64_beats_fp64(j):
    rng = np.random.default_rng(j)
    c, x = _cancelling_terms(rng, j)
    A = TF()
    for k in range(j):
        mac24(A, c[k], float(x[k]))
        if k % 4 == 3:
            A.renorm()
    terms = [Fraction(float(ci)) * Fraction(float(xi)) for ci, xi in zip(c, x)]
    exact, mag = sum(terms), sum(abs(t) for t in terms)
    assert abs(A.value() - exact) <= Fraction(2) ** -60 * mag
    # double-float does not reach that bound on the same sum
    S = [F32(0.0), F32(0.0)]
    for k in range(j):
        df_mac24(S, c[k], float(x[k]))
    if j >= 37:
        assert abs(Fraction(float(S[0])) + Fraction(float(S[1])) - exact) > Fraction(2) ** -60 * mag


@pytest.mark.parametrize("j", [5, 64])
def test_three_word_sum_of_fp64_products_beats_fp64(j):
    rng = np.random.default_rng(100 + j)
    u = rng.standard_normal(j) * np.exp2(rng.integers(-5, 5, j))
    x = rng.standard_normal(j) * np.exp2(rng.integers(-5, 5, j))
    A = TF()
    for k in range(j):
        mac53(A, float(u[k]), float(x[k]))
        if k % 4 == 3:
            A.renorm()
    terms = [Fraction(float(a)) * Fraction(float(b)) for a, b in zip(u, x)]
    exact, mag = sum(terms), sum(abs(t) for t in terms)
    assert abs(A.value() - exact) <= Fraction(2) ** -60 * mag


def _f2d_bits(u: int) -> int:
    """The integer FP32 -> FP64 conversion of the mixed path's outer operator, restated:
    (sign, exponent + 896, fraction << 29); zero keeps its sign, the all-ones exponent
    maps to FP64's; subnormal inputs are left to the conversion instruction (None)."""
    e = (u >> 23) & 0xFF
    m = u & 0x7FFFFF
    sg = u & 0x80000000
    if e == 0:
        return None if m else sg << 32
    hi = sg | ((0x7FF if e == 0xFF else e + 896) << 20) | (m >> 3)
    return (hi << 32) | ((m << 29) & 0xFFFFFFFF)


def test_integer_fp32_to_fp64_conversion_is_exact():
    rng = np.random.default_rng(5)
    bits = list(rng.integers(0, 2**32, size=20000, dtype=np.uint64))
    bits += [0x00000000, 0x80000000, 0x7F800000, 0xFF800000, 0x7F7FFFFF, 0x00800000, 0x80800000,
             0x3F800000, 0x7FC00000, 0x7F800001, 0x00000001, 0x807FFFFF]
    for u in bits:
        u = int(u)
        got = _f2d_bits(u)
        if got is None:
            continue
        with np.errstate(invalid="ignore"):
            ref = np.array([u], dtype=np.uint32).view(np.float32).astype(np.float64).view(np.uint64)[0]
        x = np.array([u], dtype=np.uint32).view(np.float32)[0]
        if np.isnan(x):
            # NaN stays NaN (quiet bit and payload carried in the fraction)
            assert (got >> 52) & 0x7FF == 0x7FF and got & ((1 << 52) - 1) != 0
            continue
        assert got == int(ref), hex(u)
