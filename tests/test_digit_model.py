"""Exact model of the digit recurrences behind the binary64 v1_hypot of the
tree kernels (integer long division and integer square root from FP32
estimates), checking the bounds their correctness rests on -- not an
oracle: nothing here is compared with the GPU.

Each FP32 step is emulated with correctly rounded binary32 arithmetic; the
hardware reciprocal and reciprocal-square-root approximations are modelled
as the correctly rounded value moved by up to PERT ulps either way, so the
bounds hold for any approximation at least that good.  Checked:

- the rounded 54-bit quotient: with the last digit the FP32 estimate of
  W2 2^13 / B rounded to nearest, the remainder before the correction lies
  in [-B, B) (so a negative remainder is the only correction), and
  (floor(Num 2^53 / B) + 1) / 2 is RN(Num 2^52 / B) (no ties in division);
- the integer square root of (2^52 + F) 2^(52 + o): the candidate TT is the
  floor or one above it, the intermediate remainders stay below 2^36 and
  2^43, and TT - 1 + [W3 > -TT] + [W3 > TT] is RN(sqrt(N));
- the paired form's square root (o = 0): the last digit taken for
  2 sqrt(N) (the same estimate times 2), TT2 = 2 Tp + T3 the floor of
  2 sqrt(N) or one above it, W3 = 4 N - TT2^2, and
  (TT2 - [W3 < 0] + 1) / 2 is RN(sqrt(N));
- two identities of the restricted pow's integer steps: the final
  round-to-nearest-even as one carry, and 128-bit negation as
  (v ^ mask) - mask.
"""
import math
import random
import struct
from fractions import Fraction

import numpy as np

PERT = 64
HID = 1 << 52
M64 = (1 << 64) - 1


def f32(x):
    return np.float32(x)


def fbits(f):
    return struct.unpack("<I", struct.pack("<f", float(f)))[0]


def bitsf(u):
    return np.float32(struct.unpack("<f", struct.pack("<I", u & 0xFFFFFFFF))[0])


def rn32(v):
    """Round an exact rational to the nearest binary32 (ties to even)."""
    if v == 0:
        return f32(0.0)
    f = np.float32(float(v))
    cands = [f, np.nextafter(f, np.float32(np.inf)), np.nextafter(f, np.float32(-np.inf))]
    return min(cands, key=lambda c: (abs(Fraction(float(c)) - v), fbits(c) & 1))


def mul32(a, b):
    return rn32(Fraction(float(a)) * Fraction(float(b)))


def fma32(a, b, c):
    return rn32(Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c)))


def i2f(v):
    return rn32(Fraction(v))


def s64(v):
    v &= M64
    return v - (1 << 64) if v >> 63 else v


def round_small(t):
    """Nearest integer of |t| < 2^22 (the kernels' 1.5 2^23 magic add)."""
    assert abs(float(t)) < 2 ** 22
    magic = f32(1.5 * 2 ** 23)
    return fbits(rn32(Fraction(float(t)) + Fraction(float(magic)))) - fbits(magic)


class Approx:
    """The FP32 estimates, perturbed by up to PERT ulps."""

    def __init__(self, rng):
        self.rng = rng

    def _pert(self, f):
        return bitsf(fbits(f) + self.rng.randint(-PERT, PERT))

    def rcp(self, x):
        return self._pert(rn32(1 / Fraction(float(x))))

    def rsqrt(self, x):
        return self._pert(f32(1.0 / math.sqrt(float(x))))


def div_54r(num, b, ap, stats):
    """The rounded quotient RN(num 2^52 / b), num in [b, 2b), b in [2^52, 2^53)."""
    bhi = b >> 29
    fb = bitsf(0x4B000000 | (bhi - (1 << 23)))
    assert float(fb) == bhi
    r0 = ap.rcp(fb)
    r = fma32(r0, fma32(-fb, r0, f32(1)), r0)
    q1 = round_small(mul32(mul32(i2f(num >> 29), r), f32(2.0 ** 20)))
    w1 = s64((num << 20) - q1 * b)
    assert abs(w1) < 2 * b
    q2 = round_small(mul32(mul32(i2f(w1 >> 24), r), f32(2.0 ** 15)))
    w2 = s64((w1 << 20) - q2 * b)
    assert abs(w2) < 3 * b
    q3 = round_small(mul32(mul32(i2f(w2 >> 24), r), f32(2.0 ** 8)))
    w3 = s64((w2 << 13) - q3 * b)
    stats["div"] = max(stats["div"], abs(Fraction(w3, b)))
    assert -b <= w3 < b, "remainder outside [-B, B): a second correction would be needed"
    q54 = (q1 << 33) + (q2 << 13) + q3 - (1 if w3 < 0 else 0)
    assert q54 == (num << 53) // b
    return (q54 + 1) >> 1


def isqrt_rn(f, o, ap, stats):
    """RN(sqrt(N)) for N = (2^52 + f) 2^(52 + o)."""
    sint = (HID + f) << o
    fs = bitsf((0x3F800000 + (o << 23)) | (f >> 29)) if f < HID else f32(2.0)
    y0 = ap.rsqrt(fs)
    e = fma32(-mul32(fs, y0), y0, f32(1))
    y = fma32(mul32(y0, f32(0.5)), e, y0)
    t1 = round_small(mul32(mul32(fs, y), f32(2.0 ** 20)))
    w1 = s64(sint - ((t1 * t1) << 12))
    assert abs(w1) < 2 ** 36
    t2 = round_small(mul32(mul32(i2f(w1 >> 8), y), f32(2.0 ** -5)))
    w2 = s64((w1 << 28) - ((2 * t1 * t2) << 20) - t2 * t2)
    assert abs(w2) < 2 ** 43
    t3 = round_small(mul32(mul32(i2f(w2 >> 16), y), f32(2.0 ** -13)))
    tp = (t1 << 32) + (t2 << 12)
    w3 = s64((w2 << 24) - ((tp * t3) << 1) - t3 * t3)
    tt = tp + t3
    n = sint << 52
    assert w3 == n - tt * tt
    fl = math.isqrt(n)
    stats["sqrt"].add(tt - fl)
    assert tt - fl in (0, 1), "candidate is not the floor or one above it"
    return tt - 1 + (1 if w3 > -tt else 0) + (1 if w3 > tt else 0)


def isqrt_rn2(sint, ap, stats):
    """RN(sqrt(N)) for N = sint 2^52, sint = 2^52 + f in [2^52, 2^53]: the
    paired kernels' form (the FP32 value of sint 2^-52 from sint's bits, the
    first remainder from (T1 2^6)^2, the last digit for 2 sqrt(N))."""
    fs = bitsf(0x3F000000 + ((sint >> 29) & 0xFFFFFFFF))
    assert fs == (bitsf(0x3F800000 | ((sint - HID) >> 29)) if sint < 2 * HID else f32(2.0))
    y0 = ap.rsqrt(fs)
    e = fma32(-mul32(fs, y0), y0, f32(1))
    y = fma32(mul32(y0, f32(0.5)), e, y0)
    t1 = round_small(mul32(mul32(fs, y), f32(2.0 ** 20)))
    assert 0 <= t1 << 6 < 2 ** 32
    w1 = s64(sint - (t1 << 6) * (t1 << 6))
    assert w1 == s64(sint - ((t1 * t1) << 12)) and abs(w1) < 2 ** 36
    t2 = round_small(mul32(mul32(i2f(w1 >> 8), y), f32(2.0 ** -5)))
    # the cross term as one signed 32 x 32 product: t1 2^10 and t2 2^11 fit
    assert 0 <= t1 * 1024 < 2 ** 31 and -2 ** 31 <= t2 * 2048 < 2 ** 31
    w2 = s64((w1 << 28) - (t1 * 1024) * (t2 * 2048) - t2 * t2)
    assert w2 == s64((w1 << 28) - ((2 * t1 * t2) << 20) - t2 * t2)
    assert abs(w2) < 2 ** 43
    stats["t2"] = max(stats.get("t2", 0), abs(t2))
    t3 = round_small(mul32(mul32(i2f(w2 >> 16), y), f32(2.0 ** -12)))
    tp2 = (t1 << 33) + (t2 << 13)
    w3 = s64((w2 << 26) - s64(tp2 * 2 * t3) - t3 * t3)
    n = sint << 52
    tt2 = tp2 + t3
    assert w3 == 4 * n - tt2 * tt2
    fl2 = math.isqrt(4 * n)
    stats["sqrt2"].add(tt2 - fl2)
    assert tt2 - fl2 in (0, 1), "candidate is not the floor of 2 sqrt(N) or one above it"
    u = tp2 + (t3 + 1 + (-1 if w3 < 0 else 0))
    assert u - 1 == fl2
    # the bits of s = RN(sqrt(N)) 2^-52 with 1/2's added doubled before the halving
    sbits = (tp2 + (0x3FE0000000000000 << 1) + (t3 + 1 + (-1 if w3 < 0 else 0))) >> 1
    assert sbits == 0x3FF0000000000000 | ((u >> 1) & (HID - 1))
    return (u & M64) >> 1


def rn_quotient(num, b):
    fl, rem = divmod(num << 52, b)
    return fl + (1 if 2 * rem > b or (2 * rem == b and fl & 1) else 0)


def rn_sqrt(n):
    s = math.isqrt(n)
    return s + (1 if n - s * s > s else 0)


def test_rounded_quotient_digits():
    rng = random.Random(11)
    ap = Approx(random.Random(12))
    stats = {"div": Fraction(0)}
    cases = []
    for b in (HID, HID + 1, 2 * HID - 1, HID + (1 << 29), HID + (1 << 29) - 1, 3 << 51):
        for num in (b, b + 1, 2 * b - 1, b + (b >> 1)):
            cases.append((num, b))
    for _ in range(1500):
        b = HID | rng.getrandbits(52)
        cases.append((b + rng.randrange(b), b))
        # quotients next to a rounding boundary of the 53-bit result
        k = (1 << 53) + rng.getrandbits(53)
        num = (k * b + rng.randrange(-3, 4) * (b >> 1)) >> 53
        if b <= num < 2 * b:
            cases.append((num, b))
    for num, b in cases:
        assert div_54r(num, b, ap, stats) == rn_quotient(num, b), (num, b)
    # the remainder before the correction stays near half a divisor
    assert stats["div"] < Fraction(51, 100)


def test_rounded_square_root_digits():
    rng = random.Random(21)
    ap = Approx(random.Random(22))
    stats = {"sqrt": set()}
    fs = [0, 1, 2, HID - 1, HID - 2, 1 << 51, (1 << 51) + 1]
    for _ in range(1500):
        fs.append(rng.getrandbits(52))
        # roots next to a half-integer: N close to t^2 + t
        t = (1 << 52) + rng.getrandbits(52)
        f2 = ((t * t + t) >> 52) - HID
        if 0 <= f2 < HID:
            fs.append(f2)
    for o in (0, 1):
        for f in fs + ([HID] if o == 0 else []):
            n = ((HID + f) << o) << 52
            assert isqrt_rn(f, o, ap, stats) == rn_sqrt(n), (f, o)
    assert stats["sqrt"] <= {0, 1}


def test_rounded_square_root_paired_form():
    rng = random.Random(31)
    ap = Approx(random.Random(32))
    stats = {"sqrt2": set()}
    fs = [0, 1, 2, HID - 1, HID - 2, HID, 1 << 51, (1 << 51) + 1]
    for _ in range(2000):
        fs.append(rng.getrandbits(52))
        t = (1 << 52) + rng.getrandbits(52)
        f2 = ((t * t + t) >> 52) - HID   # roots next to a half-integer
        if 0 <= f2 < HID:
            fs.append(f2)
        f3 = ((t * t) >> 52) - HID       # roots next to an integer
        if 0 <= f3 < HID:
            fs.append(f3)
    for f in fs:
        n = (HID + f) << 52
        assert isqrt_rn2(HID + f, ap, stats) == rn_sqrt(n), f
    assert stats["sqrt2"] == {0, 1}
    # |T2| <= 2^20 |2^20 sqrt(S 2^-52) - T1| + small, and T1 is within
    # 1/2 + 0.18 (the estimate) + 0.09 (the truncated fS) of 2^20 sqrt(S 2^-52)
    assert stats["t2"] < 0.8 * 2 ** 20


def test_division_has_no_ties():
    """The fact that lets the kernels round the quotient from one extra bit:
    2 Num 2^52 / B is never an odd integer for 53-bit significands (it would
    need 2^53 to divide B); checked exhaustively on a scaled-down format
    (p = 10 bits) and by the divisibility argument on random 53-bit ones."""
    p = 10
    lo, hi = 1 << (p - 1), 1 << p
    for b in range(lo, hi):
        for a in range(lo, hi):
            num = a if a >= b else 2 * a
            q2, r = divmod(num << p, b)
            assert not (r == 0 and q2 & 1), (a, b)
    rng = random.Random(5)
    for _ in range(2000):
        b = HID | rng.getrandbits(52)
        num = b + rng.randrange(b)
        q2, r = divmod(num << 53, b)
        assert not (r == 0 and q2 & 1)


def test_dividend_shifts_of_the_paired_form():
    """The paired form takes Num 2^20 (mod 2^64) and floor(Num 2^-29) as single
    shifts of A (Num = A or 2A): A << s and A >> (49 - s), s = 20 or 21."""
    rng = random.Random(41)
    for _ in range(5000):
        a, b = HID | rng.getrandbits(52), HID | rng.getrandbits(52)
        num = a if a >= b else a << 1
        s = 20 if a >= b else 21
        assert (a << s) & M64 == (num << 20) & M64
        assert a >> (49 - s) == num >> 29


def test_pow_final_rounding_by_carry():
    """The restricted pow's last step rounds P in [2^126, 2^128) (two 64-bit
    words) to 53 bits, ties to even, as one carry: q = hi >> sh, the bits
    below q (hi mod 2^sh, with lo != 0 OR-ed into bit 0 as a sticky bit,
    which lies below the half bit since sh >= 10) plus half - 1 plus q's
    last bit carry into bit sh exactly when q rounds up."""
    rng = random.Random(51)
    cases = []
    for _ in range(20000):
        top = rng.randrange(2)
        hi = (1 << (62 + top)) | rng.getrandbits(62 + top)
        lo = rng.getrandbits(64) if rng.random() < 0.7 else 0
        sh = 10 + top
        # push some cases to exact halves and to the neighbours of halves
        if rng.random() < 0.3:
            hi = (hi >> sh << sh) | (1 << (sh - 1)) | rng.choice([0, 0, 1])
            if rng.random() < 0.5:
                lo = 0
        cases.append((hi, lo))
    cases.append(((1 << 64) - 1, (1 << 64) - 1))  # rounds up to 2^53
    for hi, lo in cases:
        top = hi >> 63
        sh = 10 + top
        q = hi >> sh
        half = 1 << (sh - 1)
        low = (hi & (2 * half - 1)) | (1 if lo else 0)
        m = q + ((low + (half - 1) + (q & 1)) >> sh)
        # reference: round half to even of (hi 2^64 + lo) / 2^(64 + sh)
        num, den = (hi << 64) | lo, 1 << (64 + sh)
        fl, rem = divmod(num, den)
        ref = fl + (1 if 2 * rem > den or (2 * rem == den and fl & 1) else 0)
        assert m == ref, (hex(hi), hex(lo))


def test_masked_negation_of_128_bit_values():
    """(v ^ mask) - mask is v for mask = 0 and -v (mod 2^128) for mask = all
    ones, the form the restricted pow uses to take |W| and to give the sign
    back, applied to the two 64-bit words with a borrow between them."""
    rng = random.Random(52)
    M128 = (1 << 128) - 1
    for _ in range(5000):
        v = rng.getrandbits(128)
        for neg in (False, True):
            mk = M128 if neg else 0
            got = ((v ^ mk) - mk) & M128
            assert got == ((-v) & M128 if neg else v)
            # word by word: the low word's borrow enters the high word
            m64 = (1 << 64) - 1 if neg else 0
            vh, vl = v >> 64, v & ((1 << 64) - 1)
            lo = (vl ^ m64) - m64
            borrow = 1 if lo < 0 else 0
            hi = ((vh ^ m64) - m64 - borrow) & ((1 << 64) - 1)
            assert (hi << 64) | (lo & ((1 << 64) - 1)) == got
