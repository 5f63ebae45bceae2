"""Bitwise pins of the oracle's pow against the correctly rounded x^y.

Listing 5 (Section 4) leaves pow to the platform; this library defines its
own (binary64 in fixed-point integer arithmetic, binary32 in double-word
arithmetic), and the kernels reproduce that definition bit for bit.  These
tests pin the definition to something other than itself: the exact value
x^y from mpmath at 300 bits, rounded to nearest-even in the format by
integer arithmetic here.

- binary64: within 0.5 + 2^-8 ulp everywhere sampled, and bitwise equal to
  RN(x^y) wherever x^y lies more than 2^-8 ulp from a rounding midpoint
  (a nearly correctly rounded pow: any error above 2^-8 ulp before the final
  rounding -- a dropped series term, a wrong table entry, a truncated
  product -- fails here).
- binary32: within 0.75 ulp, and bitwise RN(x^y) wherever x^y lies more than
  0.25 ulp from a midpoint.

Operands cover the two domains v1_lp uses (Q in [0, 1] with y = p/2, Z in
[1, 2] with y = 1/p, both rounded in the format as the tree does), their
ends next to 1, and for binary64 a wide domain (x near 1 with large y,
subnormal x, |y log2 x| up to 1100, random bit patterns).
"""
import math
import random
import struct

import mpmath
import numpy as np
import pytest

import oracle

PREC = 300


def _rn(ex, mant, emin):
    """RN-even of the positive mpmath value ex in a binary format with `mant`
    fraction bits and smallest normal exponent `emin`: returns (value as a
    Python float, distance of ex from the nearest rounding midpoint in ulps,
    quantum exponent)."""
    man, exp = int(ex.man), int(ex.exp)  # ex = man 2^exp exactly
    e = exp + man.bit_length() - 1      # floor(log2 ex)
    q = max(e, emin) - mant             # quantum of the binade (subnormals: 2^(emin - mant))
    sh = q - exp
    if sh <= 0:                         # ex is a multiple of the quantum (man odd, <= 53 bits)
        return math.ldexp(man, exp), 0.5, q
    fl = man >> sh
    rem = man - (fl << sh)
    half = 1 << (sh - 1)
    if rem > half or (rem == half and (fl & 1)):
        fl += 1
    dist = abs(rem - half) / (1 << sh)  # exact integers, one rounding
    return math.ldexp(fl, q), dist, q


def _ulp_err(v, ex, q):
    return float(abs(mpmath.mpf(float(v)) - ex) / mpmath.ldexp(1, q))


def _lp_domain(dt, n, seed):
    """Operands of the two pows of v1_lp: S = pow(Q, h), h = p/2 rounded in
    dt, Q = RN(m/M) in [0, 1]; C = pow(Z, ip), ip = 1/p rounded in dt,
    Z = RN(1 + S^2) in [1, 2]; p from the paper's Table 4 values, the
    benchmark's and random ones; x drawn plainly and next to 1."""
    r = random.Random(seed)
    ps = [0.5, 2 / 3, 1.0 + 1e-9, 1.5, math.sqrt(2), math.e, math.pi, 3.0, 7.5, 64.0]
    xs, ys = np.empty(n, dt), np.empty(n, dt)
    for i in range(n):
        p = dt(r.choice(ps) if r.random() < 0.5 else r.uniform(0.3, 40.0))
        kind = i % 4
        if kind == 0:
            x, y = r.random() ** r.choice([1, 2, 5, 20, 60]), p * dt(0.5)
        elif kind == 1:
            x, y = 1.0 + r.random(), dt(1) / p
        elif kind == 2:
            x, y = 1.0 - r.random() * 2.0 ** -r.randint(1, 40), p * dt(0.5)
        else:
            x, y = 1.0 + r.random() * 2.0 ** -r.randint(1, 40), dt(1) / p
        xs[i], ys[i] = x, y
    ok = xs > 0
    return xs[ok], ys[ok]


def _bits_d(u):
    return struct.unpack("<d", struct.pack("<Q", u))[0]


def _wide_domain_d(n, seed):
    r = random.Random(seed)
    xs, ys = [], []
    while len(xs) < n:
        kind = len(xs) % 6
        if kind == 0:
            x = 1 + r.uniform(-1, 1) * 2.0 ** r.randint(-52, -1)
            y = r.uniform(0.5, 2) * 2.0 ** r.randint(-60, 60)
        elif kind == 1:
            x = r.uniform(0.5, 2) * 2.0 ** r.randint(-1074, -1000)
            y = r.uniform(0.01, 1.1)
        elif kind == 2:
            x = r.uniform(0.1, 4)
            y = abs(r.uniform(-1, 1) * 1100 / max(abs(math.log2(x)), 1e-3)) or 1.0
        elif kind == 3:
            x = _bits_d(r.getrandbits(63))
            y = _bits_d(r.getrandbits(63))
        elif kind == 4:
            x = r.random() ** r.choice([1, 3, 20])
            y = r.uniform(0.01, 12)
        else:
            x = 1 + r.random()
            y = 1 / r.uniform(0.05, 40)
        if not (math.isfinite(x) and math.isfinite(y)) or x == 0 or y == 0:
            continue
        xs.append(x)
        ys.append(y)
    return np.array(xs), np.array(ys)


def _check(x, y, dt, max_ulp, margin):
    """Returns (cases checked, cases decided bitwise, worst ulp error);
    asserts the error bound and bitwise RN away from the midpoints."""
    mant, emin, emax = (52, -1022, 1024) if dt == np.float64 else (23, -126, 128)
    tiny = mpmath.ldexp(1, emin - mant - 1)  # half the smallest subnormal
    big = mpmath.ldexp(1, emax)
    v = oracle.pow_arr(x.astype(dt), y.astype(dt))
    checked = decided = 0
    worst = 0.0
    with mpmath.workprec(PREC):
        for i in range(x.size):
            xi, yi, vi = float(x[i]), float(y[i]), float(v[i])
            ex = mpmath.mpf(xi) ** mpmath.mpf(yi)
            if ex >= big:
                assert vi == math.inf, (xi.hex(), yi.hex(), vi)
                continue
            if ex <= tiny:  # rounds to +0 (a tie at half the smallest subnormal goes to even, +0)
                assert vi == 0.0, (xi.hex(), yi.hex(), vi)
                continue
            want, dist, q = _rn(ex, mant, emin)
            err = _ulp_err(vi, ex, q)
            worst = max(worst, err)
            assert err <= max_ulp, (xi.hex(), yi.hex(), err)
            checked += 1
            if dist > margin:
                decided += 1
                assert vi == want, ("not RN(x^y)", xi.hex(), yi.hex(), vi, want, dist)
    return checked, decided, worst


def test_rounding_helper_on_known_values():
    """_rn against values whose rounding is known: exact binary64 values,
    midpoints (ties to even), values just off a midpoint, subnormals."""
    with mpmath.workprec(PREC):
        one = mpmath.mpf(1)
        u = mpmath.ldexp(1, -52)
        assert _rn(one, 52, -1022)[0] == 1.0
        assert _rn(one + u / 2, 52, -1022)[0] == 1.0                   # tie -> even
        assert _rn(one + 3 * u / 2, 52, -1022)[0] == 1.0 + 2 * 2.0 ** -52  # tie -> even (up)
        v, d, _ = _rn(one + u / 2 + mpmath.ldexp(1, -200), 52, -1022)
        assert v == 1.0 + 2.0 ** -52 and d < 1e-40
        v, d, _ = _rn(one + u / 4, 52, -1022)
        assert v == 1.0 and abs(d - 0.25) < 1e-15
        assert _rn(mpmath.ldexp(3, -1075), 52, -1022)[0] == 2 * 5e-324  # 1.5 quanta -> 2 (even)
        assert _rn(mpmath.ldexp(5, -1076), 52, -1022)[0] == 5e-324      # 1.25 quanta -> 1
        assert _rn(mpmath.mpf(1) / 3, 23, -126)[0] == float(np.float32(1 / 3))
        assert _rn(mpmath.sqrt(2), 52, -1022)[0] == math.sqrt(2)


def test_pow_d_correctly_rounded_on_lp_domains():
    """1.2e5 operand pairs of v1_lp's two pows in binary64."""
    x, y = _lp_domain(np.float64, 120000, seed=31)
    checked, decided, worst = _check(x, y, np.float64, 0.5 + 2.0 ** -8, 2.0 ** -8)
    assert checked > 100000 and decided > 0.98 * checked
    assert worst > 0.45  # the sample reaches the rounding error itself


def test_pow_d_correctly_rounded_wide():
    """3e4 binary64 pairs from the wide domain (large y next to x = 1,
    subnormal x, results near overflow and in the subnormal range, raw
    bits)."""
    x, y = _wide_domain_d(30000, seed=37)
    checked, decided, worst = _check(x, y, np.float64, 0.5 + 2.0 ** -8, 2.0 ** -8)
    assert checked > 20000 and decided > 0.98 * checked


def test_pow_s_nearly_correctly_rounded_on_lp_domains():
    """1.2e5 operand pairs of v1_lp's two pows in binary32: within 0.75 ulp,
    and RN(x^y) wherever x^y is more than 0.25 ulp from a midpoint."""
    x, y = _lp_domain(np.float32, 120000, seed=41)
    checked, decided, worst = _check(x, y, np.float32, 0.75, 0.25)
    assert checked > 100000 and decided > 0.4 * checked
    assert worst > 0.45


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_pin_catches_a_planted_error(dt):
    """The pin is sharp enough to see a one-ulp slip: the oracle's pow with
    its result moved by one ulp on 1 case in 64 fails the bitwise check."""
    x, y = _lp_domain(dt, 4000, seed=43)
    v = oracle.pow_arr(x, y)
    bad = v.copy()
    idx = np.arange(0, v.size, 64)
    bad[idx] = np.nextafter(v[idx], dt(np.inf))
    mant, emin = (52, -1022) if dt == np.float64 else (23, -126)
    margin = 2.0 ** -8 if dt == np.float64 else 0.25
    caught = 0
    with mpmath.workprec(PREC):
        for i in idx:
            ex = mpmath.mpf(float(x[i])) ** mpmath.mpf(float(y[i]))
            want, dist, _ = _rn(ex, mant, emin)
            if dist > margin and float(bad[i]) != want:
                caught += 1
    assert caught > 0.5 * idx.size
