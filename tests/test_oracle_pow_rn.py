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


def _powr_domain(n, seed):
    """Operands of or_powr_d, the binary64 pow of v1_lp for 1 < p <= 2^17:
    S = pow(Q, p/2) with Q in [0, 1) and C = pow(Z, 1/p) with Z in [1, 2],
    p/2 and 1/p rounded as the tree rounds them; p from the paper's Table 4
    values above 1, the benchmark's, the ends of the range and random ones;
    x drawn plainly, next to 1 on both sides, and with results near the
    flush limit 2^-28."""
    r = random.Random(seed)
    ps = [1.0 + 2.0 ** -40, 1.5, math.sqrt(2), math.e, math.pi, 3.0, 7.5, 64.0, 1000.0, 2.0 ** 17]
    xs, ys = [], []
    while len(xs) < n:
        p = r.choice(ps) if r.random() < 0.5 else math.exp(r.uniform(0.0, 17 * math.log(2)))
        if p == 2.0 or p <= 1.0:
            continue
        h, ip = p * 0.5, 1.0 / p
        kind = len(xs) % 6
        if kind == 0:
            x, y = r.random() ** r.choice([1, 2, 5, 20, 60]), h
        elif kind == 1:
            x, y = 1.0 + r.random(), ip
        elif kind == 2:
            x, y = 1.0 - r.random() * 2.0 ** -r.randint(1, 52), h
        elif kind == 3:
            x, y = 1.0 + r.random() * 2.0 ** -r.randint(1, 52), ip
        elif kind == 4:
            x, y = 2.0 ** (-r.uniform(26.0, 30.0) / h), h
        else:
            x, y = r.uniform(0.0, 1.0) ** r.uniform(0, 60), h
        if x < 0 or x > 2 or x == 1.0:
            continue
        xs.append(x)
        ys.append(y)
    return np.array(xs), np.array(ys)


def test_powr_d_correctly_rounded_on_lp_domains():
    """1.2e5 operand pairs of or_powr_d: RN(x^y) bit for bit wherever x^y
    is more than 2^-8 ulp from a rounding midpoint, within 0.5 + 2^-8 ulp
    everywhere, for results from 2^-28 up; below 2^-28 (down to 2^-28 less
    2^-8 ulp, which may round either way) the result is +0 or below 2^-27,
    so that RN(1 + S^2) = 1 as for the exact S.  Where it is not flushed it
    equals or_pow_d away from the midpoints (both are RN there)."""
    x, y = _powr_domain(120000, seed=53)
    v = oracle.powr_arr(x, y)
    g = oracle.pow_arr(x, y)
    lim = mpmath.ldexp(1, -28)
    checked = decided = flushed = 0
    worst = 0.0
    with mpmath.workprec(PREC):
        for i in range(x.size):
            xi, yi, vi = float(x[i]), float(y[i]), float(v[i])
            ex = mpmath.mpf(xi) ** mpmath.mpf(yi)
            if ex < lim:
                assert vi < 2.0 ** -27 and 1.0 + vi * vi == 1.0, (xi.hex(), yi.hex(), vi)
                flushed += vi == 0.0
                continue
            want, dist, q = _rn(ex, 52, -1022)
            err = _ulp_err(vi, ex, q)
            worst = max(worst, err)
            assert err <= 0.5 + 2.0 ** -8, (xi.hex(), yi.hex(), err)
            checked += 1
            if dist > 2.0 ** -8:
                decided += 1
                assert vi == want, ("not RN(x^y)", xi.hex(), yi.hex(), vi, want, dist)
                assert float(g[i]) == want
    assert checked > 80000 and decided > 0.98 * checked and flushed > 10000
    assert worst > 0.45


def test_powr_d_exact_cases():
    """pow(0, y) = 0 and pow(1, y) = 1; x = 2^a with a y an integer gives
    2^(ay) exactly (u = 0 in the reductions, no series term, t an
    integer); pow(2, y) for y = 2^-k."""
    xs = [0.0, 0.0, 1.0, 1.0, 0.25, 0.5, 0.5, 2.0 ** -10, 2.0, 2.0, 0.125, 2.0 ** -28, 2.0 ** -7]
    ys = [0.75, 2.0 ** 16, 0.75, 2.0 ** -17, 1.5, 3.0, 28.0, 2.5, 1.0, 0.5, 9.0, 1.0, 4.0]
    want = [0.0, 0.0, 1.0, 1.0, 0.125, 0.125, 2.0 ** -28, 2.0 ** -25, 2.0, math.sqrt(2.0), 2.0 ** -27,
            2.0 ** -28, 2.0 ** -28]
    got = oracle.powr_arr(np.array(xs), np.array(ys))
    assert list(got) == want
    # flushed: 2^-29 and below, and x under 2^-60 for any y >= 1/2
    got = oracle.powr_arr(np.array([0.5, 2.0 ** -61, 5e-324, 0.25]), np.array([29.0, 0.5, 0.5, 14.5]))
    assert list(got) == [0.0, 0.0, 0.0, 0.0]


def test_powr_table_matches_its_definition():
    """or_powr_d's Q96 logarithm table, built by the oracle from binary128
    log2, equals RN(log2(2^9 / r1_j) 2^96) (j < 128) or RN(log2(2^8 / r1_j)
    2^96) at 400 bits, entry by entry; its constants D1..D5 are 2^95/ln 2,
    2^63/ln 2, 2^64/(3 ln 2), 2^32/(4 ln 2), 2^32/(5 ln 2) rounded to
    nearest."""
    import re
    from fractions import Fraction
    with mpmath.workprec(400):
        R1 = [512] + [int(Fraction(1 << 18, 513 + 2 * j) + Fraction(1, 2)) for j in range(1, 256)]
        rn = lambda v: int(mpmath.floor(v + mpmath.mpf("0.5")))
        T1q = [rn(mpmath.log(mpmath.mpf(512 if j < 128 else 256) / R1[j], 2) * mpmath.mpf(2) ** 96)
               for j in range(256)]
        ln2 = mpmath.log(2)
        two = mpmath.mpf(2)
        D = [rn(two ** 95 / ln2), rn(two ** 63 / ln2), rn(two ** 64 / (3 * ln2)), rn(two ** 32 / (4 * ln2)),
             rn(two ** 32 / (5 * ln2))]
    assert oracle.powr_table() == T1q
    assert T1q[0] == 0 and T1q[255] == 0
    src = open(oracle._build.SRC).read()
    macro = lambda name: int(re.search(r"#define %s 0x([0-9a-f]+)ull" % name, src).group(1), 16)
    assert (macro("PR_D1H") << 32 | macro("PR_D1L")) == D[0]
    assert [macro("PR_D2"), macro("PR_D3"), macro("PR_D4"), macro("PR_D5")] == D[1:]


def test_powr_pin_catches_a_planted_error():
    """A one-ulp slip on 1 case in 64 of or_powr_d's results fails the
    bitwise check, as for the general pow."""
    x, y = _powr_domain(4000, seed=59)
    v = oracle.powr_arr(x, y)
    idx = [i for i in range(0, v.size, 64) if v[i] != 0.0]
    bad = v.copy()
    bad[idx] = np.nextafter(v[idx], np.inf)
    caught = 0
    with mpmath.workprec(PREC):
        for i in idx:
            ex = mpmath.mpf(float(x[i])) ** mpmath.mpf(float(y[i]))
            want, dist, _ = _rn(ex, 52, -1022)
            if dist > 2.0 ** -8 and float(bad[i]) != want:
                caught += 1
    assert caught > 0.5 * len(idx)


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
