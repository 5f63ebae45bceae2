"""Pins for the C oracle: it is checked against what the paper and the
mathematics fix, never against itself or the CUDA path.

Each test names the passage it pins.  Together they are chosen so that a
plausible slip in the oracle (a dropped term, a wrong sign, a transposed
operand, a wrong split or pairing) fails at least one of them.
"""
import math
import random
import struct

import mpmath
import numpy as np
import pytest

import oracle
from paper_2509_06220_gb300 import inputs
from conftest import golden_rows

EPS_D = 2.0 ** -53
EPS_S = 2.0 ** -24
mpmath.mp.prec = 2300  # exact for sums of squares of any binary64 values


def exact_pnorm(xs, p):
    """Exact-to-2300-bits p-norm of a short list (brute force)."""
    if p == 2:
        s = mpmath.mpf(0)
        for v in xs:
            s += mpmath.mpf(float(v)) ** 2
        return mpmath.sqrt(s)
    if p == 1:
        return sum((abs(mpmath.mpf(float(v))) for v in xs), mpmath.mpf(0))
    if p == math.inf:
        return max(abs(mpmath.mpf(float(v))) for v in xs)
    pp = mpmath.mpf(p)
    s = sum((abs(mpmath.mpf(float(v))) ** pp for v in xs), mpmath.mpf(0))
    return s ** (1 / pp)


def rel(value, exact):
    if exact == 0:
        return 0.0 if value == 0 else math.inf
    return float(abs(mpmath.mpf(float(value)) - exact) / exact)


def ub(depth, prec="D", which="H"):
    hi, lo = oracle.ub_relerr(depth, prec, which)
    return hi + lo


def rng_d(seed, n, emin=-20, emax=20):
    return inputs.vector(n, seed=seed, vec=7, dtype=np.float64, emin=emin, emax=emax)


def rng_s(seed, n, emin=-20, emax=20):
    return inputs.vector(n, seed=seed, vec=7, dtype=np.float32, emin=emin, emax=emax)


def same_bits(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return a.dtype == b.dtype and a.tobytes() == b.tobytes()


# ---------------------------------------------------------------------------
# v1_hypot (Listing 2) and Eq. reH
# ---------------------------------------------------------------------------

def test_k1_special_values():
    """Listing 2: K(a,0) = a, K(0,0) = 0 (Q = fmax(NaN,0) = 0), symmetry, the
    Pythagorean triple 3-4-5 (every step exact), infinities."""
    for dt in (np.float64, np.float32):
        assert oracle.k1(3.0, 4.0, dt) == 5.0
        assert oracle.k1(-4.0, 3.0, dt) == 5.0
        assert oracle.k1(0.0, 0.0, dt) == 0.0
        assert not math.copysign(1.0, float(oracle.k1(-0.0, 0.0, dt))) < 0
        assert math.isinf(oracle.k1(math.inf, 1.0, dt))
        assert math.isinf(oracle.k1(math.inf, math.inf, dt))
        assert math.isinf(oracle.k1(-math.inf, 0.0, dt))
    r = random.Random(1)
    for _ in range(2000):
        a = r.uniform(-1e3, 1e3) * 2.0 ** r.randint(-60, 60)
        b = r.uniform(-1e3, 1e3) * 2.0 ** r.randint(-60, 60)
        assert oracle.k1(a, 0.0) == abs(a)
        assert oracle.k1(0.0, a) == abs(a)
        assert same_bits(oracle.k1(a, b), oracle.k1(b, a))
        assert same_bits(oracle.k1(a, b), oracle.k1(-a, b))
        fa = np.float32(a)
        assert oracle.k1(fa, 0.0, np.float32) == abs(fa)


def test_k1_nan_reading():
    """Listing 2's closing comment: fmin/fmax return the other argument when
    one is a NaN, so K(NaN, y) = |y| sqrt(2)'s rounding and K(NaN, 0) = 0."""
    s2 = math.sqrt(2.0)
    assert oracle.k1(math.nan, 1.0) == s2
    assert oracle.k1(math.nan, 0.0) == 0.0
    assert math.isnan(oracle.k1(math.nan, math.nan))


@pytest.mark.parametrize("dt,eps", [(np.float64, EPS_D), (np.float32, EPS_S)])
def test_k1_within_reH(dt, eps):
    """Eq. reH: the relative error factor of v1_hypot lies strictly between
    (1-eps)^(5/2) sqrt(1 - eps(2-eps)/2) and (1+eps)^(5/2) sqrt(1 + eps(2+eps)/2)."""
    (lo_h, lo_l), (up_h, up_l) = oracle.reH_factors("D" if dt == np.float64 else "S")
    lower = mpmath.mpf(lo_h) + mpmath.mpf(lo_l)
    upper = mpmath.mpf(up_h) + mpmath.mpf(up_l)
    assert float((upper - 1) / eps) == pytest.approx(3.0, rel=1e-6)
    r = random.Random(2)
    worst = 0.0
    for _ in range(4000):
        a = dt(r.uniform(0.5, 2.0) * 2.0 ** r.randint(-30, 30))
        b = dt(r.uniform(0.5, 2.0) * 2.0 ** r.randint(-30, 30))
        h = oracle.k1(a, b, dt)
        ex = mpmath.sqrt(mpmath.mpf(float(a)) ** 2 + mpmath.mpf(float(b)) ** 2)
        f = mpmath.mpf(float(h)) / ex
        assert lower < f < upper
        worst = max(worst, abs(float(f - 1)) / eps)
    assert worst > 0.5  # the check is not vacuous


def test_reH_factors_closed_form():
    """Eq. reH evaluated by the oracle equals the formula evaluated here."""
    for prec, eps in (("D", mpmath.mpf(2) ** -53), ("S", mpmath.mpf(2) ** -24)):
        (lo_h, lo_l), (up_h, up_l) = oracle.reH_factors(prec)
        up = (1 + eps) ** mpmath.mpf(2.5) * mpmath.sqrt(1 + eps * (2 + eps) / 2)
        lo = (1 - eps) ** mpmath.mpf(2.5) * mpmath.sqrt(1 - eps * (2 - eps) / 2)
        assert abs(mpmath.mpf(up_h) + up_l - up) < mpmath.mpf(2) ** -100
        assert abs(mpmath.mpf(lo_h) + lo_l - lo) < mpmath.mpf(2) ** -100


# ---------------------------------------------------------------------------
# Table 3 / Eq. ubr
# ---------------------------------------------------------------------------

def test_table3_bounds():
    """The bound evaluator reproduces the A and H columns of Table 3 for
    n = 2^k, k = 1..30 (depth k), to the 18 printed digits."""
    rows = golden_rows("table3_ub_relerr.txt")
    assert len(rows) == 30
    for k, a_s, h_s in rows:
        k = int(k)
        for which, printed in (("A", a_s), ("H", h_s)):
            hi, lo = oracle.ub_relerr(k, "D", which)
            v = mpmath.mpf(hi) + mpmath.mpf(lo)
            # printed with 18 significant digits: compare to half a unit there
            p = mpmath.mpf(printed)
            assert abs(v - p) <= mpmath.mpf(10) ** (mpmath.floor(mpmath.log10(p)) - 17) * 0.51, (k, which)


# ---------------------------------------------------------------------------
# Tree shape: Eq. r, the Y_D(16,x) example, P = 1, slot form
# ---------------------------------------------------------------------------

def test_eq_r_order_n7():
    """Eq. r: completion order of R_x on 7 elements."""
    kinds = {"leaf1": 1, "leaf2": 2, "node": 3}
    expect = [(kinds[k], int(a), int(b)) for _, k, a, b in golden_rows("eq_r_order_n7.txt")]
    assert oracle.R_trace(7) == expect


def test_R_split_rule():
    """Listing 1: left part ceil(n/2) >= right part; R on n = 3 is
    K(K(x1,x2), |x3|) and n = 5 is K(K(K(x1,x2),|x3|), K(x4,x5))."""
    x = rng_d(3, 5)
    k = oracle.k1
    assert oracle.R(x[:3]) == k(k(x[0], x[1]), abs(x[2]))
    assert oracle.R(x) == k(k(k(x[0], x[1]), abs(x[2])), k(x[3], x[4]))
    assert oracle.R(x[:1]) == abs(x[0])


def test_yd16_lane_grouping():
    """Section 3, Y_D(16, x) with 4 lanes: lane l pairs (x_l, x_{l+4}) and
    (x_{l+8}, x_{l+12})."""
    x = rng_d(4, 16)
    f = oracle.Z(x, 4)
    k = oracle.k1
    for lane, a, b in golden_rows("yd16_lanes.txt"):
        l = int(lane) - 1
        i, j = (int(t) - 1 for t in a.split(","))
        u, v = (int(t) - 1 for t in b.split(","))
        assert f[l] == k(k(x[i], x[j]), k(x[u], x[v]))


def test_head_tail_example_n13_p8():
    """Section 3's n = 13, p = 8 picture: one full vector then a TAIL of 5
    elements padded with zero lanes; lanes >= 5 keep |x_l| alone."""
    x = rng_d(5, 13)
    f = oracle.Z(x, 8)
    k = oracle.k1
    for l in range(8):
        if l < 5:
            assert f[l] == k(x[l], x[8 + l])
        else:
            assert f[l] == k(x[l], 0.0) == abs(x[l])


def test_p1_equals_R():
    """With one lane, Z is R (the vector recursion reduces to Listing 1)."""
    for n in (1, 2, 3, 7, 31, 64, 100, 1000):
        x = rng_d(n, n)
        assert same_bits(oracle.nrm(x, P=1), oracle.R(x))
        xs = rng_s(n, n)
        assert same_bits(oracle.nrm(xs, P=1), oracle.R(xs))


def test_scalar_norm_is_abs():
    """Section 1: the norm of a scalar is |x| (all p, both precisions)."""
    for v in (1.5, -3.25, 2.0 ** -1074, -(2.0 ** 1023), 0.0):
        for p in (2.0, 1.0, 3.0, math.inf):
            assert oracle.nrm(np.array([v])) == abs(v)
            assert oracle.nrm(np.array([v]), p=p) == abs(v)
            assert oracle.nrm(np.array([v], np.float32), p=p) == abs(np.float32(v))


@pytest.mark.parametrize("P", [4, 8, 64])
def test_slot_form_equals_Z_double(P):
    """The slot form (perfect tree, slot j occupied iff brev(j) < m) equals
    Listing 4's recursion bit for bit, for every n up to 40 rows and random
    larger n."""
    ns = list(range(1, 40 * P + 1)) if P < 64 else list(range(1, 4 * P + 1)) + list(range(4 * P, 3000 * 1, 7))
    r = random.Random(P)
    ns += [r.randint(1, 200000) for _ in range(10)]
    base = rng_d(11, max(ns))
    for n in ns:
        x = base[:n]
        for p in (2.0, 1.0):
            assert same_bits(oracle.nrm(x, p, P), oracle.nrm_slot(x, p, P)), (n, p)


@pytest.mark.parametrize("P", [8, 128])
def test_slot_form_equals_Z_single(P):
    r = random.Random(P + 1)
    ns = list(range(1, 3 * P + 2)) + [r.randint(1, 300000) for _ in range(8)]
    base = rng_s(12, max(ns))
    for n in ns:
        x = base[:n]
        for p in (2.0, 3.0):
            assert same_bits(oracle.nrm(x, p, P), oracle.nrm_slot(x, p, P)), (n, p)


def test_lane_width_changes_bits():
    """Section 3: the vectorised results are reproducible only for a fixed
    lane count -- different widths pair the elements differently."""
    x = rng_d(13, 100000)
    vals = {float(oracle.nrm(x, P=P)) for P in (1, 8, 16, 64)}
    assert len(vals) > 1


# ---------------------------------------------------------------------------
# accuracy: brute force, bounds, closed forms
# ---------------------------------------------------------------------------

def test_brute_force_small_n_within_bound():
    """Theorem 3 / Eq. ubr: for n <= 16 the relative error against the exact
    norm is below the bound for the tree's depth (H column closed form)."""
    r = random.Random(5)
    for trial in range(300):
        n = r.randint(1, 16)
        for dt, eps, prec in ((np.float64, EPS_D, "D"), (np.float32, EPS_S, "S")):
            x = inputs.vector(n, seed=trial, vec=n, dtype=dt, emin=-30, emax=30)
            P = oracle.P_D if dt == np.float64 else oracle.P_S
            v = oracle.nrm(x)
            ex = exact_pnorm(x, 2)
            d = oracle.tree_depth(n, P)
            assert rel(v, ex) <= ub(d, prec) * eps, (n, dt)


def test_binary128_reference_vs_mpmath():
    """The binary128 reference agrees with a 2300-bit evaluation."""
    for n in (1, 5, 16, 100, 1000):
        for p in (2.0, 1.0, 3.0, 7.5, math.inf):
            x = rng_d(n + 1, n)
            hi, lo = oracle.ref_q128(x, p)
            ex = exact_pnorm(x, p)
            assert float(abs(mpmath.mpf(hi) + lo - ex) / ex) < 1e-30, (n, p)


def test_config0_accuracy():
    """n = 2^20 binary64 moderately varying data: relerr below the bound for
    depth 20 and (soft, Section 2's observation) below 3 eps."""
    x = inputs.vector(1 << 20, seed=0, vec=0)
    v = oracle.nrm(x)
    e = oracle.relerr(v, x, nthreads=4)
    assert e <= ub(oracle.tree_depth(x.size, 64)) * EPS_D
    assert e <= 3 * EPS_D
    xs = inputs.vector(1 << 20, seed=0, vec=0, dtype=np.float32)
    vs = oracle.nrm(xs)
    es = oracle.relerr(vs, xs, nthreads=4)
    assert es <= ub(oracle.tree_depth(xs.size, 128), "S") * EPS_S
    assert es <= 3 * EPS_S


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_constant_vector_closed_forms(dt):
    """Closed forms on constant vectors c repeated n times:
    p = 2 -> |c| sqrt(n) within the bound; p = 1 and n = 2^k -> n|c| exactly;
    p in {1.5, 3, 7.5}, n = 2^16: each of the 16 levels combines equal values,
    so the result is |c| * C applied 16 times with C = pow(2, 1/p), within
    1e-14 (D) / 5e-6 (S) of |c| n^(1/p)."""
    eps = EPS_D if dt == np.float64 else EPS_S
    prec = "D" if dt == np.float64 else "S"
    tol = 1e-14 if dt == np.float64 else 5e-6
    P = oracle.P_D if dt == np.float64 else oracle.P_S
    for c in (1.0, -3.0, 1.7, 0.1234):
        for n in (1000, 4096, 65536, 100003):
            x = np.full(n, c, dtype=dt)
            v = oracle.nrm(x)
            ex = abs(mpmath.mpf(float(dt(c)))) * mpmath.sqrt(n)
            assert rel(v, ex) <= ub(oracle.tree_depth(n, P), prec) * eps
        for k in (0, 5, 12, 16):
            x = np.full(1 << k, c, dtype=dt)
            assert oracle.nrm(x, p=1.0) == dt(abs(dt(c)) * (1 << k))
        n = 1 << 16
        for p in (1.5, 3.0, 7.5):
            x = np.full(n, c, dtype=dt)
            v = oracle.nrm(x, p=p)
            ex = abs(mpmath.mpf(float(dt(c)))) * mpmath.mpf(n) ** (1 / mpmath.mpf(float(dt(p))))
            assert rel(v, ex) <= tol, (c, p)


def test_scaling_and_sign_invariance():
    """Scaling all entries by 2^k scales the result by exactly 2^k (no
    over/underflow: every step of v1_hypot / v1_lp is scale-free except
    M * s), and sign flips change nothing."""
    x = rng_d(21, 5000)
    xs = rng_s(21, 5000)
    sgn = np.where(np.arange(5000) % 3 == 0, -1.0, 1.0)
    for p in (2.0, 1.0, 3.0, math.inf):
        v = oracle.nrm(x, p)
        for k in (-900, -37, 1, 600, 960):
            assert oracle.nrm(x * 2.0 ** k, p) == v * 2.0 ** k
        assert same_bits(oracle.nrm(x * sgn, p), v)
        vs = oracle.nrm(xs, p)
        for k in (-90, -5, 3, 90):
            assert oracle.nrm(xs * np.float32(2.0 ** k), p) == vs * np.float32(2.0 ** k)
        assert same_bits(oracle.nrm(xs * sgn.astype(np.float32), p), vs)


def test_overflow_probe_small_n():
    """Entries near 2^1020 (D) / 2^125 (S): no undue overflow, the result is
    finite and accurate (a plain sum of squares would overflow)."""
    for n in (2, 5, 16):
        x = inputs.vector(n, seed=n, vec=1, emin=1020, emax=1020)
        assert not np.isfinite(np.sum(x * x))
        v = oracle.nrm(x)
        assert np.isfinite(v)
        assert rel(v, exact_pnorm(x, 2)) <= ub(oracle.tree_depth(n, 64)) * EPS_D
        xs = inputs.vector(n, seed=n, vec=1, dtype=np.float32, emin=125, emax=125)
        vs = oracle.nrm(xs)
        assert np.isfinite(vs)
        assert rel(vs, exact_pnorm(xs, 2)) <= ub(oracle.tree_depth(n, 128), "S") * EPS_S


def test_overflow_to_inf_when_norm_exceeds_range():
    """When the true norm exceeds the format's range, +inf (not NaN)."""
    x = inputs.vector(1 << 12, seed=1, vec=1, emin=1020, emax=1020)
    v = oracle.nrm(x)
    assert math.isinf(v) and v > 0


def test_underflow_probe():
    """Entries in [2^-1022, 2^-1021) (D) / [2^-126, 2^-125) (S): squares
    would underflow, the recursion does not."""
    for n in (3, 16, 1000):
        x = inputs.vector(n, seed=n, vec=2, emin=-1022, emax=-1022)
        assert np.sum(x * x) == 0.0
        v = oracle.nrm(x)
        hi, lo = oracle.ref_q128(x)
        assert abs(v - hi) / hi <= ub(oracle.tree_depth(n, 64)) * EPS_D
        xs = inputs.vector(n, seed=n, vec=2, dtype=np.float32, emin=-126, emax=-126)
        vs = oracle.nrm(xs)
        hs, _ = oracle.ref_q128(xs)
        assert abs(float(vs) - hs) / hs <= ub(oracle.tree_depth(n, 128), "S") * EPS_S


# ---------------------------------------------------------------------------
# v1_lp and the in-repo pow (Listing 5, Section 4)
# ---------------------------------------------------------------------------

def ulp_err(v, ex, dt):
    if ex == 0:
        return 0.0 if v == 0 else math.inf
    e = int(mpmath.floor(mpmath.log(abs(ex), 2)))
    mant = 52 if dt == np.float64 else 23
    emin = -1022 if dt == np.float64 else -126
    u = mpmath.mpf(2) ** (max(e, emin) - mant)
    return float(abs(mpmath.mpf(float(v)) - ex) / u)


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_pow_accuracy(dt):
    """pow(x, y) within 1 ulp of x^y on the two domains v1_lp uses:
    Q in [0,1] with y = p/2 and Z in [1,2] with y = 1/p."""
    r = random.Random(9)
    worst = 0.0
    for _ in range(3000):
        p = r.choice([0.5, 2 / 3, 1.5, math.sqrt(2), math.e, math.pi, 3.0, 7.5, r.uniform(0.5, 20)])
        if r.random() < 0.5:
            x = r.random() ** r.choice([1, 3, 20])
            y = p * 0.5
        else:
            x = 1.0 + r.random()
            y = 1.0 / p
        x, y = dt(x), dt(y)
        v = oracle.pow_(x, y, dt)
        ex = mpmath.mpf(float(x)) ** mpmath.mpf(float(y))
        if dt == np.float32 and ex < mpmath.mpf(2) ** -126:
            continue
        if dt == np.float64 and ex < mpmath.mpf(2) ** -1022:
            continue
        e = ulp_err(v, ex, dt)
        worst = max(worst, e)
    assert worst <= 1.0, worst


def test_pow_exact_cases():
    for dt in (np.float64, np.float32):
        for y in (0.25, 0.5, 1.0, 3.75, 100.0):
            assert oracle.pow_(0.0, y, dt) == 0.0
            assert oracle.pow_(1.0, y, dt) == 1.0
        assert oracle.pow_(2.0, 1.0, dt) == 2.0
        assert oracle.pow_(0.25, 0.5, dt) == 0.5
        assert oracle.pow_(4.0, 1.5, dt) == 8.0
        assert oracle.pow_(0.5, 3.0, dt) == 0.125


def test_pow_constants_are_correctly_rounded():
    """The binary64 pow's fixed-point constants are 2^127/ln 2 and 2^64 ln 2
    rounded to nearest; the binary32 pow's double-word constants ln 2 and
    1/ln 2 are (RN(c), c - RN(c) to 2^-47)."""
    import re
    src = open(oracle._build.SRC).read()

    def macro(name):
        m = re.search(r"#define %s (\S+)" % name, src)
        return m.group(1)

    with mpmath.workprec(400):
        iln2 = int(mpmath.floor(mpmath.mpf(2) ** 127 / mpmath.log(2) + mpmath.mpf("0.5")))
        ln2 = int(mpmath.floor(mpmath.log(2) * mpmath.mpf(2) ** 64 + mpmath.mpf("0.5")))
    hexint = lambda t: int(t.rstrip("ull").rstrip("u"), 16)
    assert (hexint(macro("PW_ILN2_HI")) << 64) | hexint(macro("PW_ILN2_LO")) == iln2
    assert hexint(macro("PW_LN2")) == ln2

    def const(name):
        return float.fromhex(macro(name).rstrip("f"))

    for hi_n, lo_n, c in (("LN2F_HI", "LN2F_LO", mpmath.log(2)), ("ILN2F_HI", "ILN2F_LO", 1 / mpmath.log(2))):
        hi, lo = const(hi_n), const(lo_n)
        assert hi == float(np.float32(float(c))) or abs(mpmath.mpf(hi) - c) <= mpmath.mpf(2) ** -25
        assert np.float32(hi) == hi and np.float32(lo) == lo
        assert abs(mpmath.mpf(hi) + lo - c) < mpmath.mpf(2) ** -47


def _pow_table_definitions():
    """The binary64 pow's tables from their definitions, at 400 bits: the
    first multiplier r1_j = RN(2^18 / (513 + 2 j)) (512 for j = 0), T1_j =
    RN(log2(2^9 / r1_j) 2^88) (j < 128) or RN(log2(2^8 / r1_j) 2^88),
    T2_j2 = RN(-log2(1 - j2 2^-16) 2^96) for j2 = -256..256, TE_i =
    RN(2^(i/256) 2^63)."""
    from fractions import Fraction
    with mpmath.workprec(400):
        two = mpmath.mpf(2)
        rn = lambda v: int(mpmath.floor(v + mpmath.mpf("0.5")))
        R1 = [512] + [int(Fraction(1 << 18, 513 + 2 * j) + Fraction(1, 2)) for j in range(1, 256)]
        T1 = [rn(mpmath.log(mpmath.mpf(512 if j < 128 else 256) / R1[j], 2) * two ** 88) for j in range(256)]
        T2 = [rn(-mpmath.log(1 - mpmath.mpf(k) / 65536, 2) * two ** 96) for k in range(-256, 257)]
        TE = [rn(two ** (mpmath.mpf(i) / 256) * two ** 63) for i in range(256)]
    return R1, T1, T2, TE


def _s128(hi, lo):
    v = int(hi) << 64 | int(lo)
    return v - (1 << 128) if v >> 127 else v


def _oracle_pow_tables():
    import ctypes
    L = oracle.lib()
    f = L.or_pow_tables_d
    f.restype = None
    f.argtypes = [ctypes.c_void_p] * 4
    R1, T1, T2, TE = np.zeros(256, np.uint64), np.zeros(512, np.uint64), np.zeros(2 * 513, np.uint64), \
        np.zeros(256, np.uint64)
    f(R1.ctypes.data, T1.ctypes.data, T2.ctypes.data, TE.ctypes.data)
    return ([int(v) for v in R1], [_s128(T1[2 * j], T1[2 * j + 1]) for j in range(256)],
            [_s128(T2[2 * k], T2[2 * k + 1]) for k in range(513)], [int(v) for v in TE])


def test_pow_tables_match_their_definitions():
    """The oracle builds the binary64 pow's tables itself (binary128 log2
    and pow); every entry equals the 400-bit value rounded to nearest.
    T1_0 = T1_255 = 0 and T2_0 = 0: no cancellation next to x = 1."""
    R1, T1, T2, TE = _pow_table_definitions()
    assert _oracle_pow_tables() == (R1, T1, T2, TE)
    assert T1[0] == 0 and T1[255] == 0 and T2[256] == 0 and R1[255] == 256 and TE[0] == 1 << 63


def test_pow_reduction_bounds():
    """The two short multipliers of the reduction, over every significand
    bucket (its ends and random interior points): M r1_j is exact in 64
    bits, |u1| <= 2^-8, |j2| <= 256 (the T2 table's range), and u2 is exact
    in Q77 with |u2| < 2^-15.4 (the log series' range)."""
    R1 = _pow_table_definitions()[0]
    r = random.Random(12)
    for j in range(256):
        lo = (1 << 52) + (j << 44)
        for M in [lo, lo + (1 << 44) - 1] + [r.randrange(lo, lo + (1 << 44)) for _ in range(200)]:
            P1 = M * R1[j]
            assert P1 < 1 << 62
            U1 = P1 - (1 << 61)
            assert abs(U1) <= 1 << 53
            j2 = (U1 + (1 << 44)) >> 45
            assert abs(j2) <= 256
            U2 = ((U1 - j2 * (1 << 45)) << 16) - U1 * j2
            assert U2 == (M * R1[j] * (65536 - j2) << 0) - (1 << 77)  # (1 + u1)(1 - j2 2^-16) - 1 exactly
            assert abs(U2) < 2 ** 61.6


def test_kernel_pow_tables_match_the_definitions():
    """The kernels' copy of the tables (paper_2509_06220_gb300/csrc/
    nrm_pow_tables.h, written by gen_pow_tables.py beside it) holds the same
    values as the definitions, and its constants 2^127/ln 2 and 2^64 ln 2."""
    import os
    import re
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2509_06220_gb300",
                        "csrc", "nrm_pow_tables.h")
    src = open(path).read()

    def block(name, pattern=r"0x([0-9a-f]+)ull", base=16):
        body = src[src.index(name):]
        body = body[body.index("{") + 1:body.index("};")]
        return [int(v, base) for v in re.findall(pattern, body)]

    R1, T1, T2, TE = _pow_table_definitions()
    assert block("kPowR1[256]", r"(\d+),", 10) == R1
    t1 = block("kPowT1[256][2]")
    t2 = block("kPowT2[513][2]")
    assert [_s128(t1[2 * j], t1[2 * j + 1]) for j in range(256)] == T1
    assert [_s128(t2[2 * k], t2[2 * k + 1]) for k in range(513)] == T2
    assert block("kPowTE[256]") == TE
    with mpmath.workprec(400):
        iln2 = int(mpmath.floor(mpmath.mpf(2) ** 127 / mpmath.log(2) + mpmath.mpf("0.5")))
        ln2 = int(mpmath.floor(mpmath.log(2) * mpmath.mpf(2) ** 64 + mpmath.mpf("0.5")))
    const = lambda name: int(re.search(r"%s = 0x([0-9a-f]+)u" % name, src).group(1), 16)
    assert (const("kPowILN2_HI") << 64 | const("kPowILN2_LO")) == iln2 and const("kPowLN2") == ln2
    # the restricted pow of v1_lp (1 < p <= 2^17): T1 in Q96 and the series constants
    with mpmath.workprec(400):
        two, l2 = mpmath.mpf(2), mpmath.log(2)
        rn = lambda v: int(mpmath.floor(v + mpmath.mpf("0.5")))
        T1q = [rn(mpmath.log(mpmath.mpf(512 if j < 128 else 256) / R1[j], 2) * two ** 96) for j in range(256)]
        D = [rn(two ** 95 / l2), rn(two ** 63 / l2), rn(two ** 64 / (3 * l2)), rn(two ** 32 / (4 * l2)),
             rn(two ** 32 / (5 * l2))]
    t1q = block("kPowT1Q96[256][2]")
    assert [_s128(t1q[2 * j], t1q[2 * j + 1]) for j in range(256)] == T1q
    assert (const("kPrD1H") << 32 | const("kPrD1L")) == D[0]
    assert [const("kPrD2"), const("kPrD3"), const("kPrD4"), const("kPrD5")] == D[1:]


def _bits_d(v):
    return struct.unpack("<d", struct.pack("<Q", v))[0]


def test_pow_d_nearly_correctly_rounded_wide():
    """The fixed-point binary64 pow stays within 0.6 ulp of x^y (0.5 is the
    rounding itself) on the wider domain: x near 1 with large y, subnormal x,
    |y log2 x| up to 1100 (results near the overflow and subnormal limits),
    and arbitrary bit patterns; results that overflow are +inf and those
    below 2^-1075 are +0."""
    r = random.Random(21)
    worst = 0.0
    with mpmath.workprec(300):
        for i in range(4000):
            kind = i % 6
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
            v = float(oracle.pow_(x, y))
            ex = mpmath.mpf(x) ** mpmath.mpf(y)
            if ex >= mpmath.mpf(2) ** 1024:
                assert v == math.inf, (x, y)
                continue
            if ex < mpmath.mpf(2) ** -1075:
                assert v == 0.0, (x, y)
                continue
            e = int(mpmath.floor(mpmath.log(ex, 2)))
            u = mpmath.mpf(2) ** (max(e, -1022) - 52)
            err = float(abs(mpmath.mpf(v) - ex) / u)
            worst = max(worst, err)
            assert err <= 0.6, (x.hex(), y.hex(), err)
    assert worst > 0.4  # the sample reaches the rounding error itself


def test_pow_d_exact_powers_of_two():
    """pow(2^a, b) = 2^(ab) exactly whenever ab is an integer (step 7 then has
    r = 0), including the subnormal results, the tie 2^-1075 -> +0 (to even),
    and the overflow 2^1024 -> +inf; pow(x, 0) = 1; pow(x, inf) = 0 or inf."""
    for a in range(-1074, 1024, 7):
        for b in (1.0, 0.5, 2.0, 0.25, 3.0):
            ab = a * b
            if ab != int(ab):
                continue
            want = math.ldexp(1.0, int(ab)) if -1074 <= ab <= 1023 else (0.0 if ab < -1074 else math.inf)
            assert float(oracle.pow_(math.ldexp(1.0, a), b)) == want, (a, b)
    assert float(oracle.pow_(0.5, 1074.0)) == 5e-324
    assert float(oracle.pow_(0.5, 1075.0)) == 0.0
    assert float(oracle.pow_(2.0, 1023.0)) == 2.0 ** 1023
    assert float(oracle.pow_(2.0, 1024.0)) == math.inf
    for x in (1e-300, 0.3, 1.7, 1e300):
        assert float(oracle.pow_(x, 0.0)) == 1.0
        assert float(oracle.pow_(x, math.inf)) == (0.0 if x < 1 else math.inf)


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_lp_combine_brute_force(dt):
    """Eq. sp: v1_lp(x, y) ~ (|x|^p + |y|^p)^(1/p) to a few ulps; p = 2 via
    Listing 5 differs from v1_hypot by at most a few ulps; v1_lp(a, 0) = a."""
    r = random.Random(10)
    eps = EPS_D if dt == np.float64 else EPS_S
    for _ in range(1500):
        p = r.choice([0.5, 1.5, 3.0, 7.5, math.pi])
        a = dt(r.uniform(0.5, 2) * 2.0 ** r.randint(-20, 20))
        b = dt(r.uniform(-2, 2) * 2.0 ** r.randint(-20, 20))
        v = oracle.lp(p, a, b, dt)
        pp = mpmath.mpf(float(dt(p)))
        ex = (abs(mpmath.mpf(float(a))) ** pp + abs(mpmath.mpf(float(b))) ** pp) ** (1 / pp)
        assert rel(v, ex) <= 6 * eps, (p, a, b)
        assert oracle.lp(p, a, 0.0, dt) == abs(a)


@pytest.mark.parametrize("p", [1.0, 1.5, 3.0, 7.5, 0.5, math.inf])
def test_pnorm_against_binary128(p):
    """xNRMP on moderately varying data (e in [-8, 8], the p-norm workload)
    against the binary128 reference: D within 1e-14, S within 5e-6; the D
    error is of the magnitude of Table 4 (a few eps)."""
    x = inputs.vector(1 << 16, seed=3, vec=4, emin=-8, emax=8)
    v = oracle.nrm(x, p)
    e = oracle.relerr(v, x, p, nthreads=4)
    assert e <= 1e-14
    assert e <= 8 * EPS_D
    xs = inputs.vector(1 << 16, seed=3, vec=4, dtype=np.float32, emin=-8, emax=8)
    vs = oracle.nrm(xs, p)
    assert oracle.relerr(vs, xs, p, nthreads=4) <= 5e-6


def test_table4_magnitude_soft():
    """Table 4 reports max relerr between 1.25 and 4.2 eps for p in
    {1/2, 2/3, 1, sqrt 2, e, pi}; ours is of the same magnitude (< 10 eps)."""
    x = inputs.vector(1 << 18, seed=4, vec=5, emin=-8, emax=8)
    for row in golden_rows("table4_pnorm_relerr.txt"):
        p = float(row[0])
        e = oracle.relerr(oracle.nrm(x, p), x, p, nthreads=4) / EPS_D
        assert e < 10.0, (p, e)


def test_nrm_batch_matches_single():
    x, off = inputs.ragged_batch(40, seed=1, max_log2=12)
    out = oracle.nrm_batch(x, off)
    for i in range(40):
        assert out[i] == oracle.nrm(x[off[i]:off[i + 1]])


def test_empty_is_zero():
    """n = 0: +0 (Listing 1 assumes n > 0; +0 is the norm of the empty array)."""
    assert oracle.nrm(np.zeros(0)) == 0.0
    assert oracle.nrm(np.zeros(0, np.float32)) == 0.0


@pytest.mark.parametrize("dt,cut", [(np.float64, 2.0 ** 53), (np.float32, 2.0 ** 24)])
def test_pow_cutoff_p_prime(dt, cut):
    """Section 4's cut-off p': the smallest p with pow(z, 1/p) = 1 for all z
    in [1, 2] lies in (2^52, 2^53] (binary64) and (2^23, 2^24] (binary32),
    the ranges the paper reports for cr_pow / cr_powf; at the cut-off power
    of two v1_lp returns max(|x|, |y|) bit for bit (so xNRMP may switch to
    the p = inf code), below it it does not."""
    one = dt(1.0)
    two = dt(2.0)

    def is_one(p):
        return oracle.pow_(two, one / dt(p), dt) == 1.0

    assert not is_one(cut / 2) and is_one(cut)
    lo, hi = cut / 2, cut  # bisection on the smallest p with pow(2, 1/p) = 1
    for _ in range(80):
        mid = dt((lo + hi) / 2)
        if mid <= lo or mid >= hi:
            break
        if is_one(mid):
            hi = float(mid)
        else:
            lo = float(mid)
    assert cut / 2 < hi <= cut
    r = random.Random(11)
    zs = [dt(1 + r.random()) for _ in range(2000)] + [dt(2.0), dt(1.0), np.nextafter(dt(2.0), dt(0))]
    assert all(oracle.pow_(z, one / dt(cut), dt) == 1.0 for z in zs)
    diff_below = 0
    for _ in range(3000):
        a = dt(r.uniform(0.5, 2) * 2.0 ** r.randint(-30, 30))
        b = dt(r.uniform(-2, 2) * 2.0 ** r.randint(-30, 30))
        assert oracle.lp(cut, a, b, dt) == max(abs(a), abs(b))
        assert oracle.lp(cut * 64, a, b, dt) == max(abs(a), abs(b))
        assert oracle.lp(cut, a, -a, dt) == abs(a)
        # below the cut-off, Q^(p/2) vanishes unless |x| = |y|; there Z = 2
        # and pow(2, 1/p) > 1
        diff_below += oracle.lp(cut / 4, a, -a, dt) != abs(a)
    assert diff_below > 2000
    x = inputs.vector(5000, seed=12, vec=3, dtype=dt)
    assert oracle.nrm(x, cut) == oracle.nrm(x, math.inf) == np.max(np.abs(x))


def test_strided_and_matrix_definitions():
    """Section 3 (incx) and Section 3.1 (leading dimension): a strided vector
    is its logical vector (incx < 0 taken backwards); a matrix with lda == M
    is the one vector of M N elements; with lda > M the column norms are
    combined by the same tree, and the result is accurate within the bound of
    the two stacked trees against binary128 over all M N elements."""
    x = rng_d(40, 100000)
    assert same_bits(oracle.nrm_strided(x, 100000, 1), oracle.nrm(x))
    assert same_bits(oracle.nrm_strided(x, 33333, 3), oracle.nrm(x[::3][:33333]))
    assert same_bits(oracle.nrm_strided(x, 25000, -4), oracle.nrm(x[:100000:4][::-1][-25000:][:25000]))
    assert same_bits(oracle.nrm_strided(x, 1000, -1), oracle.nrm(x[:1000][::-1]))
    M, N, lda = 3000, 20, 3100
    A = x[:N * lda]
    cols = [A[j * lda:j * lda + M] for j in range(N)]
    v = oracle.nrm_matrix(A, M, N, lda)
    c = np.array([oracle.nrm(cc) for cc in cols])
    assert same_bits(v, oracle.nrm(c))
    allv = np.concatenate(cols)
    hi, lo = oracle.ref_q128(allv)
    depth = oracle.tree_depth(M, 64) + oracle.tree_depth(N, 64)
    assert abs(float(v) - hi) / hi <= ub(depth) * EPS_D
    assert same_bits(oracle.nrm_matrix(A, M, N, M), oracle.nrm(A[:M * N]))
    for p in (1.0, 3.0, math.inf):
        vp = oracle.nrm_matrix(A, M, N, lda, p)
        hi, _ = oracle.ref_q128(allv, p)
        assert abs(float(vp) - hi) / hi <= 1e-14


def test_complex_as_reals():
    """Section 1: |z|^2 = Re^2 + Im^2, so a complex array's Frobenius norm is
    the norm of its interleaved real parts (accurate against the exact
    sum of |z_i|^2)."""
    re = rng_d(41, 5000)
    im = rng_d(42, 5000)
    inter = np.empty(10000)
    inter[0::2], inter[1::2] = re, im
    v = oracle.nrm(inter)
    ex = mpmath.sqrt(sum(mpmath.mpf(float(a)) ** 2 + mpmath.mpf(float(b)) ** 2 for a, b in zip(re, im)))
    assert rel(v, ex) <= ub(oracle.tree_depth(10000, 64)) * EPS_D


def _exact_rn_hypot(x, y, dt):
    """RN(sqrt(x^2 + y^2)) in format dt, decided exactly: candidates from a
    high-precision estimate, then exact rational comparisons with the
    midpoints (ties to even)."""
    from fractions import Fraction
    S = Fraction(float(x)) ** 2 + Fraction(float(y)) ** 2
    est = mpmath.sqrt(mpmath.mpf(float(x)) ** 2 + mpmath.mpf(float(y)) ** 2)
    c = dt(float(est))
    if not np.isfinite(c):
        return c
    cands = sorted({c, np.nextafter(c, dt(np.inf)), np.nextafter(c, dt(0)),
                    np.nextafter(np.nextafter(c, dt(0)), dt(0))}, key=float)
    best = None
    for v in cands:
        lo = Fraction(float(np.nextafter(v, dt(0)))) if v > 0 else Fraction(0)
        hi = Fraction(float(np.nextafter(v, dt(np.inf))))
        mlo, mhi = (lo + Fraction(float(v))) / 2, (hi + Fraction(float(v))) / 2
        below = mlo * mlo < S or (mlo * mlo == S and int(np.asarray(v).view(np.uint64 if dt == np.float64 else np.uint32)) % 2 == 0)
        above = S < mhi * mhi or (S == mhi * mhi and int(np.asarray(v).view(np.uint64 if dt == np.float64 else np.uint32)) % 2 == 0)
        if below and above:
            best = v
    return best


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_cr_hypot_is_correctly_rounded(dt):
    """Section 2: A uses a correctly rounded hypot (|eps_h| <= eps).  The
    oracle's cr_hypot equals RN(sqrt(x^2 + y^2)) decided exactly, on random
    pairs with every exponent gap around the shortcut threshold, subnormals,
    exact Pythagorean triples (3-4-5 scaled) and near-ties."""
    r = random.Random(17)
    big = 1000 if dt == np.float64 else 120
    small = -1070 if dt == np.float64 else -148
    thr = 28 if dt == np.float64 else 14
    cases = [(3.0, 4.0), (5.0, 12.0), (1.0, 1.0), (0.0, 2.5), (np.finfo(dt).tiny, np.finfo(dt).tiny),
             (np.finfo(dt).smallest_subnormal, np.finfo(dt).smallest_subnormal)]
    for _ in range(3000):
        e = r.randint(small, big)
        g = r.choice([0, 0, 1, 2, thr - 2, thr - 1, thr, thr + 1, r.randint(0, 2 * thr)])
        cases.append(((1 + r.random()) * 2.0 ** e, (1 + r.random()) * 2.0 ** (e - g)))
    for _ in range(300):
        m, n = r.randint(1, 2 ** 11), r.randint(1, 2 ** 11)
        k = r.randint(-40, 40)
        cases.append(((m * m - n * n) * 2.0 ** k, (2 * m * n) * 2.0 ** k))
    checked = 0
    for a, b in cases:
        a, b = dt(a), dt(b)
        if not (np.isfinite(a) and np.isfinite(b)):
            continue
        want = _exact_rn_hypot(a, b, dt)
        if want is None:
            continue
        got = oracle.cr_hypot(a, b, dt)
        assert same_bits(np.asarray(got, dt), np.asarray(want, dt)), (a, b, got, want)
        checked += 1
    assert checked > 3000
    assert oracle.cr_hypot(3.0, 4.0, dt) == 5.0


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_za_variant(dt):
    """Section 3's recommendation: Z with A for the final reduction.  It is
    accurate within Theorem 3's bound with the v1_hypot factor (Eq. reH) on
    the vector-row levels and eps' = eps on the lane levels, and equals the
    H form when only one lane is nonzero."""
    P = oracle.P_D if dt == np.float64 else oracle.P_S
    eps = EPS_D if dt == np.float64 else EPS_S
    prec = "D" if dt == np.float64 else "S"
    x = inputs.vector(1 << 18, seed=50, vec=0, dtype=dt)
    v = oracle.nrm_za(x)
    hi, lo = oracle.ref_q128(x)
    rows = oracle.tree_depth(x.size, P) - int(math.log2(P))
    (_, _), (uh, ul) = oracle.reH_factors(prec)
    bound = ((mpmath.mpf(uh) + ul) ** rows * (1 + mpmath.mpf(eps)) ** int(math.log2(P)) - 1)
    assert abs(float(v) - hi) / hi <= float(bound)
    one = np.zeros(5 * P, dtype=dt)
    one[7] = dt(-2.5)
    assert oracle.nrm_za(one) == oracle.nrm(one) == dt(2.5)
    assert oracle.nrm_za(np.zeros(0, dt)) == 0.0


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_nan_operand_is_missing_data(dt):
    """Listings 2 and 5 take m = fmin(X, Y) and M = fmax(X, Y); C's Annex F
    has these treat a NaN argument as missing data, so v1_hypot(NaN, a) =
    v1_hypot(a, a), v1_lp(NaN, a) = v1_lp(a, a) and max(|NaN|, |a|) = |a|,
    for quiet and signalling NaNs alike (checked through the array entry
    points, which keep a signalling NaN's bits)."""
    ui = np.uint64 if dt == np.float64 else np.uint32
    qnan, snan = (0x7FF8000000000001, 0x7FF0000000000001) if dt == np.float64 else (0x7FC00001, 0x7F800001)
    a = np.array([3.0, 1e-30, 0.0, 7.5], dt)
    for nb in (qnan, snan):
        nan = np.full(a.shape, nb, ui).view(dt)
        assert np.isnan(nan).all()
        for p in (0.5, 3.0, 7.5):
            assert same_bits(oracle.lp_arr(p, nan, a), oracle.lp_arr(p, a, a))
            assert same_bits(oracle.lp_arr(p, a, nan), oracle.lp_arr(p, a, a))
        x = np.concatenate([nan[:1], a[:1]])
        assert oracle.nrm(x, math.inf) == a[0]
        assert oracle.nrm(x, 2.0) == oracle.nrm(a[:1].repeat(2), 2.0)


# ---------------------------------------------------------------------------
# the exponent-scaled hypotenuse K2 (a division-free hypot[f], Section 2)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_k2_exact_cases_and_symmetry(dt):
    """K2(a, 0) = |a| exactly (sqrt(RN(a^2)) = |a|), K2(0, 0) = 0, K2 is
    symmetric and sign-blind, inf gives inf, a NaN is missing data."""
    r = random.Random(31)
    info = np.finfo(dt)
    vals = [dt(r.uniform(1, 2) * 2.0 ** r.randint(int(info.minexp) - 20, int(info.maxexp) - 1)) for _ in range(3000)]
    vals += [info.max, info.tiny, info.smallest_subnormal, dt(1), dt(3)]
    for v in vals:
        assert oracle.k2(v, 0, dt) == abs(v), v
        assert oracle.k2(0, -v, dt) == abs(v), v
    assert oracle.k2(0, 0, dt) == 0
    for _ in range(2000):
        a = dt(r.uniform(-2, 2) * 2.0 ** r.randint(-30, 30))
        b = dt(r.uniform(-2, 2) * 2.0 ** r.randint(-30, 30))
        v = oracle.k2(a, b, dt)
        assert v == oracle.k2(b, a, dt) == oracle.k2(-a, b, dt) == oracle.k2(a, -b, dt)
    assert math.isinf(oracle.k2(np.inf, 1.0, dt))
    x = np.array([np.nan, 3.0, 1e-30], dt)
    y = np.array([3.0, np.nan, np.nan], dt)
    assert same_bits(oracle.k2_arr(x, y), oracle.k2_arr(np.array([3.0, 3.0, 1e-30], dt), np.array([3.0, 3.0, 1e-30], dt)))


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_k2_accuracy_monotone_and_scaling(dt):
    """|K2(x, y) - hypot(x, y)| <= 1.75 eps (1 + 2^-20) hypot(x, y) against
    mpmath when nothing underflows; K2 is non-decreasing in |x| (and |y|);
    K2(2^j x, 2^j y) = 2^j K2(x, y) while nothing over- or underflows; the
    largest finite pairs stay finite when the hypotenuse fits."""
    r = random.Random(32)
    eps = EPS_D if dt == np.float64 else EPS_S
    worst = 0.0
    with mpmath.workprec(300):
        for _ in range(4000):
            a = dt(r.uniform(1, 2) * 2.0 ** r.randint(-60, 60))
            b = dt(r.uniform(1, 2) * 2.0 ** (math.floor(math.log2(a)) - r.choice([0, 0, 1, 2, 5, 12, 30])))
            v = oracle.k2(a, b, dt)
            ex = mpmath.sqrt(mpmath.mpf(float(a)) ** 2 + mpmath.mpf(float(b)) ** 2)
            e = float(abs(mpmath.mpf(float(v)) - ex) / ex)
            worst = max(worst, e)
            assert e <= 1.75 * eps * (1 + 2.0 ** -20), (a, b, e / eps)
            a2 = np.nextafter(a, dt(np.inf))
            assert oracle.k2(a2, b, dt) >= v
            assert oracle.k2(a, np.nextafter(b, dt(np.inf)), dt) >= v
            j = r.randint(-20, 20)
            assert oracle.k2(a * dt(2.0 ** j), b * dt(2.0 ** j), dt) == v * dt(2.0 ** j)
    assert worst > 0.5 * eps
    big = np.finfo(dt).max
    assert math.isfinite(oracle.k2(big / dt(2), big / dt(2), dt))
    assert math.isinf(oracle.k2(big, big, dt))


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_nrm_es_against_binary128(dt):
    """xNRMF with K2 in the whole tree: a scalar's norm is |x|; on moderately
    varying data (n = 2^16 and 5000) the error against the binary128
    reference is within ((1 + 1.75 eps')^depth - 1) with eps' = eps (1 +
    2^-20), the depth of the tree (ceil(lg m) + lg P levels); c repeated n
    times gives |c| sqrt(n) within the same bound."""
    eps = EPS_D if dt == np.float64 else EPS_S
    P = 64 if dt == np.float64 else 128
    for v in (dt(3.5), dt(-1e-30), dt(7e20)):
        assert oracle.nrm_es(np.array([v], dt)) == abs(v)
    for n in (5000, 1 << 16):
        x = inputs.vector(n, seed=33, vec=n % 7, dtype=dt)
        v = oracle.nrm_es(x)
        depth = oracle.tree_depth(n, P)
        bound = (1 + 1.75 * eps * (1 + 2.0 ** -20)) ** depth - 1
        e = oracle.relerr(v, x, 2.0, nthreads=4)
        assert e <= bound, (n, e, bound)
    c = dt(1.7)
    n = 1 << 14
    v = float(oracle.nrm_es(np.full(n, c, dt)))
    bound = (1 + 1.75 * eps * (1 + 2.0 ** -20)) ** oracle.tree_depth(n, P) - 1
    assert abs(v - 1.7 * math.sqrt(n)) <= bound * 1.7 * math.sqrt(n) + 1.7 * math.sqrt(n) * eps


def test_thread_driver_is_bitwise_the_serial_tree():
    """The oracle's all-cores driver (the top splits of Listing 4's recursion
    evaluated on separate threads) gives the serial oracle's bits for every
    thread count, length and combine."""
    r = random.Random(77)
    for trial in range(24):
        n = r.choice([1, 2, 63, 64, 65, 129, 1000, 12345, 1 << 16, (1 << 18) + 7, r.randint(1, 400000)])
        dt = np.float64 if trial % 2 == 0 else np.float32
        p = r.choice([2.0, 1.0, 3.0, 1.5, math.inf])
        x = inputs.vector(n, seed=trial, vec=1, dtype=dt)
        want = oracle.nrm(x, p)
        for t in (1, 2, 3, 8, 16):
            got = oracle.nrm_par(x, p, threads=t)
            assert got.tobytes() == want.tobytes(), (n, dt, p, t)
