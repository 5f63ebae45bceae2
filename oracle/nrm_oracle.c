/*
 * nrm_oracle.c -- plain, slow, serial C oracle for xNRMF / xNRMP
 * (Novakovic, "Recursive vectorized computation of the vector p-norm",
 * arXiv 2509.06220).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the tests, the smoke check and the benchmark's CPU
 * baseline leg do.  It shares no code with the CUDA library: every formula
 * below is written out again here from the paper.
 *
 * Build: C11, -O2 -ffp-contract=off, no fast-math, no FTZ.  With contraction
 * off every C arithmetic operator below is one IEEE-754 binary64/binary32
 * operation rounded to nearest-even, and fma() is the only fused operation,
 * which is what Section 1 assumes ("rounding to nearest") and what the
 * one-statement-one-instruction reading of Listing 2 requires.
 *
 * What is here (each function cites the passage it follows):
 *   or_k1_d / or_k1_s      v1_hypot, Listing 2 (Section 2)
 *   or_lp_d / or_lp_s      v1_lp, Listing 5 (Section 4, Eqs. sp and qp)
 *   sumabs / maxabs        Eqs. vp1 and vpI (Section 4)
 *   or_pow_d / or_pow_s    the pow[f] that v1_lp needs (Section 4 leaves the
 *                          choice open); written here from the textbook
 *                          identities x^y = 2^(y log2 x), ln f = 2 atanh(s),
 *                          s = (f-1)/(f+1), and the Taylor series of atanh
 *                          and exp: binary64 in exact fixed-point integer
 *                          arithmetic, binary32 with double-word (Dekker)
 *                          arithmetic.
 *   or_powr_d              the binary64 pow of v1_lp for 1 < p <= 2^17,
 *                          restricted to its two operand ranges (log2 x in
 *                          plain Q96 fixed point, results below 2^-28 as 0)
 *   or_R_*                 R_x, Listing 1 / Eq. r (Section 2)
 *   or_Z_*                 Z_x generalised to p lanes, Listing 4 (Section 3)
 *   or_nrm_*               xNRMF / xNRMP = Z then a final R over the lanes
 *                          (Section 3, recommendation for xNRMF)
 *   or_nrm_par_*           the same on several threads (the top splits of
 *                          Z evaluated concurrently, bitwise equal; used
 *                          only to time the oracle on all host cores)
 *   or_cr_hypot_*          the correctly rounded hypot of the algorithm A
 *                          (Section 2), from its definition with integers
 *   or_nrm_za_*            Z then A for the final reduction (Section 3's
 *                          recommendation for xNRMF)
 *   or_k2_* / or_nrm_es_*  the exponent-scaled hypotenuse K2 (a division-
 *                          free hypot[f] admitted by Section 2) and xNRMF
 *                          with it in place of v1_hypot
 *   or_nrm_strided_*       a strided vector (BLAS incx, Section 3)
 *   or_nrm_matrix_*        a matrix with a leading dimension (Section 3.1)
 *   or_nrm_slot_*          the same tree evaluated in "slot form" (a perfect
 *                          tree whose empty slots are skipped); a second,
 *                          independent evaluation used to pin or_nrm_*
 *   or_ref_q128            binary128 reference norm (stands in for the
 *                          2048-bit MPFR reference of Section 2, Eq. relerr)
 *   or_ub_relerr           closed-form upper bound of Eq. ubr / Table 3
 *
 * Parity status: every function here is pinned by the tests under tests/
 * (see test_oracle_pins.py); none is "parity unpinned".
 */
#define _GNU_SOURCE
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#if defined(__aarch64__)
typedef long double q128; /* IEEE binary128 on AArch64 Linux */
#define Q_SQRT sqrtl
#define Q_POW powl
#define Q_FABS fabsl
#define Q_LOG2 log2l
#define Q_FLOOR floorl
#elif defined(__x86_64__)
#include <quadmath.h>
typedef __float128 q128;
#define Q_SQRT sqrtq
#define Q_POW powq
#define Q_FABS fabsq
#define Q_LOG2 log2q
#define Q_FLOOR floorq
#else
#error "binary128 reference needs AArch64 long double or x86-64 __float128"
#endif

#define OR_API __attribute__((visibility("default")))

/* ------------------------------------------------------------------------ */
/* combine operations                                                        */
/* ------------------------------------------------------------------------ */

static inline uint64_t bits_d(double x);
static inline double from_bits_d(uint64_t u);
static inline uint32_t bits_s(float x);
static inline float from_bits_s(uint32_t u);

/* Combine op selector: which per-node operation the tree applies. */
enum { OP_HYPOT = 0, OP_LP = 1, OP_SUMABS = 2, OP_MAXABS = 3, OP_K2 = 4 };

/* fmin / fmax of Listings 2 and 5 with C's Annex F rule written out: a NaN
 * argument counts as missing data and the other one is returned.  The rule
 * is applied to signalling NaNs too (some libms return a NaN for those,
 * e.g. one built on AArch64's FMINNM), so that the result does not depend
 * on the host's libm. */
static double min_d(double a, double b) { return isnan(a) ? b : isnan(b) ? a : (b < a ? b : a); }
static double max_d(double a, double b) { return isnan(a) ? b : isnan(b) ? a : (b > a ? b : a); }
static float min_s(float a, float b) { return isnan(a) ? b : isnan(b) ? a : (b < a ? b : a); }
static float max_s(float a, float b) { return isnan(a) ? b : isnan(b) ? a : (b > a ? b : a); }

/* v1_hypot (the algorithm of Listing 2, Section 2): the hypotenuse written
 * as big sqrt(1 + (small/big)^2) with big = max(|x|, |y|) and small =
 * min(|x|, |y|), so that no square of an input is formed; each of its
 * operations -- the ratio, the guard that makes a NaN ratio (0/0, inf/inf)
 * count as 0, the fused 1 + r^2, the square root and the product -- is one
 * IEEE operation rounded to nearest.  min/max treat a NaN as missing data,
 * which makes K(a, 0) = a and K(0, 0) = 0 exact. */
OR_API double or_k1_d(double x, double y)
{
    const double ax = fabs(x), ay = fabs(y);
    const double big = max_d(ax, ay), small = min_d(ax, ay);
    double r = small / big;
    r = max_d(r, 0.0);
    const double root = sqrt(fma(r, r, 1.0));
    return big * root;
}

/* The binary32 form (Section 2: the S routines use float and the
 * f-suffixed functions). */
OR_API float or_k1_s(float x, float y)
{
    const float ax = fabsf(x), ay = fabsf(y);
    const float big = max_s(ax, ay), small = min_s(ax, ay);
    float r = small / big;
    r = max_s(r, 0.0f);
    const float root = sqrtf(fmaf(r, r, 1.0f));
    return big * root;
}

/* 2^e as a double (binary32: a float) for e in [-1074, 1023] ([-149, 127]),
 * built from its bit pattern. */
static double p2_d(int e)
{
    if (e >= -1022) return from_bits_d((uint64_t)(e + 1023) << 52);
    return from_bits_d(1ull << (e + 1074));
}

static float p2_s(int e)
{
    if (e >= -126) return from_bits_s((uint32_t)(e + 127) << 23);
    return from_bits_s(1u << (e + 149));
}

/*
 * K2: the exponent-scaled hypotenuse, a division-free hypot[f] for the tree
 * (Section 2 admits any hypot that avoids undue overflow and underflow, is
 * monotone in |x| and |y| and accurate to a small multiple of eps; this is
 * the variant the scope lists next to A).  With m = min(|x|,|y|), M = max
 * (a NaN is missing data, as in v1_hypot) and k the binade of M (k = emin
 * for a subnormal M):
 *   a = M 2^-k (exact), b = RN(m 2^-k), S = RN(fma(a, a, RN(b b))),
 *   s = RN(sqrt(S)), K2 = RN(s 2^k);
 * M = 0 gives +0, M = inf gives +inf, two NaNs give a NaN.  Each step is one
 * IEEE operation rounded to nearest; K2(a, 0) = |a| exactly (sqrt(RN(a^2))
 * = |a|), and the relative error is at most 1.75 eps + O(eps^2) when nothing
 * underflows (b b contributes eps b^2/S <= eps/2 to S, the fma eps, their
 * square root half of it, and the root itself eps).
 */
OR_API double or_k2_d(double x, double y)
{
    const double X = fabs(x);
    const double Y = fabs(y);
    const double m = min_d(X, Y);
    const double M = max_d(X, Y);
    if (isnan(M)) return M;
    if (M == 0.0) return 0.0;
    if (isinf(M)) return M;
    const int k = M < 0x1p-1022 ? -1022 : ilogb(M);
    const double a = M * p2_d(-k);
    const double b = m * p2_d(-k);
    const double S = fma(a, a, b * b);
    const double s = sqrt(S);
    return s * p2_d(k);
}

OR_API float or_k2_s(float x, float y)
{
    const float X = fabsf(x);
    const float Y = fabsf(y);
    const float m = min_s(X, Y);
    const float M = max_s(X, Y);
    if (isnan(M)) return M;
    if (M == 0.0f) return 0.0f;
    if (isinf(M)) return M;
    const int k = M < 0x1p-126f ? -126 : ilogbf(M);
    const float a = M * p2_s(-k);
    const float b = m * p2_s(-k);
    const float S = fmaf(a, a, b * b);
    const float s = sqrtf(S);
    return s * p2_s(k);
}

/* ------------------------------------------------------------------------ */
/* cr_hypot: the correctly rounded hypotenuse of the algorithm A (Section 2) */
/* ------------------------------------------------------------------------ */

typedef unsigned __int128 u128;

/* floor(sqrt(N)) for N < 2^127: a binary64 estimate, then exact steps. */
static uint64_t isqrt_u128(u128 N)
{
    double approx = (double)(uint64_t)(N >> 64) * 0x1p64 + (double)(uint64_t)N;
    uint64_t g = (uint64_t)sqrt(approx);
    while ((u128)g * g > N) --g;
    while ((u128)(g + 1) * (g + 1) <= N) ++g;
    return g;
}

/* 192-bit unsigned integers as hi * 2^128 + lo, for exact comparisons. */
typedef struct { uint64_t hi; u128 lo; } u192;

static u192 u192_shl(u128 v, int s) /* v * 2^s, 0 <= s <= 64 */
{
    u192 r;
    if (s == 0) { r.hi = 0; r.lo = v; return r; }
    r.hi = (uint64_t)(v >> (128 - s));
    r.lo = v << s;
    return r;
}

static u192 u192_add(u192 a, u192 b)
{
    u192 r;
    r.lo = a.lo + b.lo;
    r.hi = a.hi + b.hi + (r.lo < a.lo);
    return r;
}

static int u192_cmp(u192 a, u192 b)
{
    if (a.hi != b.hi) return a.hi < b.hi ? -1 : 1;
    if (a.lo != b.lo) return a.lo < b.lo ? -1 : 1;
    return 0;
}

/* integer significand and exponent: v = sig * 2^e, sig in [2^52, 2^53)
 * (subnormals normalised), v finite and nonzero */
static void decompose_d(double v, uint64_t *sig, int *e)
{
    uint64_t b = bits_d(v) & 0x7fffffffffffffffull;
    int ex = (int)(b >> 52);
    uint64_t m = b & 0x000fffffffffffffull;
    if (ex == 0) { /* subnormal: m * 2^-1074 */
        int sh = 0;
        while (!(m & (1ull << 52))) { m <<= 1; ++sh; }
        *sig = m;
        *e = -1074 - sh;
    } else {
        *sig = m | (1ull << 52);
        *e = ex - 1075;
    }
}

/*
 * or_cr_hypot_d(x, y) = RN(sqrt(x^2 + y^2)) exactly (the cr_hypot the
 * algorithm A uses; the paper takes it from CORE-MATH, which is not
 * available here, so it is computed from its definition with integers):
 *   X = max(|x|,|y|) = A 2^ex, Y = min = B 2^ey, d = ex - ey >= 0;
 *   d >= 28: Y/X < 2^-27 and the exact value lies below X (1 + 2^-55), so
 *   the result is X;
 *   else S = A^2 4^d + B^2 (x^2 + y^2 = S 4^ey) and the result is
 *   RN(sqrt(S / 4^d)) 2^ex, rounded to 53 bits by comparing 4S with the
 *   squares of the midpoints (ties go to even);
 *   both operands subnormal: RN(sqrt(a^2 + b^2)) 2^-1074 with a, b the
 *   integer multiples of 2^-1074.
 */
OR_API double or_cr_hypot_d(double x, double y)
{
    double X = fabs(x), Y = fabs(y);
    if (isinf(X) || isinf(Y)) return INFINITY;
    if (isnan(X) || isnan(Y)) return x + y;
    if (X < Y) { double t = X; X = Y; Y = t; }
    if (Y == 0.0) return X;
    if (X < 0x1p-1022) { /* both subnormal */
        const u128 a = bits_d(X), b = bits_d(Y);
        const u128 N = a * a + b * b;
        uint64_t T = isqrt_u128(N);
        const u128 m = (u128)(2 * T + 1) * (2 * T + 1); /* (2T+1)^2 vs 4N */
        const u128 N4 = N << 2;
        if (N4 > m || (N4 == m && (T & 1))) ++T;
        return from_bits_d(T); /* T < 2^53: subnormal or the smallest binade */
    }
    uint64_t A, B;
    int ex, ey;
    decompose_d(X, &A, &ex);
    decompose_d(Y, &B, &ey);
    const int d = ex - ey;
    if (d >= 28) return X;
    const u128 A2 = (u128)A * A, B2 = (u128)B * B;
    const u192 S = u192_add(u192_shl(A2, 2 * d), u192_shl(B2, 0));
    const u192 S4 = u192_add(u192_shl(A2, 2 * d + 2), u192_shl(B2, 2));
    const u128 Sd = A2 + (B2 >> (2 * d)); /* floor(S / 4^d) */
    (void)S;
    uint64_t T = isqrt_u128(Sd);
    int e = ex;
    int k = d; /* V = sqrt(S / 4^k) */
    if (T >> 53) { /* V >= 2^53: round V / 2 instead */
        T = isqrt_u128(Sd >> 2);
        k = d + 1;
        e = ex + 1;
    }
    const u128 m = (u128)(2 * T + 1) * (2 * T + 1);
    const int c = u192_cmp(S4, u192_shl(m, 2 * k));
    if (c > 0 || (c == 0 && (T & 1))) ++T;
    if (T >> 53) { T >>= 1; e += 1; }
    const int biased = e + 52 + 1023;
    if (biased >= 2047) return INFINITY;
    return from_bits_d(((uint64_t)biased << 52) | (T & 0x000fffffffffffffull));
}

/* binary32: the same with 24-bit significands; a gap of 14 or more gives X */
OR_API float or_cr_hypot_s(float x, float y)
{
    float X = fabsf(x), Y = fabsf(y);
    if (isinf(X) || isinf(Y)) return INFINITY;
    if (isnan(X) || isnan(Y)) return x + y;
    if (X < Y) { float t = X; X = Y; Y = t; }
    if (Y == 0.0f) return X;
    if (X < 0x1p-126f) {
        const uint64_t a = bits_s(X), b = bits_s(Y);
        const u128 N = (u128)a * a + (u128)b * b;
        uint64_t T = isqrt_u128(N);
        const u128 m = (u128)(2 * T + 1) * (2 * T + 1);
        if ((N << 2) > m || ((N << 2) == m && (T & 1))) ++T;
        return from_bits_s((uint32_t)T);
    }
    uint32_t bx = bits_s(X), by = bits_s(Y);
    uint64_t A = (bx & 0x7fffff) | 0x800000, B;
    int ex = (int)(bx >> 23) - 150, ey;
    if ((by >> 23) == 0) {
        B = by & 0x7fffff;
        int sh = 0;
        while (!(B & 0x800000)) { B <<= 1; ++sh; }
        ey = -149 - sh;
    } else {
        B = (by & 0x7fffff) | 0x800000;
        ey = (int)(by >> 23) - 150;
    }
    const int d = ex - ey;
    if (d >= 14) return X;
    const u128 A2 = (u128)A * A, B2 = (u128)B * B;
    const u128 S4 = ((A2 << (2 * d)) + B2) << 2;
    const u128 Sd = A2 + (B2 >> (2 * d));
    uint64_t T = isqrt_u128(Sd);
    int e = ex, k = d;
    if (T >> 24) {
        T = isqrt_u128(Sd >> 2);
        k = d + 1;
        e = ex + 1;
    }
    const u128 m = ((u128)(2 * T + 1) * (2 * T + 1)) << (2 * k);
    if (S4 > m || (S4 == m && (T & 1))) ++T;
    if (T >> 24) { T >>= 1; e += 1; }
    const int biased = e + 23 + 127;
    if (biased >= 255) return INFINITY;
    return from_bits_s(((uint32_t)biased << 23) | (uint32_t)(T & 0x7fffff));
}

/* ------------------------------------------------------------------------ */
/* pow for v1_lp                                                             */
/* ------------------------------------------------------------------------ */

static inline uint64_t bits_d(double x) { uint64_t u; memcpy(&u, &x, 8); return u; }
static inline double from_bits_d(uint64_t u) { double x; memcpy(&x, &u, 8); return x; }
static inline uint32_t bits_s(float x) { uint32_t u; memcpy(&u, &x, 4); return u; }
static inline float from_bits_s(uint32_t u) { float x; memcpy(&x, &u, 4); return x; }

/* 2^k as a binary32 for -149 <= k <= 127, built from its bit pattern. */
static float pow2_s(int k)
{
    if (k >= -126) return from_bits_s((uint32_t)(k + 127) << 23);
    return from_bits_s(1u << (k + 149));
}

/* ln 2 and 1/ln 2 as binary32 double-word constants (hi = RN(c),
 * lo ~ c - hi), for the binary32 pow. */
#define LN2F_HI 0x1.62e430p-1f
#define LN2F_LO -0x1.05c610p-29f
#define ILN2F_HI 0x1.715476p+0f
#define ILN2F_LO 0x1.4ae0c0p-26f
#define SQRT2_S 0x1.6a09e6p+0f

/*
 * or_pow_d(x, y) ~ x^y for x >= 0 and y > 0: the binary64 pow of Listing 5.
 * The paper leaves the pow to the platform (cr_pow, __builtin_pow, SLEEF);
 * this one is defined here in fixed-point integer arithmetic, so that the
 * oracle and the GPU compute the same bits and the pow needs no FP64
 * operation.  x^y = 2^(y log2 x); log2 x is reduced by two multipliers with
 * few bits (so that both products are exact in 64-bit integers), in the
 * manner of table-driven logarithms with short reciprocals, and 2^t by a
 * table of 2^(i/256).  A "Qk" integer v stands for v 2^-k; every right shift
 * of a magnitude is a floor.  Steps:
 *  1. x = M 2^(E-52), M in [2^52, 2^53); j = the top 8 fraction bits of M;
 *     for j >= 128, E += 1 (x = 2^E M/2^53, M/2^53 in [3/4, 1)).
 *  2. r1 = RN(2^17 / (256.5 + j)) (r1 = 512 for j = 0), an integer in
 *     [256, 512]; U1 = M r1 - 2^61 exactly: 1 + u1 = M r1 / 2^61 with
 *     |u1| <= 2^-8; log2 x = E + T1_j + log2(1 + u1), T1_j = log2(2^9/r1)
 *     (j < 128) or log2(2^8/r1) (j >= 128), so T1_0 = T1_255 = 0 and x next
 *     to 1 keeps its full relative precision.
 *  3. j2 = round(u1 2^16) = (U1 + 2^44) >> 45 (|j2| <= 256) and
 *     (1 + u1)(1 - j2 2^-16) = 1 + u2 exactly: U2 = (U1 - j2 2^45) 2^16 -
 *     U1 j2 in Q77, |u2| < 2^-15.4; log2(1 + u1) = T2_j2 + log2(1 + u2),
 *     T2_j2 = -log2(1 - j2 2^-16).
 *  4. ln(1 + u) = u - u^2 C, C = 1/2 - u/3 + u^2/4 - u^3/5 (the series to
 *     u^5/5; the first omitted term is below 2^-79 of u), with u = s a:
 *     C2 = 1/4 -+ a/5 in Q31 from the top 32 bits of a, C1 = 1/3 -+ a C2 in
 *     Q63 (a 32 x 32-bit product), C = 1/2 -+ a C1 in Q63, then a^2 C from
 *     the top words (a normalised: a = an 2^-(77+lg)); |ln(1+u)| = a -+ a^2 C
 *     as a 128-bit value with one bit of headroom (an 2^63 -+ a^2 C 2^(140+lg));
 *     log2(1+u) = that times ILN2 = RN(2^127/ln 2) (the three high partial
 *     products).  Every right shift here is a floor, and a shift by the word
 *     size or more gives 0 (for a tiny u these terms vanish).
 *  5. log2 x = E + T1_j + T2_j2 + log2(1+u2) in Q116 (T1 in Q88 and T2 in
 *     Q96 from the tables), or, when E = 0, T1_j = 0 and j2 = 0 (x within
 *     2^-17 of 1), the 128-bit log2(1+u2) with its exponent.
 *  6. t = y log2 x from y's 53-bit significand (192-bit product), truncated
 *     to Q64; |t| >= 2^11 overflows or underflows.
 *  7. k = floor(t), t - k = i/256 + rho (rho < 2^-8); v = rho ln 2 in Q70
 *     (ln 2 = RN(2^64 ln 2)); e^v by its Taylor series to degree 6 by Horner
 *     (the v^6, v^5 and v^4 coefficients in Q32 from the top 32 bits of v,
 *     the rest in Q63); 2^(t-k) = TE_i e^v with TE_i = RN(2^(i/256) 2^63)
 *     (a Q126 product).
 *  8. 2^k 2^(t-k) rounded to nearest (ties to even) to 53 bits, or to a
 *     multiple of 2^-1074 below 2^-1022; above 2^1024 it is +inf.
 * The tables: r1 from its integer definition; T1, T2 and TE from binary128
 * log2 and pow, rounded to nearest (pinned to the 400-bit values in the
 * tests).  Exact cases: pow(0,y) = 0, pow(1,y) = 1, pow(inf,y) = inf,
 * pow(x,0) = 1, pow(x,inf) = 0 (x < 1) or inf (x > 1), and pow(2^a, b) =
 * 2^(ab) whenever ab is an integer (then u1 = u2 = 0, T1 = T2 = 0, the
 * fraction of t is 0 and TE_0 e^0 = 2^126).
 */
#define PW_ILN2_HI 0xb8aa3b295c17f0bbull /* RN(2^127 / ln 2), high word */
#define PW_ILN2_LO 0xbe87fed0691d3e89ull /* low word */
#define PW_LN2 0xb17217f7d1cf79acull     /* RN(2^64 ln 2) */
#define PW_J2MAX 256

typedef __int128 i128;

static int clz64(uint64_t v) { return v ? __builtin_clzll(v) : 64; }

/* floor(v / 2^s) of a 192-bit value (hi 2^128 + lo), 0 <= s */
static u128 u192_shr(u192 v, int s)
{
    if (s >= 192) return 0;
    if (s >= 128) return (u128)(v.hi >> (s - 128));
    if (s == 0) return v.lo;
    return (v.lo >> s) | ((u128)v.hi << (128 - s));
}

/* r1_j = RN(2^18 / (513 + 2 j)), r1_0 = 512 */
static uint32_t pw_r1(int j)
{
    if (j == 0) return 512;
    const uint32_t den = 513u + 2u * (uint32_t)j, q = (1u << 18) / den, r = (1u << 18) % den;
    return q + (2 * r >= den ? 1u : 0u);
}

static i128 PW_T1[256];            /* Q88 */
static i128 PW_T1Q96[256];         /* the same logarithms in Q96, for or_powr_d */
static i128 PW_T2[2 * PW_J2MAX + 1]; /* Q96, index j2 + PW_J2MAX */
static uint64_t PW_TE[256];        /* Q63 */
static pthread_once_t pw_once = PTHREAD_ONCE_INIT;

static i128 q_round(q128 v) { return (i128)Q_FLOOR(v + (q128)0.5); }

static void pw_init(void)
{
    const q128 two88 = (q128)309485009821345068724781056.0;      /* 2^88 */
    const q128 two96 = two88 * (q128)256.0;                      /* 2^96 */
    for (int j = 0; j < 256; ++j) {
        const q128 r1 = (q128)pw_r1(j);
        PW_T1[j] = q_round(Q_LOG2((j < 128 ? (q128)512 : (q128)256) / r1) * two88);
        PW_T1Q96[j] = q_round(Q_LOG2((j < 128 ? (q128)512 : (q128)256) / r1) * two96);
    }
    for (int j2 = -PW_J2MAX; j2 <= PW_J2MAX; ++j2)
        PW_T2[j2 + PW_J2MAX] = q_round(-Q_LOG2((q128)1 - (q128)j2 / (q128)65536) * two96);
    for (int i = 0; i < 256; ++i)
        PW_TE[i] = (uint64_t)q_round(Q_POW((q128)2, (q128)i / 256) * (q128)9223372036854775808.0); /* 2^63 */
}

/* the tables, for the tests (r1 as integers, T1 and T2 as two's complement
 * {hi, lo} pairs) */
OR_API void or_pow_tables_d(uint64_t *R1, uint64_t *T1, uint64_t *T2, uint64_t *TE)
{
    pthread_once(&pw_once, pw_init);
    for (int j = 0; j < 256; ++j) {
        R1[j] = pw_r1(j);
        T1[2 * j] = (uint64_t)((u128)PW_T1[j] >> 64);
        T1[2 * j + 1] = (uint64_t)(u128)PW_T1[j];
        TE[j] = PW_TE[j];
    }
    for (int k = 0; k < 2 * PW_J2MAX + 1; ++k) {
        T2[2 * k] = (uint64_t)((u128)PW_T2[k] >> 64);
        T2[2 * k + 1] = (uint64_t)(u128)PW_T2[k];
    }
}

/* RN(P / 2^s), ties to even, for 1 <= s < 128 */
static u128 rne_shr(u128 P, int s)
{
    u128 q = P >> s;
    const u128 rem = P - (q << s), half = (u128)1 << (s - 1);
    if (rem > half || (rem == half && (q & 1))) q += 1;
    return q;
}

static uint64_t mulhi64(uint64_t a, uint64_t b) { return (uint64_t)(((u128)a * b) >> 64); }
static uint32_t mulhi32(uint32_t a, uint32_t b) { return (uint32_t)(((uint64_t)a * b) >> 32); }
/* floor(v / 2^s) for any s >= 0 (a shift by the word size or more gives 0,
 * which C leaves undefined) */
static uint32_t srl32(uint32_t v, int s) { return s >= 32 ? 0u : v >> s; }
static uint64_t srl64(uint64_t v, int s) { return s >= 64 ? 0ull : v >> s; }

OR_API double or_pow_d(double x, double y)
{
    if (isnan(x) || isnan(y)) return x + y;
    if (x == 0.0) return 0.0;
    if (x == 1.0) return 1.0;
    if (isinf(x)) return x;
    if (y == 0.0) return 1.0;
    if (isinf(y)) return x < 1.0 ? 0.0 : INFINITY;
    pthread_once(&pw_once, pw_init);
    /* step 1 */
    uint64_t M;
    int E;
    decompose_d(x, &M, &E);
    E += 52;
    const int j = (int)((M >> 44) & 255);
    if (j >= 128) E += 1;
    /* step 2 */
    const int64_t U1 = (int64_t)(M * (uint64_t)pw_r1(j) - (1ull << 61));
    /* step 3 */
    const int64_t j2 = (U1 + ((int64_t)1 << 44)) >> 45;
    const int64_t U2 = (int64_t)((uint64_t)(U1 - j2 * ((int64_t)1 << 45)) << 16) - U1 * j2;
    /* step 4: log2(1 + u2) = (s ? -1 : 1) L2m 2^-(139 + lg) */
    const int s = U2 < 0;
    u128 L2m = 0;
    int lg = 0;
    if (U2 != 0) {
        const uint64_t aint = s ? (uint64_t)(-U2) : (uint64_t)U2;
        lg = clz64(aint);
        const uint64_t an = aint << lg;
        const uint32_t ahi = (uint32_t)(an >> 32);
        const uint32_t t5 = srl32(mulhi32(ahi, 0x33333333u), 14 + lg);           /* a/5 in Q31 */
        const uint32_t C2 = s ? (1u << 29) + t5 : (1u << 29) - t5;                 /* Q31 */
        const uint64_t t1 = srl64((uint64_t)ahi * C2, 13 + lg);                     /* a C2 in Q63 */
        const uint64_t C1 = s ? 0x2aaaaaaaaaaaaaabull + t1 : 0x2aaaaaaaaaaaaaabull - t1; /* Q63 */
        const uint64_t t0 = srl64(mulhi64(an, C1), 13 + lg);                        /* a C1 in Q63 */
        const uint64_t C = s ? (1ull << 62) + t0 : (1ull << 62) - t0;               /* Q63 */
        const uint64_t sq = mulhi64(an, an);                                        /* a^2 2^(90+2lg) */
        const uint64_t m2 = mulhi64(sq, C);                                         /* a^2 C 2^(89+2lg) */
        const u128 corr = lg <= 51 ? (u128)m2 << (51 - lg) : (u128)srl64(m2, lg - 51);
        const u128 Ln = s ? ((u128)an << 63) + corr : ((u128)an << 63) - corr;     /* |ln(1+u)| 2^(140+lg) < 2^128 */
        const uint64_t Lh = (uint64_t)(Ln >> 64), Ll = (uint64_t)Ln;
        L2m = (u128)Lh * PW_ILN2_HI + (((u128)Lh * PW_ILN2_LO) >> 64) + (((u128)Ll * PW_ILN2_HI) >> 64);
    }
    /* step 5: log2 x = (neg ? -1 : 1) Lm 2^eL */
    u128 Lm;
    int eL;
    int neg;
    if (E == 0 && PW_T1[j] == 0 && j2 == 0) {
        Lm = L2m;
        eL = -(139 + lg);
        neg = s;
    } else {
        const u128 l2 = U2 != 0 ? L2m >> (23 + lg) : 0;
        const i128 Lq = (i128)E * ((i128)1 << 116) + PW_T1[j] * ((i128)1 << 28) +
                        PW_T2[j2 + PW_J2MAX] * ((i128)1 << 20) + (s ? -(i128)l2 : (i128)l2);
        neg = Lq < 0;
        Lm = neg ? (u128)(-Lq) : (u128)Lq;
        eL = -116;
    }
    /* step 6: t 2^64 = Ym Lm 2^(ey + eL + 64) */
    uint64_t Ym;
    int ey;
    decompose_d(y, &Ym, &ey);
    const u128 p0 = (u128)Ym * (uint64_t)Lm;
    const u128 p1 = (u128)Ym * (uint64_t)(Lm >> 64);
    u192 Pt;
    Pt.lo = p0 + (p1 << 64);
    Pt.hi = (uint64_t)(p1 >> 64) + (Pt.lo < p0);
    int bl;
    if (Pt.hi) bl = 192 - clz64(Pt.hi);
    else if ((uint64_t)(Pt.lo >> 64)) bl = 128 - clz64((uint64_t)(Pt.lo >> 64));
    else bl = 64 - clz64((uint64_t)Pt.lo);
    const int sh = ey + eL + 64;
    if (bl + sh > 75) return neg ? 0.0 : INFINITY;
    const u128 T64 = sh >= 0 ? Pt.lo << sh : u192_shr(Pt, -sh);
    const i128 tq = neg ? -(i128)T64 : (i128)T64;
    /* step 7 */
    const int k = (int)(tq >> 64);
    const uint64_t r = (uint64_t)tq;
    const int i = (int)(r >> 56);
    const uint64_t rho = r & ((1ull << 56) - 1);
    const uint64_t v70 = (uint64_t)(((u128)rho * PW_LN2) >> 58);
    const uint32_t v32 = (uint32_t)(v70 >> 38);                         /* v in Q32 */
    uint32_t e32 = (uint32_t)((1ull << 32) / 720);
    e32 = (uint32_t)((1ull << 32) / 120) + mulhi32(e32, v32);
    e32 = (uint32_t)((1ull << 32) / 24) + mulhi32(e32, v32);          /* Q32 */
    uint64_t Ev = (uint64_t)e32 << 31;                                  /* Q63 */
    Ev = (1ull << 63) / 6 + (mulhi64(Ev, v70) >> 6);
    Ev = (1ull << 62) + (mulhi64(Ev, v70) >> 6);
    Ev = (1ull << 63) + (mulhi64(Ev, v70) >> 6);
    Ev = (1ull << 63) + (mulhi64(Ev, v70) >> 6);
    const u128 P = (u128)PW_TE[i] * Ev; /* Q126 */
    /* step 8 */
    const int nb = (uint64_t)(P >> 64) ? 128 - clz64((uint64_t)(P >> 64)) : 64 - clz64((uint64_t)P);
    int Er = k + nb - 127;
    if (Er > 1023) return INFINITY;
    if (Er >= -1022) {
        uint64_t m = (uint64_t)rne_shr(P, nb - 53);
        if (m >> 53) { m >>= 1; Er += 1; }
        if (Er > 1023) return INFINITY;
        return from_bits_d(((uint64_t)(Er + 1023) << 52) | (m & 0x000fffffffffffffull));
    }
    const int shf = 126 - k - 1074;
    if (shf >= 128) return 0.0;
    return from_bits_d((uint64_t)rne_shr(P, shf)); /* a multiple of 2^-1074 (2^52 is 2^-1022) */
}

/*
 * or_powr_d(x, y): the pow of v1_lp for 1 < p <= 2^17 in binary64.  Its two
 * calls there are S = pow(Q, p/2), Q in [0, 1], p/2 in (1/2, 2^16], and
 * C = pow(Z, 1/p), Z in [1, 2], 1/p in [2^-17, 1); this is the domain:
 * 0 <= x < 1 with 1/2 <= y <= 2^16, or 1 <= x <= 2 with 2^-17 <= y <= 1.
 * Steps 1-3 and 7-8 are those of or_pow_d; log2 x and t = y log2 x are
 * formed differently, in plain fixed point, which the bound on y allows:
 *  4'. log2(1 + u), u = U2 2^-77, in Q96 from the series of ln(1 + u) to
 *      u^5 with the factor 1/ln 2 taken into the coefficients (the u^6
 *      term is below 2^-94): with a = |U2|,
 *        A1 = a D1 2^-76 (D1 = RN(2^95/ln 2), 96 bits, as D1h 2^32 + D1l:
 *             floor(a D1h / 2^44) + floor(a D1l / 2^76)),  |u|/ln 2
 *        sq = floor(a^2 / 2^64) (u^2 in Q90),
 *        A2 = floor(sq D2 / 2^64) 2^6 (D2 = RN(2^63/ln 2)),   u^2/(2 ln 2)
 *        cu = floor(sq a / 2^64) (|u|^3 in Q103),
 *        A3 = floor(floor(cu D3 / 2^64) / 2^7) (D3 = RN(2^64/(3 ln 2))),
 *        q4 = floor(sq/2^32)^2 (u^4 in Q116),
 *        A4 = floor(floor(q4/2^32) D4 / 2^20) (D4 = RN(2^32/(4 ln 2))),
 *        A5 = floor(floor(floor(q4/2^32) floor(a/2^32) / 2^32) D5 / 2^33)
 *             (D5 = RN(2^32/(5 ln 2))),
 *      and log2(1 + u) = A1 - A2 + A3 - A4 + A5 for u >= 0, -(A1 + A2 + A3
 *      + A4 + A5) for u < 0 (error below 2^-85).
 *  5'. W = E 2^96 + T1q_j + T2_j2 + log2(1 + u) = log2 x in Q96, T1q_j =
 *      RN(log2(2^9/r1_j) 2^96) (j < 128) or RN(log2(2^8/r1_j) 2^96).
 *  6'. y = Y 2^ey (Y the 53-bit significand): t 2^64 = sign(W) floor(Y |W|
 *      / 2^(32 - ey)) (|y| <= 2^16 keeps the error of W below 2^-69 in t).
 *  7-8 as or_pow_d with k = floor(t); the result is needed only in
 *      [2^-28, 2]: S below 2^-27 gives RN(1 + S^2) = 1 whatever S is, so
 *      k < -28 returns +0, and so does x < 2^-60 (t < -30 there).
 * The error before the final rounding stays below 2^-62 relative.  Exact
 * cases: pow(0, y) = 0, pow(1, y) = 1, and x = 2^a with ay an integer.
 */
#define PR_D1H 0xb8aa3b295c17f0bbull /* RN(2^95/ln 2) = PR_D1H 2^32 + PR_D1L */
#define PR_D1L 0xbe87fed0ull
#define PR_D2 0xb8aa3b295c17f0bcull  /* RN(2^63/ln 2) */
#define PR_D3 0x7b1c2770e80ff5d2ull  /* RN(2^64/(3 ln 2)) */
#define PR_D4 0x5c551d95ull          /* RN(2^32/(4 ln 2)) */
#define PR_D5 0x49ddb144ull          /* RN(2^32/(5 ln 2)) */

OR_API double or_powr_d(double x, double y)
{
    if (x == 0.0) return 0.0;
    if (x == 1.0) return 1.0;
    pthread_once(&pw_once, pw_init);
    /* step 1 */
    uint64_t M;
    int E;
    decompose_d(x, &M, &E);
    E += 52;
    const int j = (int)((M >> 44) & 255);
    if (j >= 128) E += 1;
    if (E < -60) return 0.0;
    /* steps 2 and 3 */
    const int64_t U1 = (int64_t)(M * (uint64_t)pw_r1(j) - (1ull << 61));
    const int64_t j2 = (U1 + ((int64_t)1 << 44)) >> 45;
    const int64_t U2 = (int64_t)((uint64_t)(U1 - j2 * ((int64_t)1 << 45)) << 16) - U1 * j2;
    /* step 4' */
    const uint64_t a = U2 < 0 ? (uint64_t)(-U2) : (uint64_t)U2;
    const u128 A1 = (((u128)a * PR_D1H) >> 44) + (((u128)a * PR_D1L) >> 76);
    const uint64_t sq = (uint64_t)(((u128)a * a) >> 64);
    const u128 A2 = (u128)(uint64_t)(((u128)sq * PR_D2) >> 64) << 6;
    const uint64_t cu = (uint64_t)(((u128)sq * a) >> 64);
    const uint64_t A3 = (uint64_t)(((u128)cu * PR_D3) >> 64) >> 7;
    const uint64_t s32 = sq >> 32;
    const uint64_t q4h = (s32 * s32) >> 32;
    const uint64_t A4 = (q4h * PR_D4) >> 20;
    const uint64_t A5 = (((q4h * (a >> 32)) >> 32) * PR_D5) >> 33;
    const i128 l = U2 < 0 ? -(i128)(A1 + A2 + A3 + A4 + A5) : (i128)(A1 + A3 + A5) - (i128)(A2 + A4);
    /* step 5' */
    const i128 W = (i128)E * ((i128)1 << 96) + PW_T1Q96[j] + PW_T2[j2 + PW_J2MAX] + l;
    /* step 6' */
    uint64_t Ym;
    int ey;
    decompose_d(y, &Ym, &ey);
    const u128 aW = W < 0 ? (u128)(-W) : (u128)W;
    const u128 p0 = (u128)Ym * (uint64_t)aW;
    const u128 p1 = (u128)Ym * (uint64_t)(aW >> 64);
    u192 Pt;
    Pt.lo = p0 + (p1 << 64);
    Pt.hi = (uint64_t)(p1 >> 64) + (Pt.lo < p0);
    const u128 T64 = u192_shr(Pt, 32 - ey);
    const i128 tq = W < 0 ? -(i128)T64 : (i128)T64;
    /* step 7 */
    const int k = (int)(tq >> 64);
    if (k < -28) return 0.0;
    const uint64_t r = (uint64_t)tq;
    const int i = (int)(r >> 56);
    const uint64_t rho = r & ((1ull << 56) - 1);
    const uint64_t v70 = (uint64_t)(((u128)rho * PW_LN2) >> 58);
    const uint32_t v32 = (uint32_t)(v70 >> 38); /* v in Q32 */
    uint32_t e32 = (uint32_t)((1ull << 32) / 720);
    e32 = (uint32_t)((1ull << 32) / 120) + mulhi32(e32, v32);
    e32 = (uint32_t)((1ull << 32) / 24) + mulhi32(e32, v32); /* Q32 */
    uint64_t Ev = (uint64_t)e32 << 31;                         /* Q63 */
    Ev = (1ull << 63) / 6 + (mulhi64(Ev, v70) >> 6);
    Ev = (1ull << 62) + (mulhi64(Ev, v70) >> 6);
    Ev = (1ull << 63) + (mulhi64(Ev, v70) >> 6);
    Ev = (1ull << 63) + (mulhi64(Ev, v70) >> 6);
    const u128 P = (u128)PW_TE[i] * Ev; /* Q126, in [2^126, 2^128) */
    /* step 8: a normal result (k in [-28, 1]) */
    const int nb = 128 - clz64((uint64_t)(P >> 64));
    int Er = k + nb - 127;
    uint64_t m = (uint64_t)rne_shr(P, nb - 53);
    if (m >> 53) { m >>= 1; Er += 1; }
    return from_bits_d(((uint64_t)(Er + 1023) << 52) | (m & 0x000fffffffffffffull));
}

/* or_powr_d serves v1_lp's pows when p/2 lies in (1/2, 2^16], i.e. for
 * 1 < p <= 2^17; other p (quasi-norms p < 1, very large p) take or_pow_d. */
static int powr_covers_d(double h) { return h > 0.5 && h <= 0x1p16; }

/*
 * or_pow_s(x, y) ~ x^y in binary32, the powf of Listing 5 for S; the same
 * five steps as or_pow_d with binary32 double-word arithmetic: atanh series
 * to z^5/13 and the exp series to degree 9.
 */
OR_API float or_pow_s(float x, float y)
{
    if (isnan(x) || isnan(y)) return x + y;
    if (x == 0.0f) return 0.0f;
    if (x == 1.0f) return 1.0f;
    if (isinf(x)) return x;
    uint32_t b = bits_s(x);
    int e = 0;
    if ((b >> 23) == 0) {
        x = x * 0x1p25f;
        b = bits_s(x);
        e = -25;
    }
    e += (int)(b >> 23) - 127;
    float f = from_bits_s((b & 0x007fffffu) | 0x3f800000u);
    if (f > SQRT2_S) { f = f * 0.5f; e = e + 1; }
    const float a = f - 1.0f;
    const float d_hi = f + 1.0f;
    const float d_lo = f - (d_hi - 1.0f);
    const float s_hi = a / d_hi;
    float rr = fmaf(-s_hi, d_hi, a);
    rr = fmaf(-s_hi, d_lo, rr);
    const float s_lo = rr / d_hi;
    const float z = s_hi * s_hi;
    float T = 1.0f / 13.0f;
    T = fmaf(T, z, 1.0f / 11.0f);
    T = fmaf(T, z, 1.0f / 9.0f);
    T = fmaf(T, z, 1.0f / 7.0f);
    T = fmaf(T, z, 1.0f / 5.0f);
    T = fmaf(T, z, 1.0f / 3.0f);
    const float c = (2.0f * s_hi) * (z * T);
    const float L_hi = 2.0f * s_hi;
    const float L_lo = fmaf(2.0f, s_lo, c);
    const float g_hi = L_hi * ILN2F_HI;
    float g_lo = fmaf(L_hi, ILN2F_HI, -g_hi);
    g_lo = fmaf(L_hi, ILN2F_LO, g_lo);
    g_lo = fmaf(L_lo, ILN2F_HI, g_lo);
    const float ed = (float)e;
    const float h = ed + g_hi;
    float l;
    if (fabsf(ed) >= fabsf(g_hi)) l = (ed - h) + g_hi;
    else l = (g_hi - h) + ed;
    l = l + g_lo;
    const float t_hi = y * h;
    float t_lo = fmaf(y, h, -t_hi);
    t_lo = fmaf(y, l, t_lo);
    if (t_hi < -200.0f) return 0.0f;
    if (t_hi > 200.0f) return INFINITY;
    const float k = rintf(t_hi);
    const float r0 = t_hi - k;
    const float r_hi = r0 + t_lo;
    const float r_lo = t_lo - (r_hi - r0);
    const float u_hi = r_hi * LN2F_HI;
    float u_lo = fmaf(r_hi, LN2F_HI, -u_hi);
    u_lo = fmaf(r_hi, LN2F_LO, u_lo);
    u_lo = fmaf(r_lo, LN2F_HI, u_lo);
    float P = 1.0f / 362880.0f;         /* 1/9! */
    P = fmaf(P, u_hi, 1.0f / 40320.0f); /* 1/8! */
    P = fmaf(P, u_hi, 1.0f / 5040.0f);  /* 1/7! */
    P = fmaf(P, u_hi, 1.0f / 720.0f);   /* 1/6! */
    P = fmaf(P, u_hi, 1.0f / 120.0f);   /* 1/5! */
    P = fmaf(P, u_hi, 1.0f / 24.0f);    /* 1/4! */
    P = fmaf(P, u_hi, 1.0f / 6.0f);     /* 1/3! */
    P = fmaf(P, u_hi, 0.5f);            /* 1/2! */
    const float E = (u_hi * u_hi) * P;
    const float m_hi = 1.0f + u_hi;
    const float m_err = (1.0f - m_hi) + u_hi;
    const float m = m_hi + (m_err + (u_lo + E));
    const int ki = (int)k;
    if (ki > 127) return INFINITY;
    if (ki < -149) return 0.0f;
    return m * pow2_s(ki);
}

/* v1_lp (Listing 5, Section 4): Eq. sp with the Eq. qp trick of squaring
 * pow(Q, p/2) inside an fma.  h = p*0.5 and ip = 1.0/p are computed once per
 * call (Section 4 hoists them to the top of the recursion).  Both pows are
 * or_powr_d for 1 < p <= 2^17 (h in (1/2, 2^16]), or_pow_d otherwise. */
OR_API double or_lp_d(double h, double ip, double x, double y)
{
    const double X = fabs(x);
    const double Y = fabs(y);
    const double m = min_d(X, Y);
    const double M = max_d(X, Y);
    const double q = m / M;
    const double Q = max_d(q, 0.0);
    const int r = powr_covers_d(h);
    const double S = r ? or_powr_d(Q, h) : or_pow_d(Q, h);
    const double Z = fma(S, S, 1.0);
    const double C = r ? or_powr_d(Z, ip) : or_pow_d(Z, ip);
    return M * C;
}

OR_API float or_lp_s(float h, float ip, float x, float y)
{
    const float X = fabsf(x);
    const float Y = fabsf(y);
    const float m = min_s(X, Y);
    const float M = max_s(X, Y);
    const float q = m / M;
    const float Q = max_s(q, 0.0f);
    const float S = or_pow_s(Q, h);
    const float Z = fmaf(S, S, 1.0f);
    const float C = or_pow_s(Z, ip);
    return M * C;
}

/* Elementwise forms of the pow and of v1_lp over arrays (one call per
 * element of the functions above), so that tests can check many operand
 * pairs at once. */
OR_API void or_pow_arr_d(int64_t n, const double *x, const double *y, double *out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = or_pow_d(x[i], y[i]);
}

OR_API void or_powr_arr_d(int64_t n, const double *x, const double *y, double *out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = or_powr_d(x[i], y[i]);
}

/* the Q96 logarithm table of or_powr_d, as two's complement {hi, lo} pairs */
OR_API void or_powr_table_d(uint64_t *T1q)
{
    pthread_once(&pw_once, pw_init);
    for (int j = 0; j < 256; ++j) {
        T1q[2 * j] = (uint64_t)((u128)PW_T1Q96[j] >> 64);
        T1q[2 * j + 1] = (uint64_t)(u128)PW_T1Q96[j];
    }
}

OR_API void or_pow_arr_s(int64_t n, const float *x, const float *y, float *out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = or_pow_s(x[i], y[i]);
}

OR_API void or_lp_arr_d(int64_t n, double h, double ip, const double *x, const double *y, double *out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = or_lp_d(h, ip, x[i], y[i]);
}

OR_API void or_lp_arr_s(int64_t n, float h, float ip, const float *x, const float *y, float *out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = or_lp_s(h, ip, x[i], y[i]);
}

/* p = 1 (Eq. vp1): |x| + |y|.  p = inf (Eq. vpI): max(|x|, |y|), exact. */
static double sumabs_d(double x, double y) { return fabs(x) + fabs(y); }
static float sumabs_s(float x, float y) { return fabsf(x) + fabsf(y); }
static double maxabs_d(double x, double y) { return max_d(fabs(x), fabs(y)); }
static float maxabs_s(float x, float y) { return max_s(fabsf(x), fabsf(y)); }

typedef struct { int op; double h, ip; } comb_d;
typedef struct { int op; float h, ip; } comb_s;

static double comb_apply_d(const comb_d *c, double x, double y)
{
    switch (c->op) {
    case OP_HYPOT: return or_k1_d(x, y);
    case OP_K2: return or_k2_d(x, y);
    case OP_LP: return or_lp_d(c->h, c->ip, x, y);
    case OP_SUMABS: return sumabs_d(x, y);
    default: return maxabs_d(x, y);
    }
}

static float comb_apply_s(const comb_s *c, float x, float y)
{
    switch (c->op) {
    case OP_HYPOT: return or_k1_s(x, y);
    case OP_K2: return or_k2_s(x, y);
    case OP_LP: return or_lp_s(c->h, c->ip, x, y);
    case OP_SUMABS: return sumabs_s(x, y);
    default: return maxabs_s(x, y);
    }
}

/* Cut-off p' (Section 4): for p at or above it, pow(Z, 1/p) = 1 for every Z
 * in [1, 2], so v1_lp returns M = max(|x|, |y|) and xNRMP may switch to the
 * p = inf code.  For this file's pow the powers of two 2^53 (binary64) and
 * 2^24 (binary32) are at or above p' (the paper finds 2^52 < p' <= 2^53 for
 * cr_pow and 2^23 < p' <= 2^24 for cr_powf); the switch changes no bit. */
#define P_CUT_D 0x1p53
#define P_CUT_S 0x1p24f

/* Choose the combine for a given p (Section 4): p = 2 is xNRMF (v1_hypot),
 * p = 1 sumabs, p = inf (or p >= the cut-off) maxabs, any other p > 0
 * v1_lp with p/2 and 1/p computed once here. */
static comb_d comb_for_d(double p)
{
    comb_d c = {OP_HYPOT, 0.0, 0.0};
    if (p == 2.0) c.op = OP_HYPOT;
    else if (p == 1.0) c.op = OP_SUMABS;
    else if (p >= P_CUT_D) c.op = OP_MAXABS;
    else { c.op = OP_LP; c.h = p * 0.5; c.ip = 1.0 / p; }
    return c;
}

static comb_s comb_for_s(float p)
{
    comb_s c = {OP_HYPOT, 0.0f, 0.0f};
    if (p == 2.0f) c.op = OP_HYPOT;
    else if (p == 1.0f) c.op = OP_SUMABS;
    else if (p >= P_CUT_S) c.op = OP_MAXABS;
    else { c.op = OP_LP; c.h = p * 0.5f; c.ip = 1.0f / p; }
    return c;
}

/* The combine the tree applies for p (Eq. vp1, v1_hypot, v1_lp, Eq. vpI with
 * the cut-off of Section 4), elementwise over arrays, for tests. */
OR_API void or_comb_arr_d(int64_t n, double p, const double *x, const double *y, double *out)
{
    const comb_d c = comb_for_d(p);
    for (int64_t i = 0; i < n; ++i) out[i] = comb_apply_d(&c, x[i], y[i]);
}

OR_API void or_comb_arr_s(int64_t n, float p, const float *x, const float *y, float *out)
{
    const comb_s c = comb_for_s(p);
    for (int64_t i = 0; i < n; ++i) out[i] = comb_apply_s(&c, x[i], y[i]);
}

/* ------------------------------------------------------------------------ */
/* R_x: the scalar recursion of Listing 1 / Eq. r                           */
/* ------------------------------------------------------------------------ */

/* R(n, x) (Listing 1, Eq. r): the norm of one element is its magnitude and
 * of two their combine; a longer array is cut after its first ceil(n/2)
 * elements and the norms of the two parts are combined (left part first). */
static double R_d(int64_t n, const double *x, const comb_d *c)
{
    if (n == 1) return fabs(x[0]);
    if (n == 2) return comb_apply_d(c, x[0], x[1]);
    const int64_t left = n - n / 2;
    const double a = R_d(left, x, c);
    const double b = R_d(n - left, x + left, c);
    return comb_apply_d(c, a, b);
}

static float R_s(int64_t n, const float *x, const comb_s *c)
{
    if (n == 1) return fabsf(x[0]);
    if (n == 2) return comb_apply_s(c, x[0], x[1]);
    const int64_t left = n - n / 2;
    const float a = R_s(left, x, c);
    const float b = R_s(n - left, x + left, c);
    return comb_apply_s(c, a, b);
}

/* The scalar algorithm H_x (R with v1_hypot) or its p-norm form.  n == 0
 * returns +0 (Listing 1 assumes n > 0; +0 is the norm of the empty array). */
OR_API double or_R_d(int64_t n, const double *x, double p)
{
    if (n <= 0) return 0.0;
    comb_d c = comb_for_d(p);
    return R_d(n, x, &c);
}

OR_API float or_R_s(int64_t n, const float *x, float p)
{
    if (n <= 0) return 0.0f;
    comb_s c = comb_for_s(p);
    return R_s(n, x, &c);
}

/* Trace of R's operations in completion order (Eq. r): for each operation
 * record (kind, first, last) with kind 1 = |x| leaf, 2 = hypot of two input
 * elements (a bold leaf of Eq. r), 3 = hypot of two partial norms; first and
 * last are the 1-based element range the operation covers. */
static void R_trace(int64_t n, int64_t off, int64_t *ops, int64_t *k)
{
    if (n == 1) { ops[3 * *k] = 1; ops[3 * *k + 1] = off + 1; ops[3 * *k + 2] = off + 1; (*k)++; return; }
    if (n == 2) { ops[3 * *k] = 2; ops[3 * *k + 1] = off + 1; ops[3 * *k + 2] = off + 2; (*k)++; return; }
    const int64_t p = (n >> 1) + (n & 1);
    R_trace(p, off, ops, k);
    R_trace(n - p, off + p, ops, k);
    ops[3 * *k] = 3; ops[3 * *k + 1] = off + 1; ops[3 * *k + 2] = off + n; (*k)++;
}

OR_API int64_t or_R_trace(int64_t n, int64_t *ops)
{
    int64_t k = 0;
    if (n > 0) R_trace(n, 0, ops, &k);
    return k;
}

/* ------------------------------------------------------------------------ */
/* Z_x: the vectorised recursion of Listing 4, generalised to P lanes       */
/* ------------------------------------------------------------------------ */

/* Z(n, x) -> f[0..P-1] (Listing 4 with 8 replaced by P):
 *   r = n mod P, m = ceil(n / P) vectors;
 *   m == 1: f = |x[0..P)|, or |TAIL| with the lanes past n set to zero;
 *   m == 2: f = op(x[0..P), second vector), the second being |TAIL| via Z
 *           when r > 0;
 *   else  : w = ceil(m/2) full vectors on the left, Z on both parts, and f =
 *           op lane-wise. */
static void Z_d(int64_t n, const double *x, int P, const comb_d *c, double *f)
{
    const int64_t r = n % P;
    const int64_t m = n / P + (r != 0);
    if (m == 1) {
        const int64_t cnt = r ? r : P;
        for (int l = 0; l < P; ++l) f[l] = (l < cnt) ? fabs(x[l]) : 0.0;
        return;
    }
    double *g = (double *)malloc(sizeof(double) * (size_t)P);
    if (m == 2) {
        if (r) Z_d(r, x + P, P, c, g);
        else for (int l = 0; l < P; ++l) g[l] = x[P + l];
        for (int l = 0; l < P; ++l) f[l] = comb_apply_d(c, x[l], g[l]);
        free(g);
        return;
    }
    const int64_t w = (m >> 1) + (m & 1);
    const int64_t p = w * P;
    const int64_t q = n - p;
    Z_d(p, x, P, c, f);
    Z_d(q, x + p, P, c, g);
    for (int l = 0; l < P; ++l) f[l] = comb_apply_d(c, f[l], g[l]);
    free(g);
}

static void Z_s(int64_t n, const float *x, int P, const comb_s *c, float *f)
{
    const int64_t r = n % P;
    const int64_t m = n / P + (r != 0);
    if (m == 1) {
        const int64_t cnt = r ? r : P;
        for (int l = 0; l < P; ++l) f[l] = (l < cnt) ? fabsf(x[l]) : 0.0f;
        return;
    }
    float *g = (float *)malloc(sizeof(float) * (size_t)P);
    if (m == 2) {
        if (r) Z_s(r, x + P, P, c, g);
        else for (int l = 0; l < P; ++l) g[l] = x[P + l];
        for (int l = 0; l < P; ++l) f[l] = comb_apply_s(c, x[l], g[l]);
        free(g);
        return;
    }
    const int64_t w = (m >> 1) + (m & 1);
    const int64_t p = w * P;
    const int64_t q = n - p;
    Z_s(p, x, P, c, f);
    Z_s(q, x + p, P, c, g);
    for (int l = 0; l < P; ++l) f[l] = comb_apply_s(c, f[l], g[l]);
    free(g);
}

/* The lane partials of Z for the given p (exported for the lane-grouping
 * pin of the p = 4, n = 16 example of Section 3). */
OR_API void or_Z_d(int64_t n, const double *x, int P, double p, double *f)
{
    comb_d c = comb_for_d(p);
    if (n <= 0) { for (int l = 0; l < P; ++l) f[l] = 0.0; return; }
    Z_d(n, x, P, &c, f);
}

OR_API void or_Z_s(int64_t n, const float *x, int P, float p, float *f)
{
    comb_s c = comb_for_s(p);
    if (n <= 0) { for (int l = 0; l < P; ++l) f[l] = 0.0f; return; }
    Z_s(n, x, P, &c, f);
}

/* xNRMF / xNRMP with lane width P: Z, then the final reduction R over the P
 * lane partials with the same combine (Section 3 recommends Z paired with a
 * recursive final reduction; here R uses the same op as the tree). */
OR_API double or_nrm_d(int64_t n, const double *x, int P, double p)
{
    if (n <= 0) return 0.0;
    comb_d c = comb_for_d(p);
    double *f = (double *)malloc(sizeof(double) * (size_t)P);
    Z_d(n, x, P, &c, f);
    const double v = R_d(P, f, &c);
    free(f);
    return v;
}

OR_API float or_nrm_s(int64_t n, const float *x, int P, float p)
{
    if (n <= 0) return 0.0f;
    comb_s c = comb_for_s(p);
    float *f = (float *)malloc(sizeof(float) * (size_t)P);
    Z_s(n, x, P, &c, f);
    const float v = R_s(P, f, &c);
    free(f);
    return v;
}

/* Thread driver (for timing the oracle on all host cores; Listing 4's
 * OpenCilk spawn of the two halves): the same Z recursion in which the
 * splits of the top `depth` levels evaluate their left part on a new thread
 * while the current thread evaluates the right part.  The split points and
 * the combine of the two halves are Z_d's, so the result is bitwise that of
 * the serial recursion; only the order in which subtrees finish changes. */
typedef struct { int64_t n; const double *x; int P; const comb_d *c; double *f; int depth; } zpar_d;
typedef struct { int64_t n; const float *x; int P; const comb_s *c; float *f; int depth; } zpar_s;
static void Z_par_d(int64_t n, const double *x, int P, const comb_d *c, double *f, int depth);
static void Z_par_s(int64_t n, const float *x, int P, const comb_s *c, float *f, int depth);
static void *zpar_thread_d(void *arg)
{
    const zpar_d *a = (const zpar_d *)arg;
    Z_par_d(a->n, a->x, a->P, a->c, a->f, a->depth);
    return NULL;
}
static void *zpar_thread_s(void *arg)
{
    const zpar_s *a = (const zpar_s *)arg;
    Z_par_s(a->n, a->x, a->P, a->c, a->f, a->depth);
    return NULL;
}

static void Z_par_d(int64_t n, const double *x, int P, const comb_d *c, double *f, int depth)
{
    const int64_t m = n / P + (n % P != 0);
    if (depth <= 0 || m <= 2) { Z_d(n, x, P, c, f); return; }
    const int64_t w = (m >> 1) + (m & 1);
    const int64_t p = w * P;
    double *g = (double *)malloc(sizeof(double) * (size_t)P);
    zpar_d left = {p, x, P, c, f, depth - 1};
    pthread_t th;
    const int spawned = pthread_create(&th, NULL, zpar_thread_d, &left) == 0;
    if (!spawned) Z_par_d(p, x, P, c, f, depth - 1);
    Z_par_d(n - p, x + p, P, c, g, depth - 1);
    if (spawned) pthread_join(th, NULL);
    for (int l = 0; l < P; ++l) f[l] = comb_apply_d(c, f[l], g[l]);
    free(g);
}

static void Z_par_s(int64_t n, const float *x, int P, const comb_s *c, float *f, int depth)
{
    const int64_t m = n / P + (n % P != 0);
    if (depth <= 0 || m <= 2) { Z_s(n, x, P, c, f); return; }
    const int64_t w = (m >> 1) + (m & 1);
    const int64_t p = w * P;
    float *g = (float *)malloc(sizeof(float) * (size_t)P);
    zpar_s left = {p, x, P, c, f, depth - 1};
    pthread_t th;
    const int spawned = pthread_create(&th, NULL, zpar_thread_s, &left) == 0;
    if (!spawned) Z_par_s(p, x, P, c, f, depth - 1);
    Z_par_s(n - p, x + p, P, c, g, depth - 1);
    if (spawned) pthread_join(th, NULL);
    for (int l = 0; l < P; ++l) f[l] = comb_apply_s(c, f[l], g[l]);
    free(g);
}

static int depth_for_threads(int nthreads)
{
    int d = 0;
    while ((1 << d) < nthreads && d < 16) ++d;
    return d;
}

/* or_nrm_* on up to 2^ceil(lg nthreads) threads, bitwise equal to it. */
OR_API double or_nrm_par_d(int64_t n, const double *x, int P, double p, int nthreads)
{
    if (n <= 0) return 0.0;
    comb_d c = comb_for_d(p);
    double *f = (double *)malloc(sizeof(double) * (size_t)P);
    Z_par_d(n, x, P, &c, f, depth_for_threads(nthreads));
    const double v = R_d(P, f, &c);
    free(f);
    return v;
}

OR_API float or_nrm_par_s(int64_t n, const float *x, int P, float p, int nthreads)
{
    if (n <= 0) return 0.0f;
    comb_s c = comb_for_s(p);
    float *f = (float *)malloc(sizeof(float) * (size_t)P);
    Z_par_s(n, x, P, &c, f, depth_for_threads(nthreads));
    const float v = R_s(P, f, &c);
    free(f);
    return v;
}

/* The paper's recommended xNRMF (Section 3): Z with v1_hypot on the vector
 * rows, then the final reduction of the P lane partials by A, i.e. R with
 * the correctly rounded hypot. */
static double R_cr_d(int64_t n, const double *x)
{
    if (n == 1) return fabs(x[0]);
    if (n == 2) return or_cr_hypot_d(x[0], x[1]);
    const int64_t p = (n >> 1) + (n & 1);
    return or_cr_hypot_d(R_cr_d(p, x), R_cr_d(n - p, x + p));
}

static float R_cr_s(int64_t n, const float *x)
{
    if (n == 1) return fabsf(x[0]);
    if (n == 2) return or_cr_hypot_s(x[0], x[1]);
    const int64_t p = (n >> 1) + (n & 1);
    return or_cr_hypot_s(R_cr_s(p, x), R_cr_s(n - p, x + p));
}

OR_API double or_nrm_za_d(int64_t n, const double *x, int P)
{
    if (n <= 0) return 0.0;
    comb_d c = comb_for_d(2.0);
    double *f = (double *)malloc(sizeof(double) * (size_t)P);
    Z_d(n, x, P, &c, f);
    const double v = R_cr_d(P, f);
    free(f);
    return v;
}

OR_API float or_nrm_za_s(int64_t n, const float *x, int P)
{
    if (n <= 0) return 0.0f;
    comb_s c = comb_for_s(2.0f);
    float *f = (float *)malloc(sizeof(float) * (size_t)P);
    Z_s(n, x, P, &c, f);
    const float v = R_cr_s(P, f);
    free(f);
    return v;
}

/* xNRMF with the exponent-scaled hypotenuse K2 in place of v1_hypot
 * everywhere: the same tree Z and final reduction R (Section 3), another
 * hypot[f] (Section 2). */
OR_API double or_nrm_es_d(int64_t n, const double *x, int P)
{
    if (n <= 0) return 0.0;
    const comb_d c = {OP_K2, 0.0, 0.0};
    double *f = (double *)malloc(sizeof(double) * (size_t)P);
    Z_d(n, x, P, &c, f);
    const double v = R_d(P, f, &c);
    free(f);
    return v;
}

OR_API float or_nrm_es_s(int64_t n, const float *x, int P)
{
    if (n <= 0) return 0.0f;
    const comb_s c = {OP_K2, 0.0f, 0.0f};
    float *f = (float *)malloc(sizeof(float) * (size_t)P);
    Z_s(n, x, P, &c, f);
    const float v = R_s(P, f, &c);
    free(f);
    return v;
}

OR_API void or_k2_arr_d(int64_t n, const double *x, const double *y, double *out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = or_k2_d(x[i], y[i]);
}

OR_API void or_k2_arr_s(int64_t n, const float *x, const float *y, float *out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = or_k2_s(x[i], y[i]);
}

/* Batched form: out[i] = or_nrm of x[off[i] .. off[i+1]). */
OR_API void or_nrm_batch_d(int64_t B, const int64_t *off, const double *x, int P, double p, double *out)
{
    for (int64_t i = 0; i < B; ++i) out[i] = or_nrm_d(off[i + 1] - off[i], x + off[i], P, p);
}

OR_API void or_nrm_batch_s(int64_t B, const int64_t *off, const float *x, int P, float p, float *out)
{
    for (int64_t i = 0; i < B; ++i) out[i] = or_nrm_s(off[i + 1] - off[i], x + off[i], P, p);
}

/* Strided vector (Section 3's incx): element i is x[i incx] for incx > 0
 * and x[(n-1-i) |incx|] for incx < 0 (taken backwards); its norm is the
 * norm of that logical vector. */
OR_API double or_nrm_strided_d(int64_t n, const double *x, int64_t incx, int P, double p)
{
    if (n <= 0) return 0.0;
    double *v = (double *)malloc(sizeof(double) * (size_t)n);
    const int64_t step = incx < 0 ? -incx : incx;
    for (int64_t i = 0; i < n; ++i) v[i] = incx > 0 ? x[i * step] : x[(n - 1 - i) * step];
    const double r = or_nrm_d(n, v, P, p);
    free(v);
    return r;
}

OR_API float or_nrm_strided_s(int64_t n, const float *x, int64_t incx, int P, float p)
{
    if (n <= 0) return 0.0f;
    float *v = (float *)malloc(sizeof(float) * (size_t)n);
    const int64_t step = incx < 0 ? -incx : incx;
    for (int64_t i = 0; i < n; ++i) v[i] = incx > 0 ? x[i * step] : x[(n - 1 - i) * step];
    const float r = or_nrm_s(n, v, P, p);
    free(v);
    return r;
}

/* Column-major M x N matrix with leading dimension lda (Section 3.1): with
 * contiguous storage (lda == M, or one column) it is one vector of M N
 * elements; otherwise the norms of the N columns are combined, here by the
 * same tree applied to the vector of column norms. */
OR_API double or_nrm_matrix_d(int64_t M, int64_t N, int64_t lda, const double *A, int P, double p)
{
    if (M <= 0 || N <= 0) return 0.0;
    if (lda == M || N == 1) return or_nrm_d(M * N, A, P, p);
    double *c = (double *)malloc(sizeof(double) * (size_t)N);
    for (int64_t j = 0; j < N; ++j) c[j] = or_nrm_d(M, A + j * lda, P, p);
    const double r = or_nrm_d(N, c, P, p);
    free(c);
    return r;
}

OR_API float or_nrm_matrix_s(int64_t M, int64_t N, int64_t lda, const float *A, int P, float p)
{
    if (M <= 0 || N <= 0) return 0.0f;
    if (lda == M || N == 1) return or_nrm_s(M * N, A, P, p);
    float *c = (float *)malloc(sizeof(float) * (size_t)N);
    for (int64_t j = 0; j < N; ++j) c[j] = or_nrm_s(M, A + j * lda, P, p);
    const float r = or_nrm_s(N, c, P, p);
    free(c);
    return r;
}

/* ------------------------------------------------------------------------ */
/* slot form: the same vector-row tree as a perfect tree with empty slots   */
/* ------------------------------------------------------------------------ */

/* Bit reversal of the low d bits of j. */
static uint64_t brev_bits(uint64_t j, int d)
{
    uint64_t r = 0;
    for (int i = 0; i < d; ++i) { r = (r << 1) | (j & 1); j >>= 1; }
    return r;
}

/*
 * Second evaluation of Z: the ceil-split tree over the m = ceil(n/P) vector
 * rows is embedded in a perfect binary tree of depth D = ceil(lg m); leaf
 * slot j holds a row iff brev_D(j) < m, occupied slots hold the rows in array
 * order, and a node with one empty child passes the other child through
 * unchanged (Listing 4 never combines with an empty part).  The combine is
 * done bottom-up, level by level.  This is the form the GPU evaluates; it
 * is written independently of Z_d above so that a test can pin one against
 * the other.
 */
OR_API double or_nrm_slot_d(int64_t n, const double *x, int P, double p)
{
    if (n <= 0) return 0.0;
    comb_d c = comb_for_d(p);
    const int64_t m = (n + P - 1) / P;
    int D = 0;
    while ((1ll << D) < m) ++D;
    const int64_t S = 1ll << D;
    /* level-D values: S slots x P lanes, plus an occupancy flag */
    double *v = (double *)malloc(sizeof(double) * (size_t)(S * P));
    unsigned char *occ = (unsigned char *)malloc((size_t)S);
    int64_t row = 0;
    for (int64_t j = 0; j < S; ++j) {
        occ[j] = brev_bits((uint64_t)j, D) < (uint64_t)m;
        if (!occ[j]) continue;
        for (int l = 0; l < P; ++l) {
            const int64_t i = row * P + l;
            v[j * P + l] = (i < n) ? fabs(x[i]) : 0.0;
        }
        ++row;
    }
    for (int64_t w = S; w > 1; w >>= 1) {
        for (int64_t j = 0; j < w / 2; ++j) {
            const int64_t a = 2 * j, b = 2 * j + 1;
            if (occ[a] && occ[b]) {
                for (int l = 0; l < P; ++l) v[j * P + l] = comb_apply_d(&c, v[a * P + l], v[b * P + l]);
            } else if (occ[a]) {
                for (int l = 0; l < P; ++l) v[j * P + l] = v[a * P + l];
            } else if (occ[b]) {
                for (int l = 0; l < P; ++l) v[j * P + l] = v[b * P + l];
            }
            occ[j] = occ[a] | occ[b];
        }
    }
    /* final reduction: perfect tree over the P lanes (P a power of two), as
     * R's ceil split gives for such P */
    for (int w = P; w > 1; w >>= 1)
        for (int l = 0; l < w / 2; ++l) v[l] = comb_apply_d(&c, v[2 * l], v[2 * l + 1]);
    const double out = (P == 1) ? fabs(v[0]) : v[0];
    free(v);
    free(occ);
    return out;
}

OR_API float or_nrm_slot_s(int64_t n, const float *x, int P, float p)
{
    if (n <= 0) return 0.0f;
    comb_s c = comb_for_s(p);
    const int64_t m = (n + P - 1) / P;
    int D = 0;
    while ((1ll << D) < m) ++D;
    const int64_t S = 1ll << D;
    float *v = (float *)malloc(sizeof(float) * (size_t)(S * P));
    unsigned char *occ = (unsigned char *)malloc((size_t)S);
    int64_t row = 0;
    for (int64_t j = 0; j < S; ++j) {
        occ[j] = brev_bits((uint64_t)j, D) < (uint64_t)m;
        if (!occ[j]) continue;
        for (int l = 0; l < P; ++l) {
            const int64_t i = row * P + l;
            v[j * P + l] = (i < n) ? fabsf(x[i]) : 0.0f;
        }
        ++row;
    }
    for (int64_t w = S; w > 1; w >>= 1) {
        for (int64_t j = 0; j < w / 2; ++j) {
            const int64_t a = 2 * j, b = 2 * j + 1;
            if (occ[a] && occ[b]) {
                for (int l = 0; l < P; ++l) v[j * P + l] = comb_apply_s(&c, v[a * P + l], v[b * P + l]);
            } else if (occ[a]) {
                for (int l = 0; l < P; ++l) v[j * P + l] = v[a * P + l];
            } else if (occ[b]) {
                for (int l = 0; l < P; ++l) v[j * P + l] = v[b * P + l];
            }
            occ[j] = occ[a] | occ[b];
        }
    }
    for (int w = P; w > 1; w >>= 1)
        for (int l = 0; l < w / 2; ++l) v[l] = comb_apply_s(&c, v[2 * l], v[2 * l + 1]);
    const float out = (P == 1) ? fabsf(v[0]) : v[0];
    free(v);
    free(occ);
    return out;
}

/* ------------------------------------------------------------------------ */
/* binary128 reference (stands in for the MPFR reference of Eq. relerr)     */
/* ------------------------------------------------------------------------ */

typedef struct {
    const void *x;
    int64_t n;
    int is_double;
    int kind; /* 0: sum x^2, 1: sum |x|, 2: sum |x|^p, 3: max |x| */
    q128 p;
    q128 result;
} q_job;

/* pairwise sum of the terms of x[0..n) (recursion on halves; the relative
 * error of such a sum is below lg(n) * 2^-113, far under the tolerances) */
static q128 q_term(const q_job *jb, int64_t i)
{
    q128 v = jb->is_double ? (q128)((const double *)jb->x)[i] : (q128)((const float *)jb->x)[i];
    v = Q_FABS(v);
    switch (jb->kind) {
    case 0: return v * v;
    case 1: return v;
    case 2: return (v == 0) ? (q128)0 : Q_POW(v, jb->p);
    default: return v;
    }
}

static q128 q_sum(const q_job *jb, int64_t lo, int64_t n)
{
    if (n <= 8) {
        q128 s = 0;
        for (int64_t i = 0; i < n; ++i) {
            q128 t = q_term(jb, lo + i);
            if (jb->kind == 3) { if (t > s) s = t; }
            else s += t;
        }
        return s;
    }
    const int64_t h = n / 2;
    q128 a = q_sum(jb, lo, h), b = q_sum(jb, lo + h, n - h);
    if (jb->kind == 3) return a > b ? a : b;
    return a + b;
}

static void *q_thread(void *arg)
{
    q_job *jb = (q_job *)arg;
    jb->result = q_sum(jb, 0, jb->n);
    return NULL;
}

/* Reference p-norm of x[0..n) in binary128, returned as a double-word
 * (hi, lo) with hi = RN_double(v) and lo = RN_double(v - hi).  p = 2 sums
 * exact squares, p = 1 sums |x|, p = inf takes max |x|, other p sum
 * |x|^p with the binary128 pow.  nthreads contiguous chunks are summed in
 * parallel and then added in chunk order. */
OR_API void or_ref_q128(int64_t n, const void *x, int is_double, double p, int nthreads, double *hi, double *lo)
{
    int kind;
    if (p == 2.0) kind = 0;
    else if (p == 1.0) kind = 1;
    else if (isinf(p)) kind = 3;
    else kind = 2;
    if (nthreads < 1) nthreads = 1;
    if (n < (int64_t)nthreads * 4096) nthreads = 1;
    q_job *jobs = (q_job *)calloc((size_t)nthreads, sizeof(q_job));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    const int64_t chunk = (n + nthreads - 1) / nthreads;
    for (int t = 0; t < nthreads; ++t) {
        const int64_t lo_i = (int64_t)t * chunk;
        int64_t cnt = n - lo_i;
        if (cnt > chunk) cnt = chunk;
        if (cnt < 0) cnt = 0;
        jobs[t].x = is_double ? (const void *)((const double *)x + lo_i) : (const void *)((const float *)x + lo_i);
        jobs[t].n = cnt;
        jobs[t].is_double = is_double;
        jobs[t].kind = kind;
        jobs[t].p = (q128)p;
        jobs[t].result = 0;
    }
    if (nthreads == 1) q_thread(&jobs[0]);
    else {
        for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, q_thread, &jobs[t]);
        for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    }
    q128 s = 0;
    for (int t = 0; t < nthreads; ++t) {
        if (kind == 3) { if (jobs[t].result > s) s = jobs[t].result; }
        else s += jobs[t].result;
    }
    q128 v;
    if (kind == 0) v = Q_SQRT(s);
    else if (kind == 1 || kind == 3) v = s;
    else v = (s == 0) ? (q128)0 : Q_POW(s, (q128)1 / (q128)p);
    const double h = (double)v;
    *hi = h;
    *lo = (double)(v - (q128)h);
    free(jobs);
    free(th);
}

/* ------------------------------------------------------------------------ */
/* error bounds                                                              */
/* ------------------------------------------------------------------------ */

/*
 * Closed form of the upper bound ub relerr (Eq. ubr) for a recursion whose
 * longest leaf-to-root path has `depth` hypot operations, each with relative
 * error factor at most 1 + eps' (Theorem 3 with equal bounds in both
 * subtrees): ub = ((1 + eps')^depth - 1) / eps.  which = 0: A (cr_hypot,
 * eps' = eps); which = 1: H (v1_hypot, 1 + eps' from Eq. reH).  prec = 0:
 * eps = 2^-53 (D); prec = 1: eps = 2^-24 (S).  Evaluated in binary128 and
 * returned as (hi, lo).  Table 3 prints this value for n = 2^k, depth = k.
 */
OR_API void or_ub_relerr(int depth, int prec, int which, double *hi, double *lo)
{
    const q128 eps = prec ? (q128)0x1p-24 : (q128)0x1p-53;
    q128 f;
    if (which == 0) f = 1 + eps;
    else {
        const q128 a = 1 + eps;
        const q128 a52 = a * a * Q_SQRT(a); /* (1+eps)^(5/2) */
        f = a52 * Q_SQRT(1 + eps * (2 + eps) / 2);
    }
    q128 pw = 1;
    for (int i = 0; i < depth; ++i) pw *= f;
    const q128 v = (pw - 1) / eps;
    const double h = (double)v;
    *hi = h;
    *lo = (double)(v - (q128)h);
}

/* Lower factor 1 + eps'^- of Eq. reH, (hi, lo), for the tests. */
OR_API void or_reH_factors(int prec, double *lo_hi, double *lo_lo, double *up_hi, double *up_lo)
{
    const q128 eps = prec ? (q128)0x1p-24 : (q128)0x1p-53;
    const q128 b = 1 - eps;
    const q128 lower = b * b * Q_SQRT(b) * Q_SQRT(1 - eps * (2 - eps) / 2);
    const q128 a = 1 + eps;
    const q128 upper = a * a * Q_SQRT(a) * Q_SQRT(1 + eps * (2 + eps) / 2);
    *lo_hi = (double)lower;
    *lo_lo = (double)(lower - (q128)*lo_hi);
    *up_hi = (double)upper;
    *up_lo = (double)(upper - (q128)*up_hi);
}

/* Tree depth of the GPU tree for n elements and lane width P: number of
 * combine levels on the longest leaf-to-root path = ceil(lg ceil(n/P)) +
 * lg P (the row tree, then R over the P lanes). */
OR_API int or_tree_depth(int64_t n, int P)
{
    if (n <= 0) return 0;
    const int64_t m = (n + P - 1) / P;
    int D = 0;
    while ((1ll << D) < m) ++D;
    int L = 0;
    while ((1 << L) < P) ++L;
    return D + L;
}
