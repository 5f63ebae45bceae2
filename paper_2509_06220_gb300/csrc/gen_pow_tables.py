"""Write nrm_pow_tables.h: the constants of the library's binary64 pow.

The pow that v1_lp uses (Listing 5; Section 4 leaves the pow to the
platform) is x^y = 2^(y log2 x) in fixed-point integer arithmetic; log2 x
is reduced by two multipliers with few bits, so that both products are exact
in 64-bit integers, in the manner of table-driven logarithms with short
reciprocals, and 2^t by a table of 2^(i/256).  This script computes its
tables with mpmath at 400 bits and rounds each entry to nearest:

  r1_j  = RN(2^18 / (513 + 2 j)) for j = 1..255 and r1_0 = 512: the first
          multiplier for the top 8 fraction bits j of x (M r1_j / 2^61 is
          within 2^-8 of 1)
  T1_j  = RN(log2(2^9 / r1_j) 2^88) (j < 128) or RN(log2(2^8 / r1_j) 2^88)
          (j >= 128, where the exponent of x is taken one higher); T1_0 =
          T1_255 = 0
  T2_j2 = RN(-log2(1 - j2 2^-16) 2^96), j2 = -256..256 (index j2 + 256)
  TE_i  = RN(2^(i/256) 2^63), i = 0..255
  ILN2  = RN(2^127 / ln 2), 128 bits
  LN2   = RN(2^64 ln 2)

and for the pow of v1_lp with 1 < p <= 2^17 (powr_d), whose logarithm is
formed in Q96 fixed point with 1/ln 2 taken into the series coefficients:

  T1q_j = RN(log2(2^9 / r1_j) 2^96) (j < 128) or RN(log2(2^8 / r1_j) 2^96)
  D1    = RN(2^95 / ln 2) (96 bits, as D1h 2^32 + D1l), D2 = RN(2^63 / ln 2),
  D3    = RN(2^64 / (3 ln 2)), D4 = RN(2^32 / (4 ln 2)), D5 = RN(2^32 / (5 ln 2))

Run from this directory: python gen_pow_tables.py (needs mpmath); the
tests pin every entry of the written header against these definitions.
"""
import os

import mpmath

mpmath.mp.prec = 400
HERE = os.path.dirname(os.path.abspath(__file__))
J2MAX = 256


def rn(v):
    return int(mpmath.floor(v + mpmath.mpf("0.5")))


def r1_of(j):
    if j == 0:
        return 512
    den = 513 + 2 * j
    q, r = divmod(1 << 18, den)
    return q + (1 if 2 * r >= den else 0)


def tables():
    two = mpmath.mpf(2)
    R1 = [r1_of(j) for j in range(256)]
    T1 = [rn(mpmath.log(mpmath.mpf(512 if j < 128 else 256) / R1[j], 2) * two ** 88) for j in range(256)]
    T2 = [rn(-mpmath.log(1 - mpmath.mpf(j2) / 65536, 2) * two ** 96) for j2 in range(-J2MAX, J2MAX + 1)]
    TE = [rn(two ** (mpmath.mpf(i) / 256) * two ** 63) for i in range(256)]
    ILN2 = rn(two ** 127 / mpmath.log(2))
    LN2 = rn(mpmath.log(2) * two ** 64)
    return R1, T1, T2, TE, ILN2, LN2


def powr_tables():
    two = mpmath.mpf(2)
    ln2 = mpmath.log(2)
    R1 = [r1_of(j) for j in range(256)]
    T1q = [rn(mpmath.log(mpmath.mpf(512 if j < 128 else 256) / R1[j], 2) * two ** 96) for j in range(256)]
    D = {"D1": rn(two ** 95 / ln2), "D2": rn(two ** 63 / ln2), "D3": rn(two ** 64 / (3 * ln2)),
         "D4": rn(two ** 32 / (4 * ln2)), "D5": rn(two ** 32 / (5 * ln2))}
    return T1q, D


def main():
    R1, T1, T2, TE, ILN2, LN2 = tables()
    M = (1 << 64) - 1
    out = []
    out.append("// nrm_pow_tables.h -- generated by gen_pow_tables.py; do not edit.")
    out.append("// Tables of the binary64 pow of v1_lp (Listing 5): see gen_pow_tables.py for")
    out.append("// the definition of every entry (each rounded to nearest from 400-bit values).")
    out.append("#pragma once")
    out.append("#include <cstdint>")
    out.append("namespace nrm {")
    out.append("// r1_j, the first multiplier of the reduction")
    out.append("static __device__ const uint16_t kPowR1[256] = {")
    for j in range(0, 256, 16):
        out.append("    " + " ".join("%d," % R1[k] for k in range(j, j + 16)))
    out.append("};")
    out.append("// T1_j = RN(log2(2^9 or 2^8 / r1_j) 2^88) as a two's-complement 128-bit {high, low}")
    out.append("static __device__ __align__(16) const uint64_t kPowT1[256][2] = {")
    for j in range(0, 256, 2):
        out.append("    " + " ".join("{0x%016xull, 0x%016xull}," % (((T1[k] >> 64) & M), T1[k] & M) for k in (j, j + 1)))
    out.append("};")
    out.append("// T2_j2 = RN(-log2(1 - j2 2^-16) 2^96), index j2 + %d, as {high, low}" % J2MAX)
    out.append("static __device__ __align__(16) const uint64_t kPowT2[%d][2] = {" % (2 * J2MAX + 1))
    for k in range(0, 2 * J2MAX + 1, 2):
        ks = [k] if k + 1 > 2 * J2MAX else [k, k + 1]
        out.append("    " + " ".join("{0x%016xull, 0x%016xull}," % (((T2[i] >> 64) & M), T2[i] & M) for i in ks))
    out.append("};")
    out.append("// TE_i = RN(2^(i/256) 2^63)")
    out.append("static __device__ const uint64_t kPowTE[256] = {")
    for i in range(0, 256, 4):
        out.append("    " + " ".join("0x%016xull," % TE[k] for k in range(i, i + 4)))
    out.append("};")
    T1q, D = powr_tables()
    out.append("// T1q_j = RN(log2(2^9 or 2^8 / r1_j) 2^96) as a two's-complement 128-bit {high, low}")
    out.append("static __device__ __align__(16) const uint64_t kPowT1Q96[256][2] = {")
    for j in range(0, 256, 2):
        out.append("    " + " ".join("{0x%016xull, 0x%016xull}," % (((T1q[k] >> 64) & M), T1q[k] & M) for k in (j, j + 1)))
    out.append("};")
    out.append("constexpr uint64_t kPrD1H = 0x%016xull; // RN(2^95 / ln 2) = kPrD1H 2^32 + kPrD1L" % (D["D1"] >> 32))
    out.append("constexpr uint64_t kPrD1L = 0x%08xull;" % (D["D1"] & 0xFFFFFFFF))
    out.append("constexpr uint64_t kPrD2 = 0x%016xull; // RN(2^63 / ln 2)" % D["D2"])
    out.append("constexpr uint64_t kPrD3 = 0x%016xull; // RN(2^64 / (3 ln 2))" % D["D3"])
    out.append("constexpr uint32_t kPrD4 = 0x%08xu; // RN(2^32 / (4 ln 2))" % D["D4"])
    out.append("constexpr uint32_t kPrD5 = 0x%08xu; // RN(2^32 / (5 ln 2))" % D["D5"])
    out.append("constexpr int kPowJ2Max = %d;" % J2MAX)
    out.append("constexpr uint64_t kPowILN2_HI = 0x%016xull; // RN(2^127 / ln 2), high word" % (ILN2 >> 64))
    out.append("constexpr uint64_t kPowILN2_LO = 0x%016xull; // low word" % (ILN2 & M))
    out.append("constexpr uint64_t kPowLN2 = 0x%016xull;     // RN(2^64 ln 2)" % LN2)
    out.append("} // namespace nrm")
    with open(os.path.join(HERE, "nrm_pow_tables.h"), "w") as f:
        f.write("\n".join(out) + "\n")


if __name__ == "__main__":
    main()
