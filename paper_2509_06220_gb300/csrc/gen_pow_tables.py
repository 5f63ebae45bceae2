"""Write nrm_pow_tables.h: the constants of the library's binary64 pow.

The pow that v1_lp uses (Listing 5; Section 4 leaves the pow to the
platform) is x^y = 2^(y log2 x) in fixed-point integer arithmetic with a
table-driven reduction in the manner of Tang's table-driven log and exp.
This script computes its tables with mpmath at 400 bits and rounds each
entry to nearest:

  C_j   = 2^52 + j 2^44 (j < 128), 2^52 + (j + 1) 2^44 (j >= 128), the
          reference significand for the top 8 fraction bits j of x
  R_j   = RN(2^179 / C_j), 128 bits, in [2^126, 2^127]
  T_j   = RN(log2(F_j) 2^80), F_j = C_j 2^-52 (j < 128) or C_j 2^-53
          (j >= 128); T_0 = T_255 = 0
  TE_i  = RN(2^(i/64) 2^63), i = 0..63
  ILN2  = RN(2^127 / ln 2), 128 bits
  LN2   = RN(2^64 ln 2)

Run from this directory: python gen_pow_tables.py (needs mpmath); the
tests pin every entry of the written header against these definitions.
"""
import os

import mpmath

mpmath.mp.prec = 400
HERE = os.path.dirname(os.path.abspath(__file__))


def rn(v):
    return int(mpmath.floor(v + mpmath.mpf("0.5")))


def c_of(j):
    return (1 << 52) + ((j + (1 if j >= 128 else 0)) << 44)


def tables():
    two = mpmath.mpf(2)
    R = [rn(two ** 179 / c_of(j)) for j in range(256)]
    T = [rn(mpmath.log(mpmath.mpf(c_of(j)) / two ** (53 if j >= 128 else 52), 2) * two ** 80) for j in range(256)]
    TE = [rn(two ** (mpmath.mpf(i) / 64) * two ** 63) for i in range(64)]
    ILN2 = rn(two ** 127 / mpmath.log(2))
    LN2 = rn(mpmath.log(2) * two ** 64)
    return R, T, TE, ILN2, LN2


def main():
    R, T, TE, ILN2, LN2 = tables()
    M = (1 << 64) - 1
    out = []
    out.append("// nrm_pow_tables.h -- generated by gen_pow_tables.py; do not edit.")
    out.append("// Tables of the binary64 pow of v1_lp (Listing 5): see gen_pow_tables.py for")
    out.append("// the definition of every entry (each rounded to nearest from 400-bit values).")
    out.append("#pragma once")
    out.append("#include <cstdint>")
    out.append("namespace nrm {")
    out.append("// R_j = RN(2^179 / C_j) as {high, low} words")
    out.append("static __device__ const uint64_t kPowR[256][2] = {")
    for j in range(0, 256, 2):
        out.append("    " + " ".join("{0x%016xull, 0x%016xull}," % (R[k] >> 64, R[k] & M) for k in (j, j + 1)))
    out.append("};")
    out.append("// T_j = RN(log2(F_j) 2^80) as a two's-complement 128-bit {high, low}")
    out.append("static __device__ const uint64_t kPowT[256][2] = {")
    for j in range(0, 256, 2):
        out.append("    " + " ".join("{0x%016xull, 0x%016xull}," % (((T[k] >> 64) & M), T[k] & M) for k in (j, j + 1)))
    out.append("};")
    out.append("// TE_i = RN(2^(i/64) 2^63)")
    out.append("static __device__ const uint64_t kPowTE[64] = {")
    for i in range(0, 64, 4):
        out.append("    " + " ".join("0x%016xull," % TE[k] for k in range(i, i + 4)))
    out.append("};")
    out.append("constexpr uint64_t kPowILN2_HI = 0x%016xull; // RN(2^127 / ln 2), high word" % (ILN2 >> 64))
    out.append("constexpr uint64_t kPowILN2_LO = 0x%016xull; // low word" % (ILN2 & M))
    out.append("constexpr uint64_t kPowLN2 = 0x%016xull;     // RN(2^64 ln 2)" % LN2)
    out.append("} // namespace nrm")
    with open(os.path.join(HERE, "nrm_pow_tables.h"), "w") as f:
        f.write("\n".join(out) + "\n")


if __name__ == "__main__":
    main()
