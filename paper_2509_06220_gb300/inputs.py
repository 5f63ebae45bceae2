"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds none of the norm arithmetic: it only builds input arrays
bit by bit from a counter-based hash, so that the host (numpy, here) and the
device (``nrm_gen_d`` / ``nrm_gen_s`` in the CUDA library, which implement
the same definition) produce identical arrays.

Definition (all arithmetic modulo 2^64):

* ``mix64`` is the SplitMix64 output function (Steele, Lea and Flood,
  "Fast splittable pseudorandom number generators", OOPSLA 2014):
  ``z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27;
  z *= 0x94D049BB133111EB; z ^= z >> 31``.
* ``key(seed, vec) = mix64(seed ^ mix64((vec + 1) * G))`` with
  ``G = 0x9E3779B97F4A7C15``.
* ``draw(key, i) = mix64(key + (i + 1) * G)``.
* Element ``i`` of vector ``vec`` (binary64): ``u = draw(key(seed, vec), i)``,
  sign = bit 63, fraction = the low 52 bits, exponent
  ``e = emin + ((((u >> 52) & 0x7FF) * (emax - emin + 1)) >> 11)``; the
  element is ``(-1)^sign * (1 + fraction/2^52) * 2^e`` built from its bits.
  Binary32: fraction = the low 23 bits, ``e = emin + ((((u >> 23) & 0xFFFF) *
  (emax - emin + 1)) >> 16)``.

The default exponent range [-20, 20] gives the moderately varying
magnitudes of the paper's test arrays (Section 2 generates them with small
magnitudes so that large n does not overflow); [-8, 8] is the range of the
p-norm workload.
"""
import numpy as np

G = np.uint64(0x9E3779B97F4A7C15)
_C1 = np.uint64(0xBF58476D1CE4E5B9)
_C2 = np.uint64(0x94D049BB133111EB)
LENGTH_STREAM = 0xFFFFFFFF  # vector id used for drawing ragged lengths

_CHUNK = 1 << 22


def mix64(z):
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = z ^ (z >> np.uint64(30))
        z = z * _C1
        z = z ^ (z >> np.uint64(27))
        z = z * _C2
        z = z ^ (z >> np.uint64(31))
    return z


def key(seed, vec):
    with np.errstate(over="ignore"):
        v = (np.asarray(vec, dtype=np.uint64) + np.uint64(1)) * G
    return mix64(np.asarray(seed, dtype=np.uint64) ^ mix64(v))


def draw(k, idx):
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix64(np.asarray(k, dtype=np.uint64) + (idx + np.uint64(1)) * G)


def _bits_d(u, emin, emax):
    span = np.uint64(emax - emin + 1)
    eb = (u >> np.uint64(52)) & np.uint64(0x7FF)
    e = (eb * span) >> np.uint64(11)  # in [0, span)
    biased = (e.astype(np.int64) + (emin + 1023)).astype(np.uint64)
    return (u & np.uint64(0x8000000000000000)) | (biased << np.uint64(52)) | (u & np.uint64((1 << 52) - 1))


def _bits_s(u, emin, emax):
    span = np.uint64(emax - emin + 1)
    eb = (u >> np.uint64(23)) & np.uint64(0xFFFF)
    e = (eb * span) >> np.uint64(16)
    biased = (e.astype(np.int64) + (emin + 127)).astype(np.uint64)
    b = ((u >> np.uint64(63)) << np.uint64(31)) | (biased << np.uint64(23)) | (u & np.uint64((1 << 23) - 1))
    return b.astype(np.uint32)


def vector(n, seed=0, vec=0, dtype=np.float64, emin=-20, emax=20, start=0):
    """Elements start .. start+n-1 of vector `vec` for `seed`."""
    if not (-1022 <= emin <= emax <= 1023) or (np.dtype(dtype) == np.float32 and not (-126 <= emin <= emax <= 127)):
        raise ValueError("exponent range outside the normal range of the format")
    dt = np.dtype(dtype)
    out = np.empty(n, dtype=dt)
    k = key(seed, vec)
    for lo in range(0, n, _CHUNK):
        hi = min(n, lo + _CHUNK)
        u = draw(k, np.arange(start + lo, start + hi, dtype=np.uint64))
        if dt == np.float64:
            out[lo:hi] = _bits_d(u, emin, emax).view(np.float64)
        else:
            out[lo:hi] = _bits_s(u, emin, emax).view(np.float32)
    return out


def ragged_lengths(B, seed=0, max_log2=18, min_log2=0):
    """Lengths L_i = floor(2^(min_log2 + (max_log2-min_log2) U_i)), U_i uniform
    in [0,1) from the LENGTH_STREAM draws; log-uniform in [2^min, 2^max]."""
    u = draw(key(seed, LENGTH_STREAM), np.arange(B, dtype=np.uint64))
    U = (u >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    L = np.floor(np.exp2(min_log2 + (max_log2 - min_log2) * U)).astype(np.int64)
    return np.clip(L, 1 << min_log2, 1 << max_log2)


def ragged_batch(B, seed=0, dtype=np.float64, max_log2=18, min_log2=0, emin=-20, emax=20, lengths=None):
    """Concatenated ragged batch: vector i has elements key(seed, i)."""
    L = ragged_lengths(B, seed, max_log2, min_log2) if lengths is None else np.asarray(lengths, np.int64)
    off = np.zeros(len(L) + 1, dtype=np.int64)
    np.cumsum(L, out=off[1:])
    x = np.empty(int(off[-1]), dtype=np.dtype(dtype))
    for i, n in enumerate(L):
        x[off[i]:off[i + 1]] = vector(int(n), seed, i, dtype, emin, emax)
    return x, off
