"""Plain serial C oracle for xNRMF / xNRMP (arXiv 2509.06220), via ctypes.

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
benchmark's CPU-baseline leg, never by the product path.  It shares no code
with the CUDA library.  See nrm_oracle.c for what each routine computes and
which passage of the paper it follows.

Lane widths of the GPU tree (fixed by the tree definition, Section 3: the
results are reproducible only for a fixed lane count): P_D = 64 lanes of
binary64 and P_S = 128 lanes of binary32, i.e. one 512-byte row.
"""
import ctypes
import numpy as np

from . import build as _build

P_D = 64
P_S = 128

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        d, f, i64, i32 = ctypes.c_double, ctypes.c_float, ctypes.c_int64, ctypes.c_int
        vp = ctypes.c_void_p
        pd = ctypes.POINTER(ctypes.c_double)
        sig = {
            "or_k1_d": (d, [d, d]),
            "or_k1_s": (f, [f, f]),
            "or_pow_d": (d, [d, d]),
            "or_pow_s": (f, [f, f]),
            "or_lp_d": (d, [d, d, d, d]),
            "or_lp_s": (f, [f, f, f, f]),
            "or_pow_arr_d": (None, [i64, vp, vp, vp]),
            "or_pow_arr_s": (None, [i64, vp, vp, vp]),
            "or_powr_d": (d, [d, d]),
            "or_powr_arr_d": (None, [i64, vp, vp, vp]),
            "or_powr_table_d": (None, [vp]),
            "or_lp_arr_d": (None, [i64, d, d, vp, vp, vp]),
            "or_lp_arr_s": (None, [i64, f, f, vp, vp, vp]),
            "or_comb_arr_d": (None, [i64, d, vp, vp, vp]),
            "or_k2_d": (d, [d, d]),
            "or_k2_s": (f, [f, f]),
            "or_k2_arr_d": (None, [i64, vp, vp, vp]),
            "or_k2_arr_s": (None, [i64, vp, vp, vp]),
            "or_nrm_es_d": (d, [i64, vp, i32]),
            "or_nrm_es_s": (f, [i64, vp, i32]),
            "or_comb_arr_s": (None, [i64, f, vp, vp, vp]),
            "or_R_d": (d, [i64, vp, d]),
            "or_R_s": (f, [i64, vp, f]),
            "or_R_trace": (i64, [i64, vp]),
            "or_Z_d": (None, [i64, vp, i32, d, vp]),
            "or_Z_s": (None, [i64, vp, i32, f, vp]),
            "or_nrm_d": (d, [i64, vp, i32, d]),
            "or_nrm_s": (f, [i64, vp, i32, f]),
            "or_nrm_par_d": (d, [i64, vp, i32, d, i32]),
            "or_nrm_par_s": (f, [i64, vp, i32, f, i32]),
            "or_nrm_batch_d": (None, [i64, vp, vp, i32, d, vp]),
            "or_nrm_batch_s": (None, [i64, vp, vp, i32, f, vp]),
            "or_cr_hypot_d": (d, [d, d]),
            "or_cr_hypot_s": (f, [f, f]),
            "or_nrm_za_d": (d, [i64, vp, i32]),
            "or_nrm_za_s": (f, [i64, vp, i32]),
            "or_nrm_strided_d": (d, [i64, vp, i64, i32, d]),
            "or_nrm_strided_s": (f, [i64, vp, i64, i32, f]),
            "or_nrm_matrix_d": (d, [i64, i64, i64, vp, i32, d]),
            "or_nrm_matrix_s": (f, [i64, i64, i64, vp, i32, f]),
            "or_nrm_slot_d": (d, [i64, vp, i32, d]),
            "or_nrm_slot_s": (f, [i64, vp, i32, f]),
            "or_ref_q128": (None, [i64, vp, i32, d, i32, pd, pd]),
            "or_ub_relerr": (None, [i32, i32, i32, pd, pd]),
            "or_reH_factors": (None, [i32, pd, pd, pd, pd]),
            "or_tree_depth": (i32, [i64, i32]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _arr(x, dtype):
    a = np.ascontiguousarray(x, dtype=dtype)
    return a, a.ctypes.data_as(ctypes.c_void_p)


def _is_d(x):
    return np.asarray(x).dtype == np.float64


def k1(x, y, dtype=np.float64):
    """v1_hypot of Listing 2 (binary64 or binary32)."""
    if np.dtype(dtype) == np.float64:
        return np.float64(lib().or_k1_d(float(x), float(y)))
    return np.float32(lib().or_k1_s(float(np.float32(x)), float(np.float32(y))))


def pow_(x, y, dtype=np.float64):
    if np.dtype(dtype) == np.float64:
        return np.float64(lib().or_pow_d(float(x), float(y)))
    return np.float32(lib().or_pow_s(float(np.float32(x)), float(np.float32(y))))


def pow_arr(x, y):
    """Elementwise pow over two arrays of one dtype (float64 or float32)."""
    dt = np.asarray(x).dtype
    xa, xp = _arr(x, dt)
    ya, yp = _arr(y, dt)
    out = np.empty(xa.shape, dt)
    f = lib().or_pow_arr_d if dt == np.float64 else lib().or_pow_arr_s
    f(xa.size, xp, yp, out.ctypes.data_as(ctypes.c_void_p))
    return out


def powr_arr(x, y):
    """Elementwise or_powr_d (the binary64 pow of v1_lp for 1 < p <= 2^17)
    over two float64 arrays."""
    xa, xp = _arr(x, np.float64)
    ya, yp = _arr(y, np.float64)
    out = np.empty(xa.shape, np.float64)
    lib().or_powr_arr_d(xa.size, xp, yp, out.ctypes.data_as(ctypes.c_void_p))
    return out


def powr_table():
    """or_powr_d's Q96 logarithm table T1q_j as Python ints."""
    t = np.zeros(512, np.uint64)
    lib().or_powr_table_d(t.ctypes.data_as(ctypes.c_void_p))
    out = []
    for j in range(256):
        v = int(t[2 * j]) << 64 | int(t[2 * j + 1])
        out.append(v - (1 << 128) if v >> 127 else v)
    return out


def lp_arr(p, x, y):
    """Elementwise v1_lp over two arrays, h = p*0.5 and ip = 1/p in their dtype."""
    dt = np.asarray(x).dtype
    xa, xp = _arr(x, dt)
    ya, yp = _arr(y, dt)
    out = np.empty(xa.shape, dt)
    if dt == np.float64:
        lib().or_lp_arr_d(xa.size, float(p) * 0.5, 1.0 / float(p), xp, yp, out.ctypes.data_as(ctypes.c_void_p))
    else:
        p32 = np.float32(p)
        lib().or_lp_arr_s(xa.size, float(np.float32(p32 * np.float32(0.5))), float(np.float32(np.float32(1) / p32)),
                          xp, yp, out.ctypes.data_as(ctypes.c_void_p))
    return out


def comb_arr(p, x, y):
    """Elementwise combine of the tree for p (v1_hypot for p = 2, |x|+|y|
    for p = 1, max for p at or above the cut-off, else v1_lp)."""
    dt = np.asarray(x).dtype
    xa, xp = _arr(x, dt)
    ya, yp = _arr(y, dt)
    out = np.empty(xa.shape, dt)
    f = lib().or_comb_arr_d if dt == np.float64 else lib().or_comb_arr_s
    f(xa.size, float(p) if dt == np.float64 else float(np.float32(p)), xp, yp, out.ctypes.data_as(ctypes.c_void_p))
    return out


def k2(x, y, dtype=np.float64):
    """The exponent-scaled hypotenuse K2 (binary64 or binary32)."""
    if np.dtype(dtype) == np.float64:
        return np.float64(lib().or_k2_d(float(x), float(y)))
    return np.float32(lib().or_k2_s(float(np.float32(x)), float(np.float32(y))))


def k2_arr(x, y):
    """Elementwise K2 over two arrays of one dtype."""
    dt = np.asarray(x).dtype
    xa, xp = _arr(x, dt)
    ya, yp = _arr(y, dt)
    out = np.empty(xa.shape, dt)
    f = lib().or_k2_arr_d if dt == np.float64 else lib().or_k2_arr_s
    f(xa.size, xp, yp, out.ctypes.data_as(ctypes.c_void_p))
    return out


def nrm_es(x):
    """xNRMF with K2 in place of v1_hypot (same tree, P = 64 / 128)."""
    dt = np.asarray(x).dtype
    a, ap = _arr(x, dt)
    if dt == np.float64:
        return np.float64(lib().or_nrm_es_d(a.size, ap, P_D))
    return np.float32(lib().or_nrm_es_s(a.size, ap, P_S))


def lp(p, x, y, dtype=np.float64):
    """v1_lp of Listing 5 with h = p*0.5, ip = 1/p computed in `dtype`."""
    if np.dtype(dtype) == np.float64:
        h, ip = float(p) * 0.5, 1.0 / float(p)
        return np.float64(lib().or_lp_d(h, ip, float(x), float(y)))
    p32 = np.float32(p)
    h = np.float32(p32 * np.float32(0.5))
    ip = np.float32(np.float32(1.0) / p32)
    return np.float32(lib().or_lp_s(float(h), float(ip), float(np.float32(x)), float(np.float32(y))))


def R(x, p=2.0):
    """The scalar recursion R_x (Listing 1) with the combine chosen by p."""
    if _is_d(x):
        a, ptr = _arr(x, np.float64)
        return np.float64(lib().or_R_d(a.size, ptr, float(p)))
    a, ptr = _arr(x, np.float32)
    return np.float32(lib().or_R_s(a.size, ptr, float(np.float32(p))))


def R_trace(n):
    ops = np.zeros(3 * max(2 * n, 1), dtype=np.int64)
    k = lib().or_R_trace(n, ops.ctypes.data_as(ctypes.c_void_p))
    return [tuple(int(v) for v in ops[3 * i:3 * i + 3]) for i in range(k)]


def Z(x, P, p=2.0):
    """Lane partials of the vectorised recursion (Listing 4) with P lanes."""
    if _is_d(x):
        a, ptr = _arr(x, np.float64)
        f = np.zeros(P, np.float64)
        lib().or_Z_d(a.size, ptr, P, float(p), f.ctypes.data_as(ctypes.c_void_p))
        return f
    a, ptr = _arr(x, np.float32)
    f = np.zeros(P, np.float32)
    lib().or_Z_s(a.size, ptr, P, float(np.float32(p)), f.ctypes.data_as(ctypes.c_void_p))
    return f


def nrm(x, p=2.0, P=None):
    """xNRMF (p = 2) / xNRMP of x: Z with P lanes, then R over the lanes."""
    if _is_d(x):
        a, ptr = _arr(x, np.float64)
        return np.float64(lib().or_nrm_d(a.size, ptr, P or P_D, float(p)))
    a, ptr = _arr(x, np.float32)
    return np.float32(lib().or_nrm_s(a.size, ptr, P or P_S, float(np.float32(p))))


def nrm_par(x, p=2.0, threads=None, P=None):
    """nrm() evaluated on `threads` host threads (default: all cores): the
    top splits of the same tree run concurrently; bitwise equal to nrm()."""
    import os
    t = int(threads or os.cpu_count() or 1)
    if _is_d(x):
        a, ptr = _arr(x, np.float64)
        return np.float64(lib().or_nrm_par_d(a.size, ptr, P or P_D, float(p), t))
    a, ptr = _arr(x, np.float32)
    return np.float32(lib().or_nrm_par_s(a.size, ptr, P or P_S, float(np.float32(p)), t))


def cr_hypot(x, y, dtype=np.float64):
    """RN(sqrt(x^2 + y^2)): the correctly rounded hypot of the algorithm A."""
    if np.dtype(dtype) == np.float64:
        return np.float64(lib().or_cr_hypot_d(float(x), float(y)))
    return np.float32(lib().or_cr_hypot_s(float(np.float32(x)), float(np.float32(y))))


def nrm_za(x, P=None):
    """Z with v1_hypot, then A (R with cr_hypot) over the lanes."""
    if _is_d(x):
        a, ptr = _arr(x, np.float64)
        return np.float64(lib().or_nrm_za_d(a.size, ptr, P or P_D))
    a, ptr = _arr(x, np.float32)
    return np.float32(lib().or_nrm_za_s(a.size, ptr, P or P_S))


def nrm_strided(buf, n, incx, p=2.0, P=None):
    """Norm of the strided vector over buf (element 0 = lowest address)."""
    if _is_d(buf):
        a, ptr = _arr(buf, np.float64)
        return np.float64(lib().or_nrm_strided_d(n, ptr, incx, P or P_D, float(p)))
    a, ptr = _arr(buf, np.float32)
    return np.float32(lib().or_nrm_strided_s(n, ptr, incx, P or P_S, float(np.float32(p))))


def nrm_matrix(buf, M, N, lda, p=2.0, P=None):
    """Norm of the column-major M x N matrix stored in buf with leading dimension lda."""
    if _is_d(buf):
        a, ptr = _arr(buf, np.float64)
        return np.float64(lib().or_nrm_matrix_d(M, N, lda, ptr, P or P_D, float(p)))
    a, ptr = _arr(buf, np.float32)
    return np.float32(lib().or_nrm_matrix_s(M, N, lda, ptr, P or P_S, float(np.float32(p))))


def nrm_slot(x, p=2.0, P=None):
    """The same tree evaluated in slot form (second, independent routine)."""
    if _is_d(x):
        a, ptr = _arr(x, np.float64)
        return np.float64(lib().or_nrm_slot_d(a.size, ptr, P or P_D, float(p)))
    a, ptr = _arr(x, np.float32)
    return np.float32(lib().or_nrm_slot_s(a.size, ptr, P or P_S, float(np.float32(p))))


def nrm_batch(x, offsets, p=2.0, P=None):
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    B = off.size - 1
    if _is_d(x):
        a, ptr = _arr(x, np.float64)
        out = np.zeros(B, np.float64)
        lib().or_nrm_batch_d(B, off.ctypes.data_as(ctypes.c_void_p), ptr, P or P_D, float(p),
                             out.ctypes.data_as(ctypes.c_void_p))
        return out
    a, ptr = _arr(x, np.float32)
    out = np.zeros(B, np.float32)
    lib().or_nrm_batch_s(B, off.ctypes.data_as(ctypes.c_void_p), ptr, P or P_S, float(np.float32(p)),
                         out.ctypes.data_as(ctypes.c_void_p))
    return out


def ref_q128(x, p=2.0, nthreads=1):
    """Binary128 reference p-norm as (hi, lo) doubles."""
    a = np.ascontiguousarray(x)
    isd = 1 if a.dtype == np.float64 else 0
    if not isd:
        a = np.ascontiguousarray(a, dtype=np.float32)
    hi, lo = ctypes.c_double(), ctypes.c_double()
    lib().or_ref_q128(a.size, a.ctypes.data_as(ctypes.c_void_p), isd, float(p), int(nthreads),
                      ctypes.byref(hi), ctypes.byref(lo))
    return hi.value, lo.value


def relerr(value, x, p=2.0, nthreads=1):
    """|ref - value| / ref against the unrounded binary128 reference (Eq.
    relerr without the division by eps)."""
    hi, lo = ref_q128(x, p, nthreads)
    if hi == 0.0:
        return 0.0 if float(value) == 0.0 else float("inf")
    v = float(value)
    return abs((hi - v) + lo) / hi


def ub_relerr(depth, prec="D", which="H"):
    hi, lo = ctypes.c_double(), ctypes.c_double()
    lib().or_ub_relerr(int(depth), 0 if prec == "D" else 1, 1 if which == "H" else 0,
                       ctypes.byref(hi), ctypes.byref(lo))
    return hi.value, lo.value


def reH_factors(prec="D"):
    v = [ctypes.c_double() for _ in range(4)]
    lib().or_reH_factors(0 if prec == "D" else 1, *[ctypes.byref(t) for t in v])
    return (v[0].value, v[1].value), (v[2].value, v[3].value)


def tree_depth(n, P):
    return lib().or_tree_depth(int(n), int(P))
