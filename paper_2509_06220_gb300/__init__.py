"""GB300 (sm_103a) xNRMF / xNRMP: recursive hypot-tree norms (arXiv 2509.06220).

A thin ctypes binding of the C ABI in include/nrm.h (libnrm.so, built in
tree by ``paper_2509_06220_gb300.build``).  PyTorch provides device memory
and streams; every step of the computation runs in the library's CUDA
kernels.  There is no CPU fallback: if the library is missing the import of
the binding raises.

Entry points (same names as the C ABI):

* ``nrmf(x)``           xNRMF of a 1-D float32/float64 CUDA tensor (0-d result on device)
* ``nrmp(x, p)``        xNRMP, p > 0 (p = 2 is xNRMF, p = 1 sum |x|, p = inf max |x|)
* ``nrm_batch(x, offsets, p)``       ragged batch -> (out, status); p a float or a
                                     CUDA float64 tensor of one p per vector
* ``nrm_batch_graph(...)``           the same, captured once as a CUDA graph
* ``nrm_host(x_host, p)``            host buffer in, Python float out (end to end)
* ``nrm_gen`` / ``nrm_gen_ragged``   seeded synthetic inputs on the device
"""
import ctypes
import os
import re

import numpy as np

from . import build as _build_mod

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(os.path.dirname(HERE), "include", "nrm.h")

NRM_OK, NRM_EINVAL, NRM_ENOMEM, NRM_ECUDA, NRM_ETIMEOUT, NRM_EBUDGET, NRM_EDEVICE = 0, -1, -2, -3, -4, -5, -6
NRM_F32, NRM_F64 = 0, 1
P_LANES = {NRM_F32: 128, NRM_F64: 64}


class NrmError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        super().__init__("%s%s" % (_status_name(status), (": " + msg) if msg else ""))


class Tuning(ctypes.Structure):
    _fields_ = [("group_log2", ctypes.c_int32), ("warps_per_block", ctypes.c_int32),
                ("item_log2", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32)]


class Request(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int32), ("emin", ctypes.c_int32), ("emax", ctypes.c_int32),
                ("p", ctypes.c_double), ("n", ctypes.c_int64), ("x_host", ctypes.c_void_p),
                ("seed", ctypes.c_uint64), ("arrival_s", ctypes.c_double)]


class SrvReport(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in ("submitted", "admitted", "rejected", "completed", "steps", "launches",
                                              "max_queue", "peak_bytes", "arena_bytes")] + \
               [(f, ctypes.c_double) for f in ("p50_ms", "p99_ms", "mean_ms", "max_ms", "wall_s", "norms_per_s",
                                               "elements_per_s", "host_launch_s", "host_retire_s", "gpu_step_s")]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def lib_path():
    return _build_mod.LIB


def load():
    """Load libnrm.so (must have been built; no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        raise ImportError("libnrm.so is not built (%s); run paper_2509_06220_gb300.build.build() or "
                          "__graft_entry__.build()" % path)
    L = ctypes.CDLL(path)
    vp, i64, i32, u64, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_size_t
    st = ctypes.c_int32
    sigs = {
        "nrm_create": (st, [ctypes.POINTER(vp), ctypes.c_int]),
        "nrm_destroy": (st, [vp]),
        "nrm_status_string": (ctypes.c_char_p, [st]),
        "nrm_last_error": (ctypes.c_char_p, [vp]),
        "nrm_reserve": (st, [vp, sz]),
        "nrm_workspace_bytes": (sz, [vp, i32, i64, i64]),
        "nrm_get_tuning": (st, [vp, ctypes.POINTER(Tuning)]),
        "nrm_set_tuning": (st, [vp, ctypes.POINTER(Tuning)]),
        "nrm_get_tuning_for": (st, [vp, i32, ctypes.POINTER(Tuning)]),
        "nrm_set_tuning_for": (st, [vp, i32, ctypes.POINTER(Tuning)]),
        "nrmf_s": (st, [vp, vp, i64, vp, vp]),
        "nrmf_d": (st, [vp, vp, i64, vp, vp]),
        "nrmp_s": (st, [vp, vp, i64, ctypes.c_float, vp, vp]),
        "nrmf_za_s": (st, [vp, vp, i64, vp, vp]),
        "nrmf_za_d": (st, [vp, vp, i64, vp, vp]),
        "nrmf_es_s": (st, [vp, vp, i64, vp, vp]),
        "nrmf_es_d": (st, [vp, vp, i64, vp, vp]),
        "nrmp_d": (st, [vp, vp, i64, ctypes.c_double, vp, vp]),
        "nrm_batch": (st, [vp, i32, vp, i64, vp, i64, ctypes.c_double, vp, vp, vp, vp]),
        "nrm_batch_graph": (st, [vp, i32, vp, i64, vp, i64, ctypes.c_double, vp, vp, vp, ctypes.POINTER(vp)]),
        "nrm_graph_launch": (st, [vp, vp]),
        "nrm_graph_destroy": (st, [vp]),
        "nrm_host": (st, [vp, i32, vp, i64, ctypes.c_double, vp]),
        "nrm_gen": (st, [i32, vp, i64, u64, u64, i64, i32, i32, vp]),
        "nrm_gen_ragged": (st, [i32, vp, i64, vp, i64, u64, i32, i32, vp]),
        "nrm_kernel_launches": (u64, [vp]),
        "nrm_autotune": (st, [vp, i32, vp, i64, ctypes.POINTER(Tuning)]),
        "nrm_tune": (st, [vp, i32, vp, i64]),
        "nrm_batch_segments": (st, [vp, i32, vp, i64, vp, vp, i64, ctypes.c_double, vp, vp, vp, vp]),
        "nrm_strided": (st, [vp, i32, vp, i64, i64, ctypes.c_double, vp, vp]),
        "nrm_matrix": (st, [vp, i32, vp, i64, i64, i64, ctypes.c_double, vp, vp]),
        "nrm_srv_create": (st, [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_size_t, ctypes.c_int, ctypes.c_int]),
        "nrm_srv_submit": (st, [vp, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]),
        "nrm_srv_poll": (st, [vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32),
                              ctypes.POINTER(ctypes.c_int32)]),
        "nrm_srv_drain": (st, [vp, ctypes.c_double]),
        "nrm_srv_report_get": (st, [vp, ctypes.POINTER(SrvReport)]),
        "nrm_srv_replay": (st, [vp, ctypes.POINTER(Request), i64, vp, vp, ctypes.POINTER(SrvReport)]),
        "nrm_srv_destroy": (st, [vp]),
        "nrm_test_inject_alloc_failures": (None, [ctypes.c_int]),
        "nrm_test_read_tickets": (st, [vp, vp, i64]),
        "nrm_probe_pipe": (st, [i32, i64, i32, vp, ctypes.POINTER(i64), vp]),
        "nrm_shard_range": (st, [i32, i64, i32, i64, ctypes.POINTER(i64), ctypes.POINTER(i64)]),
        "nrm_node_lanes": (st, [vp, i32, vp, i64, ctypes.c_double, vp, vp]),
        "nrm_combine_nodes": (st, [vp, i32, vp, i32, i64, ctypes.c_double, vp, vp]),
    }
    for name, (res, args) in sigs.items():
        if hasattr(L, name):
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
    _lib = L
    return L


def header_functions():
    """Names of the functions include/nrm.h declares."""
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*[A-Za-z_][\w\s\*]*?\b(nrm\w*)\s*\(", src, flags=re.M)
    return sorted(set(names))


def _status_name(s):
    try:
        return load().nrm_status_string(s).decode()
    except Exception:
        return "status %d" % s


# ---------------------------------------------------------------------------
# contexts
# ---------------------------------------------------------------------------

class Context:
    """Owns an nrm_ctx (device workspace, tuning, captured graphs)."""

    def __init__(self, device=0):
        L = load()
        h = ctypes.c_void_p()
        s = L.nrm_create(ctypes.byref(h), int(device))
        if s != NRM_OK:
            raise NrmError(s, "nrm_create(device=%d)" % device)
        self.h = h
        self.device = device
        self._graphs = []

    def close(self):
        if self.h:
            load().nrm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, s, what):
        if s != NRM_OK:
            msg = load().nrm_last_error(self.h).decode() if self.h else ""
            raise NrmError(s, "%s %s" % (what, msg))

    @property
    def tuning(self):
        t = Tuning()
        self.check(load().nrm_get_tuning(self.h, ctypes.byref(t)), "nrm_get_tuning")
        return t

    def tuning_for(self, dtype):
        t = Tuning()
        self.check(load().nrm_get_tuning_for(self.h, dtype, ctypes.byref(t)), "nrm_get_tuning_for")
        return t

    def set_tuning(self, group_log2=None, warps_per_block=None, item_log2=None, blocks_per_sm=None, dtype=None):
        """Set tuning fields (None keeps a field); dtype None = both types."""
        for dt in ((NRM_F32, NRM_F64) if dtype is None else (dtype,)):
            t = self.tuning_for(dt)
            for k, v in (("group_log2", group_log2), ("warps_per_block", warps_per_block),
                         ("item_log2", item_log2), ("blocks_per_sm", blocks_per_sm)):
                if v is not None:
                    setattr(t, k, int(v))
            self.check(load().nrm_set_tuning_for(self.h, dt, ctypes.byref(t)), "nrm_set_tuning_for")

    def autotune(self, dtype, lengths):
        """Pick the fastest tuning for `dtype` on vectors of these lengths
        (one length: the single-vector path; several: the ragged batch)."""
        L = np.ascontiguousarray(np.asarray(lengths, dtype=np.int64).reshape(-1))
        t = Tuning()
        self.check(load().nrm_autotune(self.h, dtype, ctypes.c_void_p(L.ctypes.data), L.size, ctypes.byref(t)),
                   "nrm_autotune")
        return {f: getattr(t, f) for f, _ in Tuning._fields_}

    def reserve(self, nbytes):
        self.check(load().nrm_reserve(self.h, int(nbytes)), "nrm_reserve")

    def workspace_bytes(self, dtype, x_len, B=1):
        return load().nrm_workspace_bytes(self.h, dtype, int(x_len), int(B))

    @property
    def launches(self):
        return load().nrm_kernel_launches(self.h)


_ctxs = {}


def context(device=None):
    import torch
    if device is None:
        device = torch.cuda.current_device()
    if isinstance(device, torch.device):
        device = device.index if device.index is not None else torch.cuda.current_device()
    c = _ctxs.get(device)
    if c is None:
        c = _ctxs[device] = Context(device)
    return c


def _dtype_code(t):
    import torch
    if t.dtype == torch.float64:
        return NRM_F64
    if t.dtype == torch.float32:
        return NRM_F32
    raise TypeError("float32 or float64 tensor required, got %s" % t.dtype)


def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _check_vec(x):
    if not x.is_cuda:
        raise ValueError("x must be a CUDA tensor")
    if x.dim() != 1 or (x.numel() > 1 and x.stride(0) != 1):
        raise ValueError("x must be a contiguous 1-D tensor")


# ---------------------------------------------------------------------------
# entry points
# ---------------------------------------------------------------------------

def nrmp(x, p=2.0, out=None, stream=None, ctx=None):
    """||x||_p of a contiguous 1-D CUDA tensor by the fixed hypot tree."""
    import torch
    _check_vec(x)
    dt = _dtype_code(x)
    c = ctx or context(x.device)
    if out is None:
        out = torch.empty((), dtype=x.dtype, device=x.device)
    L = load()
    xp = ctypes.c_void_p(x.data_ptr() if x.numel() else 0)
    op = ctypes.c_void_p(out.data_ptr())
    s = _stream(stream)
    if dt == NRM_F64:
        r = L.nrmf_d(c.h, xp, x.numel(), op, s) if p == 2.0 else L.nrmp_d(c.h, xp, x.numel(), float(p), op, s)
    else:
        r = L.nrmf_s(c.h, xp, x.numel(), op, s) if p == 2.0 else L.nrmp_s(c.h, xp, x.numel(), float(p), op, s)
    c.check(r, "nrm%s_%s" % ("f" if p == 2.0 else "p", "d" if dt == NRM_F64 else "s"))
    return out


def nrmf(x, out=None, stream=None, ctx=None):
    """xNRMF: the Frobenius norm by the recursive v1_hypot tree."""
    return nrmp(x, 2.0, out, stream, ctx)


def nrmf_es(x, out=None, stream=None, ctx=None):
    """xNRMF with the exponent-scaled hypotenuse K2 (no division) in place of
    v1_hypot throughout the tree: another hypot[f] of Section 2."""
    import torch
    _check_vec(x)
    dt = _dtype_code(x)
    c = ctx or context(x.device)
    if out is None:
        out = torch.empty((), dtype=x.dtype, device=x.device)
    f = load().nrmf_es_d if dt == NRM_F64 else load().nrmf_es_s
    c.check(f(c.h, ctypes.c_void_p(x.data_ptr() if x.numel() else 0), x.numel(), ctypes.c_void_p(out.data_ptr()),
              _stream(stream)), "nrmf_es")
    return out


def nrmf_za(x, out=None, stream=None, ctx=None):
    """xNRMF with the algorithm A (correctly rounded hypot) for the final
    reduction of the lane partials: the paper's recommended pairing."""
    import torch
    _check_vec(x)
    dt = _dtype_code(x)
    c = ctx or context(x.device)
    if out is None:
        out = torch.empty((), dtype=x.dtype, device=x.device)
    f = load().nrmf_za_d if dt == NRM_F64 else load().nrmf_za_s
    c.check(f(c.h, ctypes.c_void_p(x.data_ptr() if x.numel() else 0), x.numel(), ctypes.c_void_p(out.data_ptr()),
              _stream(stream)), "nrmf_za")
    return out


def _p_args(p, B, device):
    """(p, p_dev pointer): a scalar p for every vector, or a CUDA float64
    tensor of B values, one p per vector (then the scalar is ignored)."""
    import torch
    if isinstance(p, torch.Tensor):
        if p.dtype != torch.float64 or not p.is_cuda or p.numel() != B or not p.is_contiguous():
            raise ValueError("a per-vector p must be a contiguous float64 CUDA tensor of B values")
        return 2.0, ctypes.c_void_p(p.data_ptr() if B else 0)
    return float(p), None


def nrm_batch(x, offsets, p=2.0, out=None, status=None, stream=None, ctx=None):
    """Norms of x[offsets[i]:offsets[i+1]] for all i; returns (out, status).
    p: one value for all vectors, or a float64 CUDA tensor of one per vector."""
    import torch
    _check_vec(x)
    dt = _dtype_code(x)
    if offsets.dtype != torch.int64 or not offsets.is_cuda or not offsets.is_contiguous():
        raise ValueError("offsets must be a contiguous int64 CUDA tensor")
    B = offsets.numel() - 1
    c = ctx or context(x.device)
    if out is None:
        out = torch.empty(max(B, 0), dtype=x.dtype, device=x.device)
    if status is None:
        status = torch.empty(max(B, 0), dtype=torch.int32, device=x.device)
    ps, pd = _p_args(p, B, x.device)
    r = load().nrm_batch(c.h, dt, ctypes.c_void_p(x.data_ptr() if x.numel() else 0), x.numel(),
                         ctypes.c_void_p(offsets.data_ptr()), B, ps, pd, ctypes.c_void_p(out.data_ptr()),
                         ctypes.c_void_p(status.data_ptr()), _stream(stream))
    c.check(r, "nrm_batch")
    return out, status


class BatchGraph:
    """A ragged batch captured once as a CUDA graph (plan + tree kernel)."""

    def __init__(self, x, offsets, p=2.0, out=None, status=None, ctx=None):
        import torch
        _check_vec(x)
        dt = _dtype_code(x)
        B = offsets.numel() - 1
        self.ctx = ctx or context(x.device)
        self.x, self.offsets = x, offsets
        self.out = out if out is not None else torch.empty(B, dtype=x.dtype, device=x.device)
        self.status = status if status is not None else torch.empty(B, dtype=torch.int32, device=x.device)
        h = ctypes.c_void_p()
        ps, pd = _p_args(p, B, x.device)
        self.p = p  # a per-vector p tensor is read by every replay
        r = load().nrm_batch_graph(self.ctx.h, dt, ctypes.c_void_p(x.data_ptr()), x.numel(),
                                   ctypes.c_void_p(offsets.data_ptr()), B, ps, pd,
                                   ctypes.c_void_p(self.out.data_ptr()), ctypes.c_void_p(self.status.data_ptr()),
                                   ctypes.byref(h))
        self.ctx.check(r, "nrm_batch_graph")
        self.h = h

    def launch(self, stream=None):
        self.ctx.check(load().nrm_graph_launch(self.h, _stream(stream)), "nrm_graph_launch")
        return self.out, self.status

    def close(self):
        if self.h:
            load().nrm_graph_destroy(self.h)
            self.h = None


def nrm_batch_graph(x, offsets, p=2.0, out=None, status=None, ctx=None):
    return BatchGraph(x, offsets, p, out, status, ctx)


def nrm_host(x_host, p=2.0, ctx=None, device=0):
    """End to end: host array in (numpy or CPU tensor, ideally pinned), the
    norm as a Python float out; host->device copies overlap the tree."""
    import torch
    if isinstance(x_host, np.ndarray):
        a = np.ascontiguousarray(x_host)
        ptr, n, isd = a.ctypes.data, a.size, a.dtype == np.float64
        if a.dtype not in (np.float64, np.float32):
            raise TypeError("float32 or float64 required")
    else:
        if x_host.is_cuda or not x_host.is_contiguous():
            raise ValueError("x_host must be a contiguous CPU tensor")
        ptr, n, isd = x_host.data_ptr(), x_host.numel(), x_host.dtype == torch.float64
    dt = NRM_F64 if isd else NRM_F32
    c = ctx or context(device)
    res = (ctypes.c_double if isd else ctypes.c_float)()
    r = load().nrm_host(c.h, dt, ctypes.c_void_p(ptr), n, float(p), ctypes.byref(res))
    c.check(r, "nrm_host")
    return res.value


def nrm_gen(n, seed=0, vec=0, dtype=None, emin=-20, emax=20, start=0, device=None, out=None, stream=None):
    """Seeded synthetic vector on the device (same definition as inputs.vector)."""
    import torch
    dtype = dtype or torch.float64
    if out is None:
        out = torch.empty(n, dtype=dtype, device=device or "cuda")
    dt = _dtype_code(out)
    r = load().nrm_gen(dt, ctypes.c_void_p(out.data_ptr() if n else 0), int(n), int(seed) & (2 ** 64 - 1),
                       int(vec) & (2 ** 64 - 1), int(start), int(emin), int(emax), _stream(stream))
    if r != NRM_OK:
        raise NrmError(r, "nrm_gen")
    return out


def nrm_gen_ragged(offsets, seed=0, dtype=None, emin=-20, emax=20, out=None, stream=None):
    import torch
    dtype = dtype or torch.float64
    n = int(offsets[-1].item())
    if out is None:
        out = torch.empty(n, dtype=dtype, device=offsets.device)
    dt = _dtype_code(out)
    r = load().nrm_gen_ragged(dt, ctypes.c_void_p(out.data_ptr() if n else 0), out.numel(),
                              ctypes.c_void_p(offsets.data_ptr()), offsets.numel() - 1, int(seed) & (2 ** 64 - 1),
                              int(emin), int(emax), _stream(stream))
    if r != NRM_OK:
        raise NrmError(r, "nrm_gen_ragged")
    return out


def nrm_batch_segments(x, starts, lengths, p=2.0, out=None, status=None, stream=None, ctx=None):
    """Norms of x[starts[i] : starts[i] + lengths[i]] (device int64 arrays)."""
    import torch
    _check_vec(x)
    dt = _dtype_code(x)
    B = starts.numel()
    c = ctx or context(x.device)
    if out is None:
        out = torch.empty(B, dtype=x.dtype, device=x.device)
    if status is None:
        status = torch.empty(B, dtype=torch.int32, device=x.device)
    ps, pd = _p_args(p, B, x.device)
    r = load().nrm_batch_segments(c.h, dt, ctypes.c_void_p(x.data_ptr()), x.numel(),
                                  ctypes.c_void_p(starts.data_ptr()), ctypes.c_void_p(lengths.data_ptr()), B,
                                  ps, pd, ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(status.data_ptr()),
                                  _stream(stream))
    c.check(r, "nrm_batch_segments")
    return out, status


class Server:
    """Continuous-batching server (nrm_srv_*): admission under a device
    memory budget, steps on several streams, p50/p99 latency."""

    def __init__(self, budget_bytes=8 << 30, nstreams=2, max_batch=1024, device=0):
        h = ctypes.c_void_p()
        s = load().nrm_srv_create(ctypes.byref(h), int(device), int(budget_bytes), int(nstreams), int(max_batch))
        if s != NRM_OK:
            raise NrmError(s, "nrm_srv_create")
        self.h = h
        self._keep = []

    def submit(self, n, dtype=NRM_F64, p=2.0, seed=0, emin=-20, emax=20, x_host=None):
        """Submit one request; the input is x_host (numpy, kept alive until
        done) or generated on the device from (seed, request id)."""
        ptr = None
        if x_host is not None:
            x_host = np.ascontiguousarray(x_host)
            self._keep.append(x_host)
            ptr = x_host.ctypes.data
            n = x_host.size
            dtype = NRM_F64 if x_host.dtype == np.float64 else NRM_F32
        req = Request(int(dtype), int(emin), int(emax), float(p), int(n), ptr, int(seed), 0.0)
        rid = ctypes.c_uint64()
        r = load().nrm_srv_submit(self.h, ctypes.byref(req), ctypes.byref(rid))
        if r != NRM_OK:
            raise NrmError(r, "nrm_srv_submit")
        return rid.value

    def poll(self, rid):
        v, st, done = ctypes.c_double(), ctypes.c_int32(), ctypes.c_int32()
        r = load().nrm_srv_poll(self.h, int(rid), ctypes.byref(v), ctypes.byref(st), ctypes.byref(done))
        if r != NRM_OK:
            raise NrmError(r, "nrm_srv_poll")
        return (v.value, st.value) if done.value else None

    def drain(self, timeout_s=600.0):
        r = load().nrm_srv_drain(self.h, float(timeout_s))
        if r != NRM_OK:
            raise NrmError(r, "nrm_srv_drain")

    def report(self):
        rep = SrvReport()
        load().nrm_srv_report_get(self.h, ctypes.byref(rep))
        return rep.as_dict()

    def replay(self, reqs):
        """Replay a trace (array of Request with arrival_s); returns
        (norms, latency_ms, report)."""
        n = len(reqs)
        norms = np.zeros(n, np.float64)
        lat = np.zeros(n, np.float64)
        rep = SrvReport()
        r = load().nrm_srv_replay(self.h, reqs, n, ctypes.c_void_p(norms.ctypes.data),
                                  ctypes.c_void_p(lat.ctypes.data), ctypes.byref(rep))
        if r != NRM_OK:
            raise NrmError(r, "nrm_srv_replay")
        return norms, lat, rep.as_dict()

    def close(self):
        if self.h:
            load().nrm_srv_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def serving_trace(rate, seconds, seed=0, min_log2=4, max_log2=24, p_probs=(0.8, 0.1, 0.1), ps=(2.0, 1.5, 3.0),
                  max_requests=None):
    """Poisson arrivals at `rate` per second for `seconds`; lengths
    log-uniform in [2^min_log2, 2^max_log2]; FP32/FP64 with probability 1/2;
    p from `ps` with probabilities `p_probs`.  Returns a ctypes array of
    Request (inputs generated on the device, keyed by request id)."""
    from . import inputs
    count = int(rate * seconds * 1.2) + 16
    k = inputs.key(seed, 0xFFFFFFF0)
    u = (inputs.draw(k, np.arange(4 * count, dtype=np.uint64)) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    u = u.reshape(count, 4)
    gaps = -np.log1p(-u[:, 0]) / rate
    t = np.cumsum(gaps)
    m = int(np.searchsorted(t, seconds))
    if max_requests is not None:
        m = min(m, max_requests)
    L = np.floor(np.exp2(min_log2 + (max_log2 - min_log2) * u[:m, 1])).astype(np.int64)
    dts = np.where(u[:m, 2] < 0.5, NRM_F32, NRM_F64)
    cp = np.cumsum(p_probs)
    pidx = np.searchsorted(cp, u[:m, 3] * cp[-1], side="right")
    pv = np.asarray(ps, np.float64)[np.minimum(pidx, len(ps) - 1)]
    rec = np.zeros(m, dtype=request_dtype())
    rec["dtype"], rec["emin"], rec["emax"] = dts, -20, 20
    rec["p"], rec["n"], rec["seed"], rec["arrival_s"] = pv, L, seed, t[:m]
    return (Request * m).from_buffer(rec)  # shares (and keeps alive) rec's memory


def request_dtype():
    """numpy record layout of the C struct nrm_request (same offsets)."""
    names = [f for f, _ in Request._fields_]
    fmt = {ctypes.c_int32: np.int32, ctypes.c_double: np.float64, ctypes.c_int64: np.int64,
           ctypes.c_void_p: np.uint64, ctypes.c_uint64: np.uint64}
    return np.dtype({"names": names, "formats": [fmt[t] for _, t in Request._fields_],
                     "offsets": [getattr(Request, f).offset for f in names], "itemsize": ctypes.sizeof(Request)})


def trace_records(reqs):
    """A numpy record view of a ctypes array of Request (no copy)."""
    return np.frombuffer(reqs, dtype=request_dtype())


def nrm_strided(buf, n, incx, p=2.0, out=None, stream=None, ctx=None):
    """Norm of the n-element strided vector in the CUDA tensor buf (element
    0 at buf's start; incx < 0 takes the elements backwards, as BLAS)."""
    import torch
    dt = _dtype_code(buf)
    c = ctx or context(buf.device)
    if out is None:
        out = torch.empty((), dtype=buf.dtype, device=buf.device)
    r = load().nrm_strided(c.h, dt, ctypes.c_void_p(buf.data_ptr()), int(n), int(incx), float(p),
                           ctypes.c_void_p(out.data_ptr()), _stream(stream))
    c.check(r, "nrm_strided")
    return out


def nrm_matrix(buf, M, N, lda, p=2.0, out=None, stream=None, ctx=None):
    """Norm of the column-major M x N matrix stored in the CUDA tensor buf
    with leading dimension lda (Section 3.1)."""
    import torch
    dt = _dtype_code(buf)
    c = ctx or context(buf.device)
    if out is None:
        out = torch.empty((), dtype=buf.dtype, device=buf.device)
    r = load().nrm_matrix(c.h, dt, ctypes.c_void_p(buf.data_ptr()), int(M), int(N), int(lda), float(p),
                          ctypes.c_void_p(out.data_ptr()), _stream(stream))
    c.check(r, "nrm_matrix")
    return out


def shard_range(n, dg, j, dtype=NRM_F64):
    """(first, count): the elements of node j at depth dg of the row tree of
    a vector of n elements -- the part device j of 2^dg holds."""
    first, count = ctypes.c_int64(), ctypes.c_int64()
    r = load().nrm_shard_range(int(dtype), int(n), int(dg), int(j), ctypes.byref(first), ctypes.byref(count))
    if r != NRM_OK:
        raise NrmError(r, "nrm_shard_range")
    return first.value, count.value


def node_lanes(x, p=2.0, out=None, stream=None, ctx=None):
    """The P lane partials (one 512-byte row) of a node held as the 1-D CUDA
    tensor x (its elements in order)."""
    import torch
    _check_vec(x)
    dt = _dtype_code(x)
    c = ctx or context(x.device)
    if out is None:
        out = torch.empty(P_LANES[dt], dtype=x.dtype, device=x.device)
    c.check(load().nrm_node_lanes(c.h, dt, ctypes.c_void_p(x.data_ptr() if x.numel() else 0), x.numel(), float(p),
                                  ctypes.c_void_p(out.data_ptr()), _stream(stream)), "nrm_node_lanes")
    return out


def combine_nodes(lanes, dg, n, p=2.0, out=None, stream=None, ctx=None):
    """||x||_p from the 2^dg node rows of x (a CUDA tensor of 2^dg x P
    elements in node order; overwritten) for a vector of n elements."""
    import torch
    dt = _dtype_code(lanes)
    if not lanes.is_cuda or not lanes.is_contiguous() or lanes.numel() != (1 << dg) * P_LANES[dt]:
        raise ValueError("lanes must be a contiguous CUDA tensor of 2^dg x P elements")
    c = ctx or context(lanes.device)
    if out is None:
        out = torch.empty((), dtype=lanes.dtype, device=lanes.device)
    c.check(load().nrm_combine_nodes(c.h, dt, ctypes.c_void_p(lanes.data_ptr()), int(dg), int(n), float(p),
                                     ctypes.c_void_p(out.data_ptr()), _stream(stream)), "nrm_combine_nodes")
    return out


def nrm_sharded(x_local, n, p=2.0, group=None, ctx=None):
    """||x||_p of a vector of n elements sharded over the 2^dg ranks of a
    torch.distributed group (rank j holds shard_range(n, dg, j)'s elements
    as the CUDA tensor x_local): each rank computes its node's lanes, the
    512-byte rows are all-gathered (through host memory, so any backend
    works), and every rank combines them; bitwise the one-device result."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    dg = world.bit_length() - 1
    if world != 1 << dg:
        raise ValueError("the group size must be a power of two")
    mine = node_lanes(x_local, p, ctx=ctx).cpu()
    rows = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(rows, mine, group=group)
    lanes = torch.cat(rows).to(x_local.device)
    return combine_nodes(lanes, dg, n, p, ctx=ctx)


PIPE_DFMA, PIPE_DMUL, PIPE_FFMA = 0, 1, 2


def probe_pipe(kind=PIPE_DFMA, iters=4096, blocks_per_sm=8, reps=3, device=None):
    """Measured throughput of one SM pipe (nrm_probe_pipe): operations per
    second over all SMs, the best of `reps` launches timed with CUDA events
    on the current stream after one warm-up launch."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
    sink = torch.zeros(1, dtype=torch.float64, device=dev)
    ops = ctypes.c_int64()
    L = load()

    def launch():
        r = L.nrm_probe_pipe(int(kind), int(iters), int(blocks_per_sm), ctypes.c_void_p(sink.data_ptr()),
                             ctypes.byref(ops), _stream(None))
        if r != NRM_OK:
            raise NrmError(r, "nrm_probe_pipe")

    launch()
    torch.cuda.synchronize()
    best = None
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        launch()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    return ops.value / (best * 1e-3)


def nrmf_complex(z, out=None, stream=None, ctx=None):
    """Frobenius norm of a complex CUDA tensor: |z|^2 = Re^2 + Im^2 (Section 1),
    so it is xNRMF of the interleaved real view of 2n elements."""
    import torch
    r = torch.view_as_real(z.contiguous()).reshape(-1)
    return nrmf(r, out=out, stream=stream, ctx=ctx)
