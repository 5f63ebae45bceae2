"""GPU parity: the CUDA path (through the C ABI) against the oracle.

Bitwise for every result (the tree and every rounding are fixed), NaN-ness
for NaN results; accuracy against the binary128 reference with the stated
tolerances (1e-14 for binary64, 5e-6 for binary32) and the Eq. ubr bound.
"""
import math
import random

import numpy as np
import pytest

import oracle
from paper_2509_06220_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
EPS_D, EPS_S = 2.0 ** -53, 2.0 ** -24


@pytest.fixture(scope="module")
def nrm():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2509_06220_gb300 as m
    assert torch.cuda.is_available()
    return m


DEV = "cuda:0"
TD = {np.float64: torch.float64, np.float32: torch.float32}


def bits_equal(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    if a.dtype != b.dtype or a.shape != b.shape:
        return False
    an, bn = np.isnan(a), np.isnan(b)
    if (an != bn).any():
        return False
    return a[~an].tobytes() == b[~bn].tobytes()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


def gpu_norms(nrm, x_dev, ns, p=2.0, starts=None):
    """Norms of x_dev[s:s+n] for the given (start, n) list, one call each,
    results gathered on the device and copied back once."""
    out = torch.empty(len(ns), dtype=x_dev.dtype, device=DEV)
    for i, n in enumerate(ns):
        s = 0 if starts is None else starts[i]
        nrm.nrmp(x_dev[s:s + n], p, out=out[i])
    return out.cpu().numpy()


# ---------------------------------------------------------------------------
# inputs
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_device_generator_matches_host(nrm, dt):
    for seed, vec, emin, emax, start in ((0, 0, -20, 20, 0), (3, 7, -8, 8, 12345), (1, 2, 125, 125, 0),
                                         (9, 1, -126, -120, 5)):
        if dt == np.float64 and emin == 125:
            emin = emax = 1020
        n = (1 << 18) + 13
        h = inputs.vector(n, seed, vec, dt, emin, emax, start=start)
        d = nrm.nrm_gen(n, seed, vec, TD[dt], emin, emax, start=start, device=DEV).cpu().numpy()
        assert h.tobytes() == d.tobytes()
    x, off = inputs.ragged_batch(50, seed=4, dtype=dt, max_log2=10)
    d = nrm.nrm_gen_ragged(dev(off), seed=4, dtype=TD[dt]).cpu().numpy()
    assert x.tobytes() == d.tobytes()


# ---------------------------------------------------------------------------
# single vectors
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_all_small_n(nrm, dt):
    """Every n up to 40 rows (several groups, items and a ragged tail)."""
    P = 64 if dt == np.float64 else 128
    ns = list(range(0, 40 * P + 2))
    x = inputs.vector(max(ns), seed=1, vec=3, dtype=dt)
    got = gpu_norms(nrm, dev(x), ns)
    want = np.array([oracle.nrm(x[:n]) for n in ns], dtype=dt)
    bad = [n for n, g, w in zip(ns, got, want) if not bits_equal(g, w)]
    assert not bad, bad[:10]


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_misaligned_starts(nrm, dt):
    """Z^u == Z^a (Section 3): any element offset gives the same bits as a
    copy at an aligned address."""
    x = inputs.vector(300000, seed=2, vec=3, dtype=dt)
    xd = dev(x)
    ns, starts = [], []
    r = random.Random(3)
    for s in range(0, 9):
        for n in (1, 5, 63, 64, 65, 127, 128, 129, 1000, 4097, r.randint(1, 250000)):
            ns.append(n)
            starts.append(s)
    got = gpu_norms(nrm, xd, ns, starts=starts)
    for g, n, s in zip(got, ns, starts):
        assert bits_equal(g, oracle.nrm(x[s:s + n])), (n, s)
        aligned = dev(x[s:s + n].copy())
        assert bits_equal(g, nrm.nrmf(aligned).item() if dt == np.float64 else np.float32(nrm.nrmf(aligned).item()))


@pytest.mark.parametrize("plant", ["none", "low_edge", "inf"])
@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_misaligned_long_vectors(nrm, dt, plant):
    """Long vectors at element offsets 1-3 (not 16-byte aligned: their work
    items fill the shared-memory ring one element at a time), with full and
    partial items and a ragged tail, optionally with values below the
    branch-free range or an inf planted (the item falls back to the general
    form): bitwise equal to the oracle and to an aligned copy."""
    rng = np.random.default_rng(7 + len(plant))
    buf = inputs.vector((1 << 22) + 64, seed=8, vec=2, dtype=dt)
    lo = -88 if dt == np.float32 else -500
    for s, n in ((1, 1 << 22), (2, 3 * (1 << 20) + 17), (3, (1 << 22) - 1000)):
        x = buf[s:s + n].copy()
        if plant == "low_edge":
            q = rng.choice(n, 8, replace=False)
            x[q] = (rng.uniform(1, 2, 8) * 2.0 ** rng.integers(lo - 3, lo + 3, 8)).astype(dt)
        elif plant == "inf":
            x[rng.integers(0, n)] = np.inf
        host = np.empty(n + 8, dtype=dt)
        host[s:s + n] = x
        xd = dev(host)[s:s + n]
        got = nrm.nrmf(xd).cpu().numpy()
        want = oracle.nrm(x)
        assert bits_equal(np.asarray(got, dt), np.asarray(want, dt)), (s, n, got, want)
        assert bits_equal(np.asarray(nrm.nrmf(dev(x)).cpu().numpy(), dt), np.asarray(want, dt))


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_sizes_primes_powers(nrm, dt):
    ns = []
    for k in range(1, 23):
        ns += [(1 << k) - 1, 1 << k, (1 << k) + 1]
    ns += [1009, 65537, 999983, 1299709, 3 * (1 << 20) + 7]
    x = inputs.vector(max(ns), seed=3, vec=0, dtype=dt)
    got = gpu_norms(nrm, dev(x), ns)
    for g, n in zip(got, ns):
        assert bits_equal(g, oracle.nrm(x[:n])), n


@pytest.mark.parametrize("dt", [np.float64, np.float32])
@pytest.mark.parametrize("p", [1.0, 1.5, 3.0, 7.5, 0.5, 2.0 / 3.0, math.inf, math.pi, 2.0 ** 30, 2.0 ** 60])
def test_pnorm_parity(nrm, dt, p):
    ns = [1, 2, 63, 64, 65, 129, 1000, 8191, 65536, 100003]
    x = inputs.vector(max(ns), seed=4, vec=1, dtype=dt, emin=-8, emax=8)
    got = gpu_norms(nrm, dev(x), ns, p=p)
    for g, n in zip(got, ns):
        assert bits_equal(g, oracle.nrm(x[:n], p)), (n, p)


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_tuning_invariance(nrm, dt):
    """No tuning knob changes a bit (the tree is fixed by P alone)."""
    ns = [1, 100, 5000, 123457, 1 << 20, (1 << 21) + 3]
    x = inputs.vector(max(ns), seed=5, vec=0, dtype=dt)
    xd = dev(x)
    want = np.array([oracle.nrm(x[:n]) for n in ns], dtype=dt)
    ctx = nrm.Context(0)
    try:
        for g in (2, 3):
            for wpb in (4, 8, 16):
                for k in (g, g + 2, g + 4, g + 10):
                    for bps in (1, 4):
                        ctx.set_tuning(g, wpb, k, bps)
                        out = torch.empty(len(ns), dtype=xd.dtype, device=DEV)
                        for i, n in enumerate(ns):
                            nrm.nrmp(xd[:n], 2.0, out=out[i], ctx=ctx)
                        assert bits_equal(out.cpu().numpy(), want), (g, wpb, k, bps)
    finally:
        ctx.close()


def test_repeat_stability(nrm):
    """200 launches of the same call give the same bits (a race would show)."""
    x = dev(inputs.vector((1 << 22) + 77, seed=6, vec=0))
    out = torch.empty(200, dtype=torch.float64, device=DEV)
    for i in range(200):
        nrm.nrmf(x, out=out[i])
    o = out.cpu().numpy()
    assert len(set(o.tobytes()[i * 8:(i + 1) * 8] for i in range(200))) == 1


def test_config0_bitwise_and_accuracy(nrm):
    """n = 2^20 binary64, e in [-20, 20], seed 0: bitwise and relerr."""
    x = inputs.vector(1 << 20, seed=0, vec=0)
    g = nrm.nrmf(dev(x)).item()
    assert bits_equal(np.float64(g), oracle.nrm(x))
    e = oracle.relerr(g, x, nthreads=8)
    assert e <= 1e-14
    hi, lo = oracle.ub_relerr(oracle.tree_depth(x.size, 64))
    assert e <= (hi + lo) * EPS_D


def test_special_values(nrm):
    """Infinities give +inf; NaNs follow Listing 2 literally (NaN-ness
    compared); subnormal inputs are kept (no flush to zero)."""
    for dt in (np.float64, np.float32):
        x = inputs.vector(10000, seed=7, vec=0, dtype=dt)
        y = x.copy()
        y[1234] = np.inf
        assert math.isinf(nrm.nrmf(dev(y)).item())
        for pos in (0, 1, 63, 64, 5000, 9999):
            z = x.copy()
            z[pos] = np.nan
            for p in (2.0, 1.0, 3.0, math.inf):
                assert bits_equal(np.asarray(nrm.nrmp(dev(z), p).item(), dtype=dt), oracle.nrm(z, p)), (pos, p)
        tiny = np.finfo(dt).smallest_subnormal
        s = (np.arange(1, 3001) % 7).astype(dt) * tiny
        for p in (2.0, 1.0, 3.0):
            assert bits_equal(np.asarray(nrm.nrmp(dev(s), p).item(), dtype=dt), oracle.nrm(s, p))


def test_invalid_arguments(nrm):
    import ctypes
    L = nrm.load()
    c = nrm.context(0)
    vp = ctypes.c_void_p
    o = torch.empty(4, dtype=torch.float64, device=DEV)
    x = torch.ones(8, dtype=torch.float64, device=DEV)
    assert L.nrmf_d(c.h, vp(x.data_ptr()), -1, vp(o.data_ptr()), None) == nrm.NRM_EINVAL
    assert L.nrmf_d(c.h, vp(0), 5, vp(o.data_ptr()), None) == nrm.NRM_EINVAL
    assert L.nrmf_d(c.h, vp(x.data_ptr()), 5, vp(0), None) == nrm.NRM_EINVAL
    assert L.nrmp_d(c.h, vp(x.data_ptr()), 5, 0.0, vp(o.data_ptr()), None) == nrm.NRM_EINVAL
    assert L.nrmp_d(c.h, vp(x.data_ptr()), 5, -2.0, vp(o.data_ptr()), None) == nrm.NRM_EINVAL
    assert L.nrmp_d(c.h, vp(x.data_ptr()), 5, float("nan"), vp(o.data_ptr()), None) == nrm.NRM_EINVAL
    assert L.nrm_batch(c.h, 5, vp(x.data_ptr()), 8, vp(0), 1, 2.0, None, vp(o.data_ptr()), vp(0), None) == nrm.NRM_EINVAL
    # n == 0 gives +0
    o.fill_(7.0)
    assert L.nrmf_d(c.h, vp(0), 0, vp(o.data_ptr()), None) == nrm.NRM_OK
    torch.cuda.synchronize()
    assert o[0].item() == 0.0 and math.copysign(1, o[0].item()) > 0


def test_alloc_failure_is_reported(nrm):
    """Host-side fault injection: a failed workspace allocation returns
    NRM_ENOMEM and leaves the context usable."""
    L = nrm.load()
    ctx = nrm.Context(0)
    try:
        # the smallest power of two whose workspace exceeds what a fresh
        # context holds (4 MiB)
        n = 1 << 24
        while ctx.workspace_bytes(nrm.NRM_F64, n) <= (4 << 20):
            n <<= 1
        assert n <= 1 << 28
        x = nrm.nrm_gen(n, 8, 0, torch.float64, device=DEV)
        L.nrm_test_inject_alloc_failures(1)
        with pytest.raises(nrm.NrmError) as ei:
            nrm.nrmf(x, ctx=ctx)
        assert ei.value.status == nrm.NRM_ENOMEM
        L.nrm_test_inject_alloc_failures(0)
        g = nrm.nrmf(x, ctx=ctx).item()
        assert bits_equal(np.float64(g), oracle.nrm(x.cpu().numpy()))
    finally:
        L.nrm_test_inject_alloc_failures(0)
        ctx.close()


# ---------------------------------------------------------------------------
# full size (n = 2^28), probes
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_full_size_2e28(nrm, dt):
    """n = 2^28, seeds 1..3 (binary64 2 GiB / binary32 1 GiB): bitwise
    against the oracle on seed 1 and relerr against binary128 within the
    tolerance and the Eq. ubr bound on every seed."""
    n = 1 << 28
    P = 64 if dt == np.float64 else 128
    tol = 1e-14 if dt == np.float64 else 5e-6
    hi, lo = oracle.ub_relerr(oracle.tree_depth(n, P), "D" if dt == np.float64 else "S")
    bound = (hi + lo) * (EPS_D if dt == np.float64 else EPS_S)
    for seed in (1, 2, 3):
        xd = nrm.nrm_gen(n, seed, 0, TD[dt], device=DEV)
        g = nrm.nrmf(xd).item()
        x = xd.cpu().numpy()
        del xd
        if seed == 1:
            assert bits_equal(np.asarray(g, dtype=dt), oracle.nrm(x))
        e = oracle.relerr(g, x, nthreads=16)
        assert e <= tol and e <= bound, (seed, e)
        del x
        torch.cuda.empty_cache()


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_overflow_underflow_probes_full_size(nrm, dt):
    """Probes at n = 2^28: (i) entries in [2^1020, 2^1021) (D) /
    [2^125, 2^126) (S): the true norm exceeds the range, result +inf, no
    NaN; (iii) data x 2^k for the largest k keeping the result finite is
    exactly 2^k times the unscaled result; underflow: data x 2^-k with every
    entry still normal is exactly 2^-k times the result."""
    n = 1 << 28
    big = 1020 if dt == np.float64 else 125
    xd = nrm.nrm_gen(n, 2, 0, TD[dt], emin=big, emax=big, device=DEV)
    g = nrm.nrmf(xd).item()
    assert math.isinf(g) and g > 0
    del xd
    xd = nrm.nrm_gen(n, 3, 0, TD[dt], device=DEV)
    v = nrm.nrmf(xd).item()
    info = np.finfo(dt)
    kmax = int(math.floor(math.log2(float(info.max)) - math.log2(v))) - 1
    kmin = -int(info.minexp) - 20  # entries >= 2^-20 stay >= the smallest normal: 1002 (D), 106 (S)
    scale_up = torch.tensor(2.0 ** kmax, dtype=TD[dt], device=DEV)
    vu = nrm.nrmf(xd * scale_up).item()
    assert np.asarray(vu, dtype=dt) == np.asarray(v, dtype=dt) * np.asarray(2.0 ** kmax, dtype=dt)
    scale_dn = torch.tensor(2.0 ** (-kmin), dtype=TD[dt], device=DEV)
    xs = xd * scale_dn
    assert float(xs.abs().min()) >= float(info.tiny)
    vd = nrm.nrmf(xs).item()
    assert np.asarray(vd, dtype=dt) == np.asarray(v, dtype=dt) * np.asarray(2.0 ** (-kmin), dtype=dt)


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_underflow_probe_smallest_normal(nrm, dt):
    """All entries in [2^-1022, 2^-1021) (D) / [2^-126, 2^-125) (S): squares
    underflow, the tree does not; bitwise against the oracle and accurate
    against binary128."""
    lo_e = -1022 if dt == np.float64 else -126
    n = (1 << 22) + 5
    xd = nrm.nrm_gen(n, 4, 0, TD[dt], emin=lo_e, emax=lo_e, device=DEV)
    g = nrm.nrmf(xd).item()
    x = xd.cpu().numpy()
    assert bits_equal(np.asarray(g, dtype=dt), oracle.nrm(x))
    hi, _ = oracle.ref_q128(x, nthreads=8)
    assert abs(g - hi) / hi <= (1e-14 if dt == np.float64 else 5e-6)


# ---------------------------------------------------------------------------
# host buffers (end to end)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_nrm_host_matches_device(nrm, dt):
    for n in (0, 1, 1000, (1 << 22) + 3):
        x = inputs.vector(n, seed=9, vec=0, dtype=dt)
        for p in (2.0, 3.0):
            h = nrm.nrm_host(x, p)
            assert bits_equal(np.asarray(h, dtype=dt), oracle.nrm(x, p) if n else dt(0)), (n, p)
    xp = torch.from_numpy(inputs.vector(1 << 20, seed=9, vec=1, dtype=dt)).pin_memory()
    assert bits_equal(np.asarray(nrm.nrm_host(xp), dtype=dt), oracle.nrm(xp.numpy()))


# ---------------------------------------------------------------------------
# ragged batches
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dt", [np.float64, np.float32])
@pytest.mark.parametrize("p", [2.0, 1.0, 3.0])
def test_batch_matches_oracle(nrm, dt, p):
    x, off = inputs.ragged_batch(700, seed=10, dtype=dt, max_log2=16)
    out, st = nrm.nrm_batch(dev(x), dev(off), p)
    torch.cuda.synchronize()
    assert (st.cpu().numpy() == 0).all()
    assert bits_equal(out.cpu().numpy(), oracle.nrm_batch(x, off, p))


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_batch_config2_sampled(nrm, dt):
    """4096 vectors, lengths log-uniform in [1, 2^18] (about 86 M elements),
    generated on the device; 200 sampled vectors against the oracle, and the
    whole batch equal to one call per vector."""
    L = inputs.ragged_lengths(4096, seed=0)
    off = np.zeros(4097, np.int64)
    np.cumsum(L, out=off[1:])
    offd = dev(off)
    xd = nrm.nrm_gen_ragged(offd, seed=0, dtype=TD[dt])
    out, st = nrm.nrm_batch(xd, offd)
    single = torch.empty(4096, dtype=TD[dt], device=DEV)
    for i in range(4096):
        nrm.nrmf(xd[off[i]:off[i + 1]], out=single[i])
    o = out.cpu().numpy()
    assert (st.cpu().numpy() == 0).all()
    assert bits_equal(o, single.cpu().numpy())
    x = xd.cpu().numpy()
    for i in random.Random(1).sample(range(4096), 200):
        assert bits_equal(o[i], oracle.nrm(x[off[i]:off[i + 1]])), i


def test_batch_bad_offsets(nrm):
    x = inputs.vector(1000, seed=11, vec=0)
    off = np.array([0, 10, 5, 300, 300, 1200, 1000, -3, 1000], np.int64)
    out, st = nrm.nrm_batch(dev(x), dev(off))
    o, s = out.cpu().numpy(), st.cpu().numpy()
    want_ok = {0: (0, 10), 2: (5, 300), 3: (300, 300)}
    for i in range(len(off) - 1):
        if i in want_ok:
            a, b = want_ok[i]
            assert s[i] == 0
            assert bits_equal(o[i], oracle.nrm(x[a:b]))
        else:
            assert s[i] == nrm.NRM_EINVAL and math.isnan(o[i]), i


def test_batch_overlap_guard(nrm):
    """Overlapping offsets that would need more workspace than x_len
    implies: every vector reports NRM_ENOMEM, nothing is computed."""
    x = inputs.vector(1 << 16, seed=12, vec=0)
    n = x.size
    off = np.array([0, n, 0, n, 0, n, 0, n, 0, n], np.int64)
    out, st = nrm.nrm_batch(dev(x), dev(off))
    s = st.cpu().numpy()
    assert set(s[::2].tolist()) <= {0, nrm.NRM_ENOMEM}
    ok = s == 0
    o = out.cpu().numpy()
    for i in np.nonzero(ok)[0]:
        a, b = off[i], off[i + 1]
        assert bits_equal(o[i], oracle.nrm(x[a:b]))


def test_batch_graph_replay(nrm):
    x, off = inputs.ragged_batch(300, seed=13, max_log2=15)
    xd, offd = dev(x), dev(off)
    g = nrm.nrm_batch_graph(xd, offd)
    out, st = g.launch()
    torch.cuda.synchronize()
    assert bits_equal(out.cpu().numpy(), oracle.nrm_batch(x, off))
    # new data in the same buffers: the replay recomputes
    nrm.nrm_gen_ragged(offd, seed=14, out=xd)
    out2, _ = g.launch()
    torch.cuda.synchronize()
    assert bits_equal(out2.cpu().numpy(), oracle.nrm_batch(xd.cpu().numpy(), off))
    g.close()


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_batch_tuning_and_composition_invariance(nrm, dt):
    """A vector's norm does not depend on the batch it is in, nor on tuning."""
    x, off = inputs.ragged_batch(200, seed=15, dtype=dt, max_log2=17)
    want = oracle.nrm_batch(x, off)
    xd = dev(x)
    ctx = nrm.Context(0)
    try:
        for g, wpb, k in ((2, 4, 2), (3, 8, 7), (3, 16, 5), (2, 8, 12)):
            ctx.set_tuning(g, wpb, k, 4)
            out, _ = nrm.nrm_batch(xd, dev(off), ctx=ctx)
            assert bits_equal(out.cpu().numpy(), want), (g, wpb, k)
        # subsets and a reversed order
        idx = list(range(0, 200, 3))[::-1]
        sub_off = [0]
        parts = []
        for i in idx:
            parts.append(x[off[i]:off[i + 1]])
            sub_off.append(sub_off[-1] + off[i + 1] - off[i])
        xs = np.concatenate(parts)
        out, _ = nrm.nrm_batch(dev(xs), dev(np.array(sub_off, np.int64)), ctx=ctx)
        assert bits_equal(out.cpu().numpy(), want[idx])
    finally:
        ctx.close()


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_config3_pnorm_batch(nrm, dt):
    """1024 vectors of 2^16, e in [-8, 8], p in {1, 1.5, 3, 7.5}: 48 sampled
    vectors bitwise against the oracle; constant vectors c repeated 2^16
    times within tolerance of |c| 2^(16/p) (and exactly 2^16 |c| for p = 1)."""
    B, n = 1024, 1 << 16
    off = np.arange(B + 1, dtype=np.int64) * n
    offd = dev(off)
    xd = nrm.nrm_gen_ragged(offd, seed=16, dtype=TD[dt], emin=-8, emax=8)
    x = xd.cpu().numpy()
    tol = 1e-14 if dt == np.float64 else 5e-6
    for p in (1.0, 1.5, 3.0, 7.5):
        out, st = nrm.nrm_batch(xd, offd, p)
        o = out.cpu().numpy()
        for i in random.Random(int(p * 10)).sample(range(B), 12):
            v = x[off[i]:off[i + 1]]
            assert bits_equal(o[i], oracle.nrm(v, p)), (p, i)
            assert oracle.relerr(o[i], v, p, nthreads=8) <= tol
    for c in (1.0, -1.75, 3.0e-3):
        cv = torch.full((B * n,), c, dtype=TD[dt], device=DEV)
        for p in (1.0, 1.5, 3.0, 7.5):
            out, _ = nrm.nrm_batch(cv, offd, p)
            o = out.cpu().numpy().astype(np.float64)
            cc = abs(float(dt(c)))
            exact = cc * 2.0 ** (16.0 / float(dt(p)))
            if p == 1.0:
                assert (o == cc * n).all()
            assert np.all(np.abs(o - exact) / exact <= tol), (c, p)


def test_tickets_return_to_zero(nrm):
    """Every call leaves all node tickets at zero (each node's second
    arriver resets its ticket), across calls of different tree shapes and
    batches -- the invariant the next call's combine relies on."""
    import ctypes
    L = nrm.load()
    ctx = nrm.Context(0)
    try:
        x = dev(inputs.vector(1 << 21, seed=17, vec=0))
        for n in (1000, 4097, 62381, 1 << 21, 3, 200000, 64):
            nrm.nrmf(x[:n], ctx=ctx)
        xb, off = inputs.ragged_batch(300, seed=18, max_log2=16)
        nrm.nrm_batch(dev(xb), dev(off), ctx=ctx)
        torch.cuda.synchronize()
        t = np.zeros(1 << 16, np.uint32)
        assert L.nrm_test_read_tickets(ctx.h, ctypes.c_void_p(t.ctypes.data), t.size) == 0
        assert not t.any(), np.nonzero(t)[0][:20]
    finally:
        ctx.close()


@pytest.mark.parametrize("mode", range(7))
def test_k1_exact_matches_fp64_k1(nrm, mode):
    """The binary64 tree computes v1_hypot with integer/FP32 arithmetic
    (GB300's FP64 pipe is the bottleneck otherwise); it must equal the FP64
    v1_hypot of Listing 2 bit for bit.  2^30 generated pairs per family:
    moderate exponent gaps, close values, edge significands, raw bit patterns
    (inf, NaN, subnormal, zero), extreme exponents (overflow to inf), gaps
    around the 2^-27 shortcut, equal values."""
    import ctypes
    L = nrm.load()
    f = L.nrm_test_k1d_compare
    f.restype = ctypes.c_int32
    f.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    bad = torch.zeros(1, dtype=torch.int64, device=DEV)
    ex = torch.zeros(4, dtype=torch.float64, device=DEV)
    for rep in range(4):
        assert f(1234567 + 1000 * mode + rep, 1 << 28, mode, ctypes.c_void_p(bad.data_ptr()),
                 ctypes.c_void_p(ex.data_ptr()), None) == 0
    torch.cuda.synchronize()
    assert int(bad.item()) == 0, ex.cpu().numpy()


@pytest.mark.parametrize("mode", [0, 1, 2, 3, 5, 6])
def test_k1_fast_matches_fp64(nrm, mode):
    """The checked-group binary64 v1_hypot (rounded 54-bit quotient, rounded
    integer square root, one FP64 fma and one FP64 multiply) equals the FP64
    v1_hypot of Listing 2 bit for bit on 2^30 generated pairs per family
    inside its range [2^-500, 2^502)."""
    import ctypes
    L = nrm.load()
    f = L.nrm_test_k1d_compare
    f.restype = ctypes.c_int32
    f.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    bad = torch.zeros(1, dtype=torch.int64, device=DEV)
    ex = torch.zeros(4, dtype=torch.float64, device=DEV)
    for rep in range(4):
        assert f(2468013 + 1000 * mode + rep, 1 << 28, 8 + mode, ctypes.c_void_p(bad.data_ptr()),
                 ctypes.c_void_p(ex.data_ptr()), None) == 0
    torch.cuda.synchronize()
    assert int(bad.item()) == 0, ex.cpu().numpy()
    assert f(1, 1, 7, ctypes.c_void_p(bad.data_ptr()), ctypes.c_void_p(ex.data_ptr()), None) == nrm.NRM_EINVAL


@pytest.mark.parametrize("mode", [0, 1, 2, 3, 5, 6])
def test_k1_fast_pair_matches_fp64(nrm, mode):
    """The paired checked-group binary64 v1_hypot (two operand pairs at
    once, their FP32 estimates in paired FFMA2 / FMUL2 / FADD2 instructions)
    equals the FP64 v1_hypot of Listing 2 on both pairs, bit for bit, on
    2^29 generated pairs of pairs per family inside its range."""
    import ctypes
    L = nrm.load()
    f = L.nrm_test_k1d_compare
    f.restype = ctypes.c_int32
    f.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    bad = torch.zeros(1, dtype=torch.int64, device=DEV)
    ex = torch.zeros(4, dtype=torch.float64, device=DEV)
    for rep in range(2):
        assert f(97531 + 1000 * mode + rep, 1 << 28, 16 + mode, ctypes.c_void_p(bad.data_ptr()),
                 ctypes.c_void_p(ex.data_ptr()), None) == 0
    torch.cuda.synchronize()
    assert int(bad.item()) == 0, ex.cpu().numpy()
    assert f(1, 1, 23, ctypes.c_void_p(bad.data_ptr()), ctypes.c_void_p(ex.data_ptr()), None) == nrm.NRM_EINVAL


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_autotune_keeps_bits(nrm, dt):
    """The autotuner picks a valid tuning; results before and after are
    bitwise identical (single vector and ragged batch)."""
    ctx = nrm.Context(0)
    try:
        code = nrm.NRM_F64 if dt == np.float64 else nrm.NRM_F32
        x = inputs.vector(3 * (1 << 20) + 17, seed=19, vec=0, dtype=dt)
        xd = dev(x)
        before = nrm.nrmf(xd, ctx=ctx).item()
        best = ctx.autotune(code, [x.size])
        assert 2 <= best["group_log2"] <= 3 and best["warps_per_block"] in (4, 8, 16)
        after = nrm.nrmf(xd, ctx=ctx).item()
        assert bits_equal(np.asarray(before, dt), np.asarray(after, dt))
        assert bits_equal(np.asarray(after, dt), oracle.nrm(x))
        xb, off = inputs.ragged_batch(256, seed=20, dtype=dt, max_log2=14)
        ctx.autotune(code, np.diff(off))
        out, _ = nrm.nrm_batch(dev(xb), dev(off), ctx=ctx)
        assert bits_equal(out.cpu().numpy(), oracle.nrm_batch(xb, off))
        # nrm_tune: the same autotuner without the read-back
        import ctypes
        L = nrm.load()
        lens = np.ascontiguousarray(np.diff(off), dtype=np.int64)
        assert L.nrm_tune(ctx.h, code, ctypes.c_void_p(lens.ctypes.data), lens.size) == 0
        assert L.nrm_tune(ctx.h, code, None, 4) == nrm.NRM_EINVAL
        out, _ = nrm.nrm_batch(dev(xb), dev(off), ctx=ctx)
        assert bits_equal(out.cpu().numpy(), oracle.nrm_batch(xb, off))
    finally:
        ctx.close()


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_strided_parity(nrm, dt):
    x = inputs.vector(300000, seed=21, vec=0, dtype=dt)
    xd = dev(x)
    for n, incx in ((300000, 1), (100000, 3), (99999, -3), (1000, -1), (5, 7), (1, -5), (60000, 5), (150000, -2)):
        for p in (2.0, 3.0):
            g = nrm.nrm_strided(xd, n, incx, p).item()
            assert bits_equal(np.asarray(g, dt), oracle.nrm_strided(x, n, incx, p)), (n, incx, p)


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_matrix_parity(nrm, dt):
    x = inputs.vector(1 << 21, seed=22, vec=0, dtype=dt)
    xd = dev(x)
    for M, N, lda in ((1000, 200, 1000), (1000, 200, 1031), (64, 3000, 100), (1, 5000, 7), (70000, 3, 70001),
                      (0, 5, 5), (5, 1, 9)):
        for p in (2.0, 1.0, 3.0):
            g = nrm.nrm_matrix(xd, M, N, lda, p).item()
            assert bits_equal(np.asarray(g, dt), oracle.nrm_matrix(x, M, N, lda, p)), (M, N, lda, p)


def test_complex_parity(nrm):
    z = torch.complex(dev(inputs.vector(123457, seed=23, vec=0)), dev(inputs.vector(123457, seed=23, vec=1)))
    g = nrm.nrmf_complex(z).item()
    inter = torch.view_as_real(z).reshape(-1).cpu().numpy()
    assert bits_equal(np.float64(g), oracle.nrm(inter))


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_za_parity(nrm, dt):
    """Z with A for the final reduction (the paper's recommended xNRMF):
    bitwise against the oracle over many sizes and offsets; two-element
    vectors give cr_hypot(x0, x1) itself (random gaps around the shortcut,
    exact triples, subnormals)."""
    x = inputs.vector(600000, seed=24, vec=0, dtype=dt)
    xd = dev(x)
    for n, s in ((1, 0), (2, 0), (63, 1), (64, 0), (129, 3), (1000, 0), (65537, 5), (300000, 7), (599990, 1)):
        g = nrm.nrmf_za(xd[s:s + n]).item()
        assert bits_equal(np.asarray(g, dt), oracle.nrm_za(x[s:s + n])), (n, s)
    r = random.Random(25)
    thr = 28 if dt == np.float64 else 14
    small = -1070 if dt == np.float64 else -148
    pairs = []
    for _ in range(1500):
        e = r.randint(small, 100)
        g = r.choice([0, 1, thr - 1, thr, thr + 1, r.randint(0, 2 * thr)])
        pairs.append(((1 + r.random()) * 2.0 ** e, -(1 + r.random()) * 2.0 ** (e - g)))
    for _ in range(500):
        m, k = r.randint(1, 2 ** 11), r.randint(1, 2 ** 11)
        pairs.append((float(m * m - k * k), float(2 * m * k)))
    tiny = float(np.finfo(dt).smallest_subnormal)
    pairs += [(tiny, tiny), (3 * tiny, 4 * tiny), (float(np.finfo(dt).tiny), tiny), (float(np.finfo(dt).max), 1.0)]
    arr = np.array(pairs, dtype=dt).reshape(-1)
    ad = dev(arr)
    out = torch.empty(len(pairs), dtype=TD[dt], device=DEV)
    for i in range(len(pairs)):
        nrm.nrmf_za(ad[2 * i:2 * i + 2], out=out[i])
    o = out.cpu().numpy()
    for i, (a, b) in enumerate(pairs):
        want = oracle.cr_hypot(dt(a), dt(b), dt)
        assert bits_equal(o[i], np.asarray(want, dt)), (a, b, o[i], want)


# ---------------------------------------------------------------------------
# the pow and v1_lp combine themselves (Listing 5, Section 4), elementwise
# ---------------------------------------------------------------------------

def _pow_operands(dt, n, seed):
    """n (x, y) pairs in families: the two domains v1_lp uses (Q in [0, 1]
    with y = p/2, Z in [1, 2] with y = 1/p), x near 1 with large y, tiny and
    subnormal x, results near overflow and underflow, exact powers of two,
    and raw bit patterns (zero, inf, NaN, subnormal)."""
    with np.errstate(all="ignore"):
        return _pow_operand_families(dt, n, seed)


def _pow_operand_families(dt, n, seed):
    rng = np.random.default_rng(seed)
    k = n // 8
    it = np.uint64 if dt == np.float64 else np.uint32
    xs, ys = [], []
    xs.append(rng.random(k) ** rng.choice([1, 3, 20], k)); ys.append(rng.uniform(0.05, 10, k))
    xs.append(1 + rng.random(k)); ys.append(1 / rng.uniform(0.05, 40, k))
    xs.append(1 + rng.uniform(-1, 1, k) * 2.0 ** rng.integers(-52 if dt == np.float64 else -23, 0, k))
    ys.append(rng.uniform(0.5, 2, k) * 2.0 ** rng.integers(-20, 40, k))
    lo = -1074 if dt == np.float64 else -149
    xs.append(rng.uniform(0.5, 2, k) * 2.0 ** rng.integers(lo, lo + 80, k)); ys.append(rng.uniform(0.01, 1.1, k))
    x4 = rng.uniform(0.1, 4, k)
    xs.append(x4); ys.append(np.abs(rng.uniform(-1, 1, k) * (1100 if dt == np.float64 else 150)
                                    / np.maximum(np.abs(np.log2(x4)), 1e-3)) + 1e-3)
    xs.append(2.0 ** rng.integers(lo, 0, k).astype(np.float64)); ys.append(rng.choice([0.5, 0.25, 1.5, 3.0, 1.0, 7.5], k))
    nb = 64 if dt == np.float64 else 32
    raw = rng.integers(0, 2 ** (nb - 1), (2, k), dtype=np.uint64).astype(it)
    xs.append(raw[0].view(dt).astype(np.float64)); ys.append(raw[1].view(dt).astype(np.float64))
    rest = n - 7 * k
    xs.append(rng.random(rest)); ys.append(rng.choice([0.25, 0.75, 1.5, 3.75], rest))
    return np.concatenate(xs).astype(dt), np.concatenate(ys).astype(dt)


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_pow_parity(nrm, dt):
    """The device pow equals the oracle's bit for bit on 2^20 operand pairs
    of every family (binary64: the fixed-point integer pow)."""
    import ctypes
    L = nrm.load()
    f = L.nrm_test_pow
    f.restype = ctypes.c_int32
    f.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
    x, y = _pow_operands(dt, 1 << 20, seed=77)
    xd, yd = dev(x), dev(y)
    out = torch.empty_like(xd)
    code = nrm.NRM_F64 if dt == np.float64 else nrm.NRM_F32
    assert f(code, ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(yd.data_ptr()),
             ctypes.c_void_p(out.data_ptr()), x.size, None) == 0
    got = out.cpu().numpy()
    want = oracle.pow_arr(x, y)
    bad = ~((got.view(np.uint64 if dt == np.float64 else np.uint32) == want.view(np.uint64 if dt == np.float64 else np.uint32))
            | (np.isnan(got) & np.isnan(want)))
    assert not bad.any(), (x[bad][:4], y[bad][:4], got[bad][:4], want[bad][:4])
    assert f(code, None, None, None, -1, None) != 0


def _powr_operands(n, seed):
    """Operands of the restricted binary64 pow of v1_lp (1 < p <= 2^17) in
    its two domains: Q in [0, 1) with y = p/2 in (1/2, 2^16] and Z in [1, 2]
    with y = 1/p in [2^-17, 1): plain draws, x next to 1 on both sides, x at
    2 and at powers of two, x around 2^-60 and results around the flush
    limit 2^-28, y at the ends of its ranges."""
    rng = np.random.default_rng(seed)
    k = n // 8
    p = np.exp(rng.uniform(np.log(1.0 + 1e-12), np.log(2.0 ** 17), 8 * k))
    half = rng.random(8 * k) < 0.5
    p[half] = rng.choice([1.0 + 2.0 ** -40, 1.5, np.sqrt(2.0), np.e, np.pi, 3.0, 7.5, 64.0], half.sum())
    p[p == 2.0] = 3.0
    h, ip = p * 0.5, 1.0 / p
    xs, ys = [], []
    xs.append(rng.random(k) ** rng.choice([1, 2, 5, 20], k)); ys.append(h[:k])
    xs.append(1.0 + rng.random(k)); ys.append(ip[k:2 * k])
    xs.append(1.0 - rng.random(k) * 2.0 ** -rng.integers(1, 53, k)); ys.append(h[2 * k:3 * k])
    xs.append(1.0 + rng.random(k) * 2.0 ** -rng.integers(1, 53, k)); ys.append(ip[3 * k:4 * k])
    xs.append(2.0 ** rng.uniform(-61.5, -58.5, k)); ys.append(rng.uniform(0.5, 0.51, k))
    # results around 2^-28: y log2 x in [-29, -27]
    yy = h[5 * k:6 * k]
    xs.append(2.0 ** (-rng.uniform(27.0, 29.0, k) / yy)); ys.append(yy)
    xs.append(np.concatenate([np.full(k // 2, 2.0), 2.0 ** -rng.integers(1, 60, k - k // 2).astype(np.float64)]))
    ys.append(np.concatenate([ip[6 * k:6 * k + k // 2], rng.choice([0.5, 0.75, 1.5, 3.0, 3.75, 4.0], k - k // 2)]))
    rest = n - 7 * k
    xs.append(rng.random(rest)); ys.append(np.where(rng.random(rest) < 0.5, 2.0 ** 16, 0.5 + 2.0 ** -52))
    x, y = np.concatenate(xs), np.concatenate(ys)
    x[:4] = [0.0, 1.0, 2.0, 5e-324]
    y[:4] = [1.5, 1.5, 2.0 ** -17, 0.75]
    return x, y


def test_powr_parity(nrm):
    """The device pow of v1_lp for 1 < p <= 2^17 equals the oracle's
    or_powr_d bit for bit on 2^20 operand pairs of its two domains."""
    import ctypes
    L = nrm.load()
    f = L.nrm_test_powr
    f.restype = ctypes.c_int32
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
    x, y = _powr_operands(1 << 20, seed=79)
    xd, yd = dev(x), dev(y)
    out = torch.empty_like(xd)
    assert f(ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(yd.data_ptr()), ctypes.c_void_p(out.data_ptr()),
             x.size, None) == 0
    got = out.cpu().numpy()
    want = oracle.powr_arr(x, y)
    bad = got.view(np.uint64) != want.view(np.uint64)
    assert not bad.any(), (x[bad][:4], y[bad][:4], got[bad][:4], want[bad][:4])
    assert (want == 0).sum() > 10000 and (want != 0).sum() > 600000
    assert f(None, None, None, -1, None) != 0


@pytest.mark.parametrize("dt", [np.float64, np.float32])
@pytest.mark.parametrize("p", [0.5, 1.5, 3.0, 7.5, math.pi, 2.0 ** 40,
                               # the ends of the restricted pow's range (1 < p <= 2^17) and just past it
                               1.0 + 2.0 ** -40, 2.0 ** 17, 2.0 ** 17 * (1.0 + 2.0 ** -50)])
def test_lp_combine_parity(nrm, dt, p):
    """v1_lp on the device (binary64: integer quotient and pow, FP64 form for
    inf, NaN and subnormal operands) equals the oracle's v1_lp bit for bit on
    2^19 operand pairs: moderate and extreme exponent gaps, equal
    magnitudes, zeros, subnormals, the largest exponents, and raw bits."""
    import ctypes
    L = nrm.load()
    f = L.nrm_test_lp
    f.restype = ctypes.c_int32
    f.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                  ctypes.c_void_p]
    rng = np.random.default_rng(int(p * 1000) % 2 ** 31)
    n = 1 << 19
    k = n // 8
    emax = 1023 if dt == np.float64 else 127
    emin = -1074 if dt == np.float64 else -149
    it = np.uint64 if dt == np.float64 else np.uint32
    nb = 64 if dt == np.float64 else 32
    a = rng.uniform(1, 2, n) * rng.choice([-1.0, 1.0], n)
    b = rng.uniform(1, 2, n) * rng.choice([-1.0, 1.0], n)
    ea = rng.integers(-30, 30, n)
    gap = np.concatenate([rng.integers(-3, 4, k), rng.integers(-60, 61, k), rng.integers(-1100, 1100, k),
                          np.zeros(k, np.int64), rng.integers(-40, 41, n - 4 * k)])
    with np.errstate(over="ignore", under="ignore", invalid="ignore"):
        x = (a * 2.0 ** ea).astype(dt)
        y = (b * 2.0 ** np.clip(ea + gap, emin, emax)).astype(dt)
        y[3 * k:4 * k] = -x[3 * k:4 * k]                      # equal magnitudes
        x[4 * k:4 * k + 64] = 0                                # zeros
        y[4 * k + 32:4 * k + 96] = 0
        x[4 * k + 96:4 * k + 1000] = (a[4 * k + 96:4 * k + 1000] * 2.0 ** (emin + 10)).astype(dt)  # subnormals
        x[4 * k + 1000:4 * k + 2000] = (a[4 * k + 1000:4 * k + 2000] * 2.0 ** (emax - 1)).astype(dt)
        raw = rng.integers(0, 2 ** nb, (2, 4000), dtype=np.uint64).astype(it)
        x[-4000:] = raw[0].view(dt)
        y[-4000:] = raw[1].view(dt)
    xd, yd = dev(x), dev(y)
    out = torch.empty_like(xd)
    code = nrm.NRM_F64 if dt == np.float64 else nrm.NRM_F32
    assert f(code, float(p), ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(yd.data_ptr()),
             ctypes.c_void_p(out.data_ptr()), n, None) == 0
    got = out.cpu().numpy()
    want = oracle.lp_arr(p, x, y)
    ui = np.uint64 if dt == np.float64 else np.uint32
    bad = ~((got.view(ui) == want.view(ui)) | (np.isnan(got) & np.isnan(want)))
    assert not bad.any(), (x[bad][:4], y[bad][:4], got[bad][:4], want[bad][:4])


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_k1f_fast_steps_exhaustive(nrm, mode):
    """The branch-free binary32 v1_hypot the S trees use on checked groups
    equals Listing 2's correctly rounded steps: its square root on every S in
    [1, 2] (mode 0), its division on every pair of significands (mode 2, all
    2^46 pairs), and the FP32 reciprocal estimate it starts from scales
    exactly with the exponent over the checked range (mode 1), so the pair
    test covers every exponent there; mode 3: the square root on every S in
    [1, 8), the range of K2's binary32 form."""
    import ctypes
    L = nrm.load()
    f = L.nrm_test_k1f_exhaustive
    f.restype = ctypes.c_int32
    f.argtypes = [ctypes.c_int32, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    bad = torch.zeros(1, dtype=torch.int64, device=DEV)
    ex = torch.zeros(2, dtype=torch.float32, device=DEV)
    total = {0: (1 << 23) + 1, 1: 213 << 23, 2: 1 << 46, 3: 3 << 23}[mode]
    chunk = 1 << 40
    for s in range(0, total, chunk):
        assert f(mode, s, min(chunk, total - s), ctypes.c_void_p(bad.data_ptr()), ctypes.c_void_p(ex.data_ptr()),
                 None) == 0
        torch.cuda.synchronize()
    assert int(bad.item()) == 0, ex.cpu().numpy()


@pytest.mark.parametrize("n", [5 * (1 << 18) + 77, 1 << 21, 3 * (1 << 19) - 5])
@pytest.mark.parametrize("family", ["low_edge", "high_edge", "nan_pairs", "inf", "zeros", "subnormal", "mixed"])
@pytest.mark.parametrize("dt", [np.float32, np.float64])
def test_checked_group_boundaries(nrm, dt, family, n):
    """The trees combine checked groups (full, and partial ones whose slots
    are not all occupied) with a branch-free v1_hypot and send the others to
    the general form; results must equal the oracle's whatever values sit
    in a group: values straddling the ends of the checked range (binary32
    2^-88 and 2^118, binary64 2^-500 and 2^494), NaN pairs that meet in the
    first combine (same lane, adjacent rows), inf, zeros and subnormals.
    Sizes: rows filling 5/8 of the slots (partial groups, ragged tail), a
    power-of-two row count (every group and item full, the cp.async ring),
    and 3/4 of the slots (groups of three rows, ragged tail)."""
    x = inputs.vector(n, seed=40 + len(family), vec=1, dtype=dt)
    rng = np.random.default_rng(abs(hash((family, str(dt)))) % 2 ** 31)
    P = 128 if dt == np.float32 else 64
    pos = rng.choice(n, 64, replace=False)
    lo, hi = (-88, 118) if dt == np.float32 else (-500, 494)
    with np.errstate(all="ignore"):
        if family == "low_edge":
            x[pos] = (rng.uniform(1, 2, 64) * 2.0 ** rng.integers(lo - 4, lo + 4, 64)).astype(dt)
        elif family == "high_edge":
            x[pos] = (rng.uniform(1, 2, 64) * 2.0 ** rng.integers(hi - 4, hi + 4, 64)).astype(dt)
        elif family == "nan_pairs":
            q = pos[pos + P < n]
            x[q] = np.nan
            x[q + P] = np.nan
        elif family == "inf":
            x[pos[:4]] = np.inf
        elif family == "zeros":
            x[pos] = 0
            x[:4096] = 0  # whole groups of zeros
        elif family == "subnormal":
            tiny = np.finfo(dt).smallest_subnormal
            x[pos] = (rng.integers(1, 1000, 64) * tiny).astype(dt)
        else:
            x[pos[:16]] = (2.0 ** rng.integers(lo - 7, lo + 8, 16)).astype(dt)
            x[pos[16:32]] = (2.0 ** rng.integers(hi - 8, hi + 6, 16)).astype(dt)
            q = pos[32:40]
            q = q[q + P < n]
            x[q] = np.nan
            x[q + P] = np.nan
            x[pos[40:48]] = 0
    got = nrm.nrmf(dev(x)).cpu().numpy()
    want = oracle.nrm(x)
    assert bits_equal(np.asarray(got, dt), np.asarray(want, dt)), (family, got, want)


def _combine_operands(dt, n, seed):
    """Operand pairs for the combine functors: moderate and huge exponent
    gaps, equal and adjacent magnitudes, sums that carry into the next
    binade or round to even, subnormals (both, one), the largest finite
    values (sums overflowing to inf), zeros, and raw bit patterns."""
    rng = np.random.default_rng(seed)
    it, nb = (np.uint64, 64) if dt == np.float64 else (np.uint32, 32)
    emax = 1023 if dt == np.float64 else 127
    sub = np.finfo(dt).smallest_subnormal
    k = n // 8
    with np.errstate(all="ignore"):
        a = rng.uniform(1, 2, n) * rng.choice([-1.0, 1.0], n)
        b = rng.uniform(1, 2, n) * rng.choice([-1.0, 1.0], n)
        ea = rng.integers(-60, 60, n)
        gap = np.concatenate([rng.integers(-3, 4, k), rng.integers(-70, 71, k), rng.integers(50, 60, k),
                              np.zeros(k, np.int64), rng.integers(-30, 31, n - 4 * k)])
        x = (a * 2.0 ** ea).astype(dt)
        y = (b * 2.0 ** (ea - gap)).astype(dt)
        y[3 * k:3 * k + k // 2] = -x[3 * k:3 * k + k // 2]                         # equal magnitudes
        y[3 * k + k // 2:4 * k] = np.nextafter(x[3 * k + k // 2:4 * k], dt(np.inf))  # adjacent
        s0 = 4 * k
        x[s0:s0 + 2000] = (rng.integers(1, 2 ** 20, 2000) * sub).astype(dt)          # subnormal pairs
        y[s0:s0 + 2000] = (rng.integers(1, 2 ** 20, 2000) * sub).astype(dt)
        x[s0 + 2000:s0 + 4000] = (rng.integers(1, 2 ** 20, 2000) * sub).astype(dt)   # subnormal + normal
        big = np.finfo(dt).max
        x[s0 + 4000:s0 + 6000] = (big * rng.uniform(0.5, 1, 2000)).astype(dt)         # overflow to inf
        y[s0 + 4000:s0 + 6000] = (big * rng.uniform(0.5, 1, 2000)).astype(dt)
        x[s0 + 6000:s0 + 6100] = 0
        y[s0 + 6050:s0 + 6150] = 0
        raw = rng.integers(0, 2 ** nb, (2, 8000), dtype=np.uint64).astype(it)
        x[-8000:] = raw[0].view(dt)
        y[-8000:] = raw[1].view(dt)
    return x, y


@pytest.mark.parametrize("dt", [np.float64, np.float32])
@pytest.mark.parametrize("p", [1.0, 2.0, math.inf, 2.0 ** 60, 3.0])
def test_combine_parity(nrm, dt, p):
    """Every combine the trees apply (|x|+|y|, v1_hypot, max(|x|,|y|), v1_lp;
    for binary64 the forms without the FP64 pipe) equals the oracle's combine
    for the same p bit for bit on 2^19 operand pairs."""
    import ctypes
    L = nrm.load()
    f = L.nrm_test_combine
    f.restype = ctypes.c_int32
    f.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                  ctypes.c_void_p]
    x, y = _combine_operands(dt, 1 << 19, seed=int(min(p, 1e6) * 7) + 5)
    xd, yd = dev(x), dev(y)
    out = torch.empty_like(xd)
    code = nrm.NRM_F64 if dt == np.float64 else nrm.NRM_F32
    assert f(code, float(p), ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(yd.data_ptr()),
             ctypes.c_void_p(out.data_ptr()), x.size, None) == 0
    got = out.cpu().numpy()
    want = oracle.comb_arr(p, x, y)
    ui = np.uint64 if dt == np.float64 else np.uint32
    bad = ~((got.view(ui) == want.view(ui)) | (np.isnan(got) & np.isnan(want)))
    assert not bad.any(), (x[bad][:4], y[bad][:4], got[bad][:4], want[bad][:4])


# ---------------------------------------------------------------------------
# the exponent-scaled hypotenuse K2 (nrmf_es_*)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_es_parity(nrm, dt):
    """xNRMF with K2 equals the oracle's or_nrm_es bit for bit over sizes
    with ragged tails, full items and several work items, on moderately and
    widely varying data, with zeros, NaN pairs, inf and subnormals mixed in,
    and on vectors straddling the checked range."""
    rng = np.random.default_rng(50)
    for n in (1, 2, 3, 127, 129, 4096, 100003, 3 * (1 << 20) + 17):
        for emin, emax in ((-20, 20), (-8, 8), (-300, 300) if dt == np.float64 else (-60, 60)):
            x = inputs.vector(n, seed=51, vec=n % 11, dtype=dt, emin=emin, emax=emax)
            got = nrm.nrmf_es(dev(x)).cpu().numpy()
            assert bits_equal(np.asarray(got, dt), np.asarray(oracle.nrm_es(x), dt)), (n, emin, emax)
    n = 5 * (1 << 18) + 77
    P = 128 if dt == np.float32 else 64
    lo, hi = (-88, 118) if dt == np.float32 else (-500, 494)
    for fam in range(5):
        x = inputs.vector(n, seed=52 + fam, vec=1, dtype=dt)
        pos = rng.choice(n - P, 64, replace=False)
        with np.errstate(all="ignore"):
            if fam == 0:
                x[pos] = (2.0 ** rng.integers(lo - 4, lo + 4, 64)).astype(dt)
            elif fam == 1:
                x[pos] = (2.0 ** rng.integers(hi - 4, hi + 4, 64)).astype(dt)
            elif fam == 2:
                x[pos] = np.nan
                x[pos + P] = np.nan
            elif fam == 3:
                x[pos[:3]] = np.inf
                x[pos[3:20]] = 0
            else:
                x[pos] = (rng.integers(1, 1000, 64) * np.finfo(dt).smallest_subnormal).astype(dt)
        got = nrm.nrmf_es(dev(x)).cpu().numpy()
        assert bits_equal(np.asarray(got, dt), np.asarray(oracle.nrm_es(x), dt)), fam


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_k2_elementwise_parity(nrm, dt):
    """The general K2 the trees use outside checked groups equals the
    oracle's K2 bit for bit on 2^19 operand pairs (the combine families:
    carries, ties, subnormals, overflow to inf, zeros, raw bit patterns)."""
    import ctypes
    L = nrm.load()
    f = L.nrm_test_k2
    f.restype = ctypes.c_int32
    f.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
    x, y = _combine_operands(dt, 1 << 19, seed=61)
    xd, yd = dev(x), dev(y)
    out = torch.empty_like(xd)
    code = nrm.NRM_F64 if dt == np.float64 else nrm.NRM_F32
    assert f(code, ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(yd.data_ptr()), ctypes.c_void_p(out.data_ptr()),
             x.size, None) == 0
    got = out.cpu().numpy()
    want = oracle.k2_arr(x, y)
    ui = np.uint64 if dt == np.float64 else np.uint32
    bad = ~((got.view(ui) == want.view(ui)) | (np.isnan(got) & np.isnan(want)))
    assert not bad.any(), (x[bad][:4], y[bad][:4], got[bad][:4], want[bad][:4])


@pytest.mark.parametrize("mode", [0, 1, 2, 5, 6])
def test_k2_fast_matches_general(nrm, mode):
    """The checked-group binary64 K2 (integer square root for S in [1, 8),
    exact scalings) equals the general form with the FP64 square root on
    2^30 generated pairs per family inside its range."""
    import ctypes
    L = nrm.load()
    f = L.nrm_test_k2d_compare
    f.restype = ctypes.c_int32
    f.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    bad = torch.zeros(1, dtype=torch.int64, device=DEV)
    ex = torch.zeros(4, dtype=torch.float64, device=DEV)
    for rep in range(4):
        assert f(7654321 + 1000 * mode + rep, 1 << 28, mode, ctypes.c_void_p(bad.data_ptr()),
                 ctypes.c_void_p(ex.data_ptr()), None) == 0
    torch.cuda.synchronize()
    assert int(bad.item()) == 0, ex.cpu().numpy()
