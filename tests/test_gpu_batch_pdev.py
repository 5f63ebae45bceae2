"""GPU parity of the ragged batch with one p per vector (nrm_batch's p_dev).

xNRMP (Section 4) takes p per call; a batch with a p per vector runs one
persistent launch in which each work item is combined with its vector's
combine.  Every result must equal the oracle's norm of that vector with that
p, bit for bit, whatever the mix, the tuning and the graph replay; a p that
is <= 0 or NaN gives NaN and NRM_EINVAL for that vector only.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2509_06220_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
DEV = "cuda:0"

# p values of every kind: v1_hypot (2), sumabs (1), maxabs (inf and at or
# above the cut-off p'), v1_lp (the rest, Table 4's values among them)
P_CHOICES = [2.0, 1.0, 1.5, 3.0, 7.5, 0.5, 2.0 / 3.0, math.sqrt(2), math.e, math.pi, math.inf, 2.0 ** 60,
             2.0 ** 53, 2.0 ** 24, 2.0 ** 23 + 1.0, 1.0000001]


@pytest.fixture(scope="module")
def nrm():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2509_06220_gb300 as m
    return m


def _case(B, seed, dt, max_log2=16):
    x, off = inputs.ragged_batch(B, seed=seed, max_log2=max_log2, dtype=dt)
    rng = np.random.default_rng(seed)
    p = np.array([P_CHOICES[i] for i in rng.integers(0, len(P_CHOICES), B)], np.float64)
    return x, off, p


def _want(x, off, p, dt):
    out = np.empty(off.size - 1, dt)
    for i in range(off.size - 1):
        out[i] = oracle.nrm(x[off[i]:off[i + 1]], dt(p[i]))
    return out


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_batch_per_vector_p_matches_oracle(nrm, dt):
    x, off, p = _case(700, 51 if dt == np.float64 else 52, dt)
    bad = [3, 100, 555]
    p[bad] = [-1.0, 0.0, math.nan]
    if dt == np.float32:
        p[7] = 1e-50  # rounds to +0 in binary32: NRM_EINVAL
        bad.append(7)
    ok = np.setdiff1d(np.arange(p.size), bad)
    want = _want(x, off, np.where(np.isin(np.arange(p.size), bad), 2.0, p), dt)
    xd, offd, pd = torch.from_numpy(x).to(DEV), torch.from_numpy(off).to(DEV), torch.from_numpy(p).to(DEV)
    ctx = nrm.Context(0)
    try:
        for tuning in ({}, {"group_log2": 3, "warps_per_block": 4, "item_log2": 5, "blocks_per_sm": 2},
                       {"group_log2": 2, "warps_per_block": 16, "item_log2": 11, "blocks_per_sm": 16}):
            if tuning:
                ctx.set_tuning(**tuning)
            out, st = nrm.nrm_batch(xd, offd, pd, ctx=ctx)
            o, s = out.cpu().numpy(), st.cpu().numpy()
            assert (s[bad] == nrm.NRM_EINVAL).all() and np.isnan(o[bad]).all(), tuning
            assert (s[ok] == 0).all(), tuning
            assert o[ok].tobytes() == want[ok].tobytes(), (tuning, np.nonzero(o[ok] != want[ok]))
    finally:
        ctx.close()


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_batch_per_vector_p_equals_one_p_batches(nrm, dt):
    """The mixed launch gives, for every vector, the bits of the one-p batch
    of its p (GPU against GPU, on larger vectors than the oracle case)."""
    x, off, p = _case(300, 61, dt, max_log2=19)
    xd, offd = torch.from_numpy(x).to(DEV), torch.from_numpy(off).to(DEV)
    mixed, st = nrm.nrm_batch(xd, offd, torch.from_numpy(p).to(DEV))
    mixed = mixed.cpu().numpy()
    assert (st.cpu().numpy() == 0).all()
    for pv in np.unique(p):
        one, _ = nrm.nrm_batch(xd, offd, float(pv))
        sel = p == pv
        assert mixed[sel].tobytes() == one.cpu().numpy()[sel].tobytes(), pv


def test_batch_graph_per_vector_p_reads_p_at_replay(nrm):
    """A captured graph reads the current contents of x, offsets and p."""
    dt = np.float64
    x, off, p = _case(200, 71, dt, max_log2=14)
    xd, offd, pd = torch.from_numpy(x).to(DEV), torch.from_numpy(off).to(DEV), torch.from_numpy(p).to(DEV)
    g = nrm.nrm_batch_graph(xd, offd, pd)
    try:
        out, st = g.launch()
        torch.cuda.synchronize()
        assert out.cpu().numpy().tobytes() == _want(x, off, p, dt).tobytes()
        p2 = np.roll(p, 7)
        x2 = inputs.ragged_batch(200, seed=72, dtype=dt, lengths=np.diff(off))[0]
        pd.copy_(torch.from_numpy(p2))
        xd.copy_(torch.from_numpy(x2))
        out, st = g.launch()
        torch.cuda.synchronize()
        assert (st.cpu().numpy() == 0).all()
        assert out.cpu().numpy().tobytes() == _want(x2, off, p2, dt).tobytes()
    finally:
        g.close()


def test_segments_per_vector_p(nrm):
    """nrm_batch_segments with a p per segment: segments anywhere, in any
    order, overlapping, each with its own p."""
    dt = np.float32
    x = inputs.vector(1 << 18, seed=80, vec=0, dtype=dt)
    rng = np.random.default_rng(8)
    starts = rng.integers(0, x.size - 1, 250)
    lens = np.minimum(rng.integers(0, 30000, 250), x.size - starts)
    p = np.array([P_CHOICES[i] for i in rng.integers(0, len(P_CHOICES), 250)], np.float64)
    out, st = nrm.nrm_batch_segments(torch.from_numpy(x).to(DEV), torch.from_numpy(starts).to(DEV),
                                     torch.from_numpy(lens).to(DEV), torch.from_numpy(p).to(DEV))
    o = out.cpu().numpy()
    assert (st.cpu().numpy() == 0).all()
    for i in range(250):
        want = oracle.nrm(x[starts[i]:starts[i] + lens[i]], dt(p[i]))
        assert o[i].tobytes() == want.tobytes(), (i, p[i], lens[i])


def test_graphs_survive_workspace_growth(nrm):
    """A graph keeps the workspace it was captured with: capturing a second
    batch that needs a larger workspace (a p per vector sizes its tickets for
    finer v1_lp items), then a long single vector, grows the context's
    workspace, and both graphs still replay correctly."""
    dt = np.float64
    x, off, p = _case(150, 81, dt, max_log2=13)
    xd, offd, pd = torch.from_numpy(x).to(DEV), torch.from_numpy(off).to(DEV), torch.from_numpy(p).to(DEV)
    ctx = nrm.Context(0)
    try:
        g1 = nrm.nrm_batch_graph(xd, offd, 2.0, ctx=ctx)
        g2 = nrm.nrm_batch_graph(xd, offd, pd, ctx=ctx)
        big = nrm.nrm_gen((1 << 24) + 3, 82, 0, torch.float64, device=DEV)
        nrm.nrmf(big, ctx=ctx)
        o1, s1 = g1.launch()
        o2, s2 = g2.launch()
        torch.cuda.synchronize()
        assert o1.cpu().numpy().tobytes() == _want(x, off, np.full(p.size, 2.0), dt).tobytes()
        assert o2.cpu().numpy().tobytes() == _want(x, off, p, dt).tobytes()
        g1.close()
        g2.close()
    finally:
        ctx.close()
