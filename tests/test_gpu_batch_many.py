"""GPU parity of ragged batches with many vectors (Section 3.1's per-column
norms as one launch).

The device planner gives each of its 1024 threads a contiguous chunk of
vectors and keeps the plans' item counts in shared memory for the first
8192 plans only; a batch of 20000 vectors runs chunks of 20 vectors and
reads the later item counts back from the plans.  Every norm must equal the
oracle's bit for bit, with one p per call and with a p per vector, and
empty vectors give 0 with status NRM_OK.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2509_06220_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
DEV = "cuda:0"
B = 20000


@pytest.fixture(scope="module")
def nrm():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2509_06220_gb300 as m
    return m


def _batch(dt):
    L = inputs.ragged_lengths(B, seed=90, max_log2=9)
    L[::97] = 0                  # empty vectors
    L[5] = (1 << 18) + 5         # a few long ones among the short
    L[B // 2] = 3 << 17
    L[B - 1] = 100003
    x, off = inputs.ragged_batch(B, seed=90, dtype=dt, lengths=L)
    return x, off


def _bits(a, dt):
    return np.ascontiguousarray(a, dtype=dt).view(np.uint64 if dt == np.float64 else np.uint32)


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_many_vectors_one_p(nrm, dt):
    x, off = _batch(dt)
    want = oracle.nrm_batch(x, off)
    ctx = nrm.Context(0)
    try:
        xd, offd = torch.from_numpy(x).to(DEV), torch.from_numpy(off).to(DEV)
        # the default tuning, then small work items (many more items than warps)
        for tuning in (None, (2, 4, 4, 2)):
            if tuning:
                ctx.set_tuning(*tuning)
            out, st = nrm.nrm_batch(xd, offd, ctx=ctx)
            torch.cuda.synchronize()
            assert (st.cpu().numpy() == 0).all()
            got = out.cpu().numpy()
            assert np.array_equal(_bits(got, dt), _bits(want, dt)), (tuning, np.nonzero(_bits(got, dt) != _bits(want, dt))[0][:10])
            assert (got[::97] == 0).all()
    finally:
        ctx.close()


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_many_vectors_p_per_vector(nrm, dt):
    x, off = _batch(dt)
    choices = [2.0, 1.0, 1.5, 3.0, math.inf, 7.5]
    p = np.array([choices[i % len(choices)] for i in range(B)], np.float64)
    want = np.empty(B, dt)
    for i in range(B):
        want[i] = oracle.nrm(x[off[i]:off[i + 1]], dt(p[i])) if off[i + 1] > off[i] else dt(0)
    ctx = nrm.Context(0)
    try:
        out, st = nrm.nrm_batch(torch.from_numpy(x).to(DEV), torch.from_numpy(off).to(DEV),
                                torch.from_numpy(p).to(DEV), ctx=ctx)
        torch.cuda.synchronize()
        assert (st.cpu().numpy() == 0).all()
        got = out.cpu().numpy()
        assert np.array_equal(_bits(got, dt), _bits(want, dt)), np.nonzero(_bits(got, dt) != _bits(want, dt))[0][:10]
    finally:
        ctx.close()
