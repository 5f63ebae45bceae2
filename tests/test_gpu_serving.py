"""GPU tests of the segment batch and the continuous-batching server.

Each result of a request served in a mix must equal the same request
computed alone, bit for bit (the tree depends on the vector only); the
memory budget rejects what can never fit and queues the rest.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2509_06220_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
DEV = "cuda:0"


@pytest.fixture(scope="module")
def nrm():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2509_06220_gb300 as m
    return m


def alone(nrm, req_id, n, dtype, p, seed, emin=-20, emax=20):
    td = torch.float64 if dtype == nrm.NRM_F64 else torch.float32
    x = nrm.nrm_gen(n, seed, req_id, td, emin, emax, device=DEV)
    return nrm.nrmp(x, p).item()


def same(a, b):
    return (math.isnan(a) and math.isnan(b)) or np.float64(a).tobytes() == np.float64(b).tobytes()


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_batch_segments_any_order(nrm, dt):
    x = inputs.vector(1 << 18, seed=30, vec=0, dtype=dt)
    rng = np.random.default_rng(3)
    starts = rng.integers(0, x.size - 1, 300)
    lens = np.minimum(rng.integers(0, 20000, 300), x.size - starts)
    starts[5], lens[5] = x.size - 3, 10  # runs past the end: NRM_EINVAL, NaN
    out, st = nrm.nrm_batch_segments(torch.from_numpy(x).to(DEV), torch.from_numpy(starts).to(DEV),
                                     torch.from_numpy(lens).to(DEV), 3.0 if dt == np.float32 else 2.0)
    o, s = out.cpu().numpy(), st.cpu().numpy()
    for i in range(300):
        if i == 5:
            assert s[i] == nrm.NRM_EINVAL and math.isnan(o[i])
            continue
        want = oracle.nrm(x[starts[i]:starts[i] + lens[i]], 3.0 if dt == np.float32 else 2.0)
        assert s[i] == 0 and o[i].tobytes() == want.tobytes(), i


def test_server_results_equal_alone(nrm):
    """A bursty mixed trace (FP32/FP64, p in {2, 1.5, 3}, lengths in
    [16, 2^17]) through 2 streams with batching: each norm equals the
    request computed alone and the oracle's norm of the same input; host-
    provided inputs too."""
    tr = nrm.serving_trace(200000, 0.004, seed=5, max_log2=17)
    srv = nrm.Server(budget_bytes=1 << 30, nstreams=2, max_batch=256)
    try:
        norms, lat, rep = srv.replay(tr)
        assert rep["completed"] == len(tr) and rep["rejected"] == 0
        assert rep["steps"] < len(tr)  # requests were batched
        # one segment batch per element type and step (a p per request):
        # at most 2 groups x (plan + tree launch)
        assert rep["launches"] <= 4 * rep["steps"]
        assert 0 < rep["p50_ms"] <= rep["p99_ms"] <= rep["max_ms"]
        for i in range(len(tr)):
            r = tr[i]
            want = alone(nrm, i, r.n, r.dtype, r.p, r.seed)
            assert same(norms[i], want), (i, r.n, r.dtype, r.p, norms[i], want)
            # and the oracle on the same input, regenerated on the host from
            # (seed, request id)
            dt = np.float64 if r.dtype == nrm.NRM_F64 else np.float32
            x = inputs.vector(r.n, seed=r.seed, vec=i, dtype=dt, emin=-20, emax=20)
            assert same(norms[i], float(oracle.nrm(x, r.p))), (i, r.n, r.dtype, r.p)
        # host inputs mixed with generated ones
        xs = [inputs.vector(n, seed=31, vec=j, dtype=dt) for j, (n, dt) in
              enumerate([(1000, np.float64), (77777, np.float32), (5, np.float64), (0, np.float32)])]
        ids = [srv.submit(0, x_host=x, p=p) for x, p in zip(xs, (2.0, 3.0, 1.0, 2.0))]
        ids.append(srv.submit(12345, dtype=nrm.NRM_F32, p=2.0, seed=9))
        srv.drain(60)
        for x, p, rid in zip(xs, (2.0, 3.0, 1.0, 2.0), ids):
            v, st = srv.poll(rid)
            assert st == 0 and same(v, float(oracle.nrm(x, p)) if x.size else 0.0)
    finally:
        srv.close()


def test_server_budget_admission(nrm):
    """A request larger than the input arena is rejected (NRM_EBUDGET); a
    burst that does not fit at once is queued and completes in order."""
    srv = nrm.Server(budget_bytes=96 << 20, nstreams=2, max_batch=64)
    try:
        rep0 = srv.report()
        arena = rep0["arena_bytes"]
        assert 0 < arena < (96 << 20)
        with pytest.raises(nrm.NrmError) as ei:
            srv.submit(arena // 8 + 1, dtype=nrm.NRM_F64)
        assert ei.value.status == nrm.NRM_EBUDGET
        n = arena // 8 // 3  # three of these fill the arena
        ids = [srv.submit(n, dtype=nrm.NRM_F64, seed=40) for _ in range(8)]
        srv.drain(120)
        rep = srv.report()
        assert rep["rejected"] == 1 and rep["completed"] == 8
        assert rep["max_queue"] >= 1 and rep["peak_bytes"] <= arena
        for rid in ids:
            v, st = srv.poll(rid)
            assert st == 0 and same(v, alone(nrm, rid, n, nrm.NRM_F64, 2.0, 40))
    finally:
        srv.close()


def test_server_one_request_per_launch(nrm):
    """max_batch = 1 and one stream: the plain one-request-per-launch form,
    same results."""
    tr = nrm.serving_trace(50000, 0.003, seed=6, max_log2=14)
    a = nrm.Server(budget_bytes=1 << 30, nstreams=1, max_batch=1)
    b = nrm.Server(budget_bytes=1 << 30, nstreams=2, max_batch=512)
    try:
        na, _, ra = a.replay(tr)
        nb, _, rb = b.replay(tr)
        assert ra["steps"] == len(tr)
        assert na.tobytes() == nb.tobytes()
    finally:
        a.close()
        b.close()
