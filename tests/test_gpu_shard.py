"""GPU parity of sharding one vector across 2^dg devices (Section 2,
Eq. hr): nrm_node_lanes on every node's elements, then nrm_combine_nodes,
must equal nrmp_* on the whole vector and the oracle bit for bit -- in one
process over all nodes, and as two gloo processes (each its own node on
cuda:0, 512 bytes all-gathered on the host; no kernel waits on another)."""
import os
import socket

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


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_all_nodes_combined_equal_one_device(nrm, dt):
    td = torch.float64 if dt == np.float64 else torch.float32
    code = nrm.NRM_F64 if dt == np.float64 else nrm.NRM_F32
    P = 64 if dt == np.float64 else 128
    for n, seed in ((1, 1), (P * 3 + 1, 2), (100003, 3), ((1 << 22) + 5, 4)):
        x = nrm.nrm_gen(n, seed, 0, td, device=DEV)
        xh = x.cpu().numpy()
        for p in (2.0, 1.0, 3.0, 0.5, float("inf")):
            want = nrm.nrmp(x, p).item()
            if n < 200000:
                assert np.asarray(want, dt).tobytes() == oracle.nrm(xh, p).tobytes(), (n, p)
            for dg in (0, 1, 3, 6):
                lanes = torch.empty((1 << dg) * P, dtype=td, device=DEV)
                for j in range(1 << dg):
                    first, count = nrm.shard_range(n, dg, j, code)
                    nrm.node_lanes(x[first:first + count], p, out=lanes[j * P:(j + 1) * P])
                got = nrm.combine_nodes(lanes, dg, n, p).item()
                assert np.asarray(got, dt).tobytes() == np.asarray(want, dt).tobytes(), (n, p, dg, got, want)


def test_node_lanes_are_the_oracle_lane_partials(nrm):
    x = inputs.vector(50001, seed=6, vec=0)
    got = nrm.node_lanes(torch.from_numpy(x).to(DEV), 2.0).cpu().numpy()
    assert got.tobytes() == oracle.Z(x, 64, 2.0).tobytes()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, n, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import paper_2509_06220_gb300 as m
        torch.cuda.set_device(0)
        dg = world.bit_length() - 1
        first, count = m.shard_range(n, dg, rank)
        part = m.nrm_gen(count, 12, 0, torch.float64, start=first, device=DEV)  # this rank's elements only
        v = m.nrm_sharded(part, n).item()
        q.put((rank, np.float64(v).tobytes()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_on_one_gpu(nrm):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    n = (1 << 21) + 999
    procs = [ctx.Process(target=_rank, args=(r, 2, port, n, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=600) for _ in range(2)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    x = nrm.nrm_gen(n, 12, 0, torch.float64, device=DEV)
    want = np.float64(nrm.nrmf(x).item()).tobytes()
    assert want == oracle.nrm(x.cpu().numpy()).tobytes()
    assert all(b == want for _, b in out)
