"""CPU checks of sharding one vector across 2^dg devices (Section 2, Eq. hr:
norms of disjoint parts combine by one more combine).

The library's host-side nrm_shard_range gives device j the elements of node
j at depth dg of the vector's row tree.  Those ranges must tile [0, n) in
order, and the protocol -- each rank's node lanes (the oracle's Z over its
elements), an all-gather of the 512-byte rows, the top dg levels of the tree
(a node without rows passes its sibling through) and R over the lanes --
must reproduce the oracle's one-device norm bit for bit.  The multi-rank
form runs as gloo processes on the CPU.
"""
import os
import socket

import numpy as np
import pytest

import oracle
import paper_2509_06220_gb300 as nrm
from paper_2509_06220_gb300 import build as nb
from paper_2509_06220_gb300 import inputs


@pytest.fixture(scope="module", autouse=True)
def _lib():
    nb.build()
    nrm.load()


def _P(dt):
    return 64 if dt == np.float64 else 128


def _code(dt):
    return nrm.NRM_F64 if dt == np.float64 else nrm.NRM_F32


def combine_rows(rows, counts, p, dt):
    """The top levels of the tree over the node rows (oracle combines), then
    R over the lanes of the root."""
    rows = [np.array(r, dt) for r in rows]
    have = [c > 0 for c in counts]
    while len(rows) > 1:
        nxt, nh = [], []
        for i in range(0, len(rows), 2):
            a, b = have[i], have[i + 1]
            if a and b:
                nxt.append(oracle.comb_arr(p, rows[i], rows[i + 1]))
            else:
                nxt.append(rows[i] if a else rows[i + 1])
            nh.append(a or b)
        rows, have = nxt, nh
    return oracle.R(rows[0], p)


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_shard_ranges_tile_the_vector_in_order(dt):
    P = _P(dt)
    rng = np.random.default_rng(5)
    for n in [0, 1, P - 1, P, P + 1, 3 * P, 1000, 12345, 1 << 20, (1 << 20) + 7] + list(rng.integers(1, 10 ** 7, 20)):
        for dg in range(0, 7):
            pos = 0
            rows = []
            for j in range(1 << dg):
                first, count = nrm.shard_range(int(n), dg, j, _code(dt))
                assert count >= 0 and (count == 0 or first == pos), (n, dg, j, first, count, pos)
                pos += count
                rows.append(-(-count // P))
            assert pos == n
            m = -(-int(n) // P)
            # the node sizes are those of the ceil split applied dg times
            want = [m]
            for _ in range(dg):
                want = [s for w in want for s in ((w + 1) // 2, w // 2)]
            assert rows == want, (n, dg)


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_protocol_reproduces_the_oracle(dt):
    """Every node's lanes by the oracle, combined: the oracle's norm."""
    for n, seed in ((1, 1), (200, 2), (5 * _P(dt) + 3, 3), (77777, 4), (1 << 18, 5)):
        x = inputs.vector(n, seed=seed, vec=0, dtype=dt)
        for p in (2.0, 1.0, 3.0, float("inf")):
            want = oracle.nrm(x, p)
            for dg in (0, 1, 2, 3, 5):
                rows, counts = [], []
                for j in range(1 << dg):
                    first, count = nrm.shard_range(n, dg, j, _code(dt))
                    rows.append(oracle.Z(x[first:first + count], _P(dt), p) if count else np.zeros(_P(dt), dt))
                    counts.append(count)
                got = combine_rows(rows, counts, p, dt)
                assert got.tobytes() == want.tobytes(), (n, p, dg)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, n, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        nb.build()
        nrm.load()
        dg = world.bit_length() - 1
        x = inputs.vector(n, seed=9, vec=0, dtype=np.float64)  # every rank sees only its own shard below
        first, count = nrm.shard_range(n, dg, rank)
        mine = torch.from_numpy(oracle.Z(x[first:first + count], 64, 2.0) if count else np.zeros(64))
        rows = [torch.empty_like(mine) for _ in range(world)]
        dist.all_gather(rows, mine)
        counts = torch.tensor([count], dtype=torch.int64)
        all_counts = [torch.empty_like(counts) for _ in range(world)]
        dist.all_gather(all_counts, counts)
        got = combine_rows([r.numpy() for r in rows], [int(c) for c in all_counts], 2.0, np.float64)
        q.put((rank, got.tobytes()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_protocol_on_gloo_ranks(world):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    n = 3 * (1 << 16) + 11
    procs = [ctx.Process(target=_rank, args=(r, world, port, n, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    want = oracle.nrm(inputs.vector(n, seed=9, vec=0, dtype=np.float64)).tobytes()
    assert all(b == want for _, b in out)
