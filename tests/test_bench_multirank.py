"""The multi-rank aggregation of bench.py, on CPU with two gloo ranks:
each rank times its own problem, the job's step time is the maximum over
ranks and the value counts all ranks' bytes (weak scaling, no data-path
collective)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    total_ms = [120.0, 150.0][rank]  # rank 1 is the slowest
    ms, value = bench.aggregate(total_ms, world, 10, 3 << 30, dist, "cpu")
    q.put((rank, ms, value))
    dist.destroy_process_group()


def test_aggregate_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    want_value = 2 * 10 * (3 << 30) / 0.150 / 1e9
    for rank, ms, value in out:
        assert ms == 150.0
        assert abs(value - want_value) < 1e-6 * want_value


def test_aggregate_single_rank():
    import bench
    ms, value = bench.aggregate(100.0, 1, 5, 1 << 30, None, None)
    assert ms == 100.0 and abs(value - 5 * (1 << 30) / 0.1 / 1e9) < 1e-9
