"""The bench's multi-GPU form is replicas: two gloo ranks on the CPU check the
max-over-ranks timing and the weak-scaling aggregate (no GPU needed)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, value = bench.aggregate_ranks(10.0 * (rank + 1), ops_per_step=10 ** 9, steps=4, world=world)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ms, value))


def test_two_rank_aggregate():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    # both ranks see the slowest rank's 20 ms; the value counts both ranks' work
    for _, ms, value in out:
        assert ms == 20.0
        assert value == pytest.approx(2 * 4 * 10 ** 9 / 0.020 / 1e9)


def test_single_rank_aggregate():
    sys.path.insert(0, ROOT)
    import bench
    ms, value = bench.aggregate_ranks(8.0, ops_per_step=10 ** 9, steps=2, world=1)
    assert ms == 8.0 and value == pytest.approx(2 * 10 ** 9 / 0.008 / 1e9)
