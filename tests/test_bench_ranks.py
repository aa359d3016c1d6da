"""The multi-rank path of bench.py on CPU: world size 2 over gloo.

With N processes (one per GPU) every rank runs its own replica of the
evaluation; the bench takes the timed milliseconds of the slowest rank (an
all-reduce MAX) and reports the work of all ranks over that time.  Only the
reduction crosses ranks, so it is tested here with gloo on the host.
"""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        dist.barrier()
        # rank r was timed at 100 (r + 1) ms over 2 steps
        ms, value = bench.aggregate_over_ranks(100.0 * (rank + 1), 2, world, dist, "cpu")
        q.put((rank, ms, value))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_aggregate_throughput():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    got = sorted(q.get(timeout=10) for _ in range(world))
    for rank, ms, value in got:
        # slowest rank: 200 ms over 2 steps; two replicas -> 2 evaluations per 100 ms
        assert ms == pytest.approx(100.0), rank
        assert value == pytest.approx(20.0), rank


def test_single_rank_needs_no_process_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    ms, value = bench.aggregate_over_ranks(300.0, 3, 1, None, "cpu")
    assert ms == pytest.approx(100.0) and value == pytest.approx(10.0)
