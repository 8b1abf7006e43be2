"""The N > 1 measurement path of bench.py on CPU ranks (gloo, world size 2).

With one process per GPU each rank evaluates its own replica; the only
exchange is the measurement itself: the timed region is the maximum over
ranks and the units are summed.  The reference arm runs on rank 0 alone."""

import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t, u = bench.aggregate(1.5 + rank, 100.0 * (rank + 1))
        assert bench.dist_env() == (world, rank, rank)
        # a rank other than 0 leaves the reference arm without work
        rc = bench.run_reference(type("A", (), {"workload": "line6_l4"})()) if rank else 0
        q.put((rank, t, u, rc))
    finally:
        dist.destroy_process_group()


def test_aggregate_max_time_sum_units_two_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    got = sorted(q.get(timeout=5) for _ in range(2))
    for rank, t, u, rc in got:
        assert t == pytest.approx(2.5)
        assert u == pytest.approx(300.0)
        assert rc == 0


def test_aggregate_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(3.25, 7.0) == (3.25, 7.0)
