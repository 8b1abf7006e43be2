"""Multi-GPU split of one call (NQS_OPT_SHARD_RANK / NQS_OPT_SHARD_COUNT) on
CPU ranks (gloo, world size 2 and 3): the library's shard masks partition
the kept terms, and per-shard level sums -- here the FP64 oracle's term
values restricted to each shard's terms -- merged by the exchange of a few
doubles (nqs.merge_level_sums_distributed) equal the whole call's sums.  The
GPU side of the same split is checked in tests/test_gpu_shard.py."""

import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _workload():
    import workloads as W
    return W.random_circuit(123, 7, 40, 9, rate_lo=5e-3, rate_hi=5e-2, v_kind="ideal")


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import workloads as W
    from oracle import ir as OIR
    from oracle import o3 as O3
    from paper_2211_17028_gb300 import nqs
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = _workload()
        text = W.to_ir_text(w)
        h = nqs.nqs_load_circuit(text)
        nqs.nqs_prepare_noise(h)
        level = 3
        mask = nqs.nqs_shard_mask(h, level, rank, world)
        r = O3.approximate(OIR.parse(text), w.psi, w.v, level, threads=1)
        x = np.where(mask, r["terms"].real, 0.0)
        off = 0
        import math
        T = []
        for u in range(level + 1):
            cnt = math.comb(w.n_noise, u) * 3 ** u
            T.append(float(np.sum(x[off:off + cnt])))
            off += cnt
        merged, F = nqs.merge_level_sums_distributed(T)
        q.put((rank, mask.tolist(), merged, F, [t.real for t in r["T"]]))
        nqs.nqs_destroy(h)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_shards_partition_terms_and_merge_to_the_whole_call(world):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    got = sorted(q.get(timeout=5) for _ in range(world))
    masks = np.array([g[1] for g in got], dtype=int)
    assert np.all(masks.sum(axis=0) == 1)          # every term on exactly one shard
    assert masks[0][:1 + 3 * 9].all()              # levels 0 and 1 on shard 0
    for rank, _, merged, F, whole in got:
        for u in range(len(whole)):
            assert abs(merged[u] - whole[u]) <= 1e-14 * max(abs(whole[u]), 1e-300) + 1e-18
        assert abs(F - sum(whole)) <= 1e-14


def test_merge_level_sums_single_part_is_identity():
    sys.path.insert(0, ROOT)
    from paper_2211_17028_gb300 import nqs
    T, F = nqs.merge_level_sums([[0.5, 0.25, 1e-9]])
    assert T == [0.5, 0.25, 1e-9] and F == 0.5 + 0.25 + 1e-9
