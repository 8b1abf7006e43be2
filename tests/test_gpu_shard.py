"""The multi-GPU split of one call, run shard after shard on one GPU: each
shard's term values are zero outside its terms (nqs_shard_mask) and equal
to the unsplit call's inside them; the shards' level sums merged with
nqs.merge_level_sums equal the unsplit call's T_u -- with every checkpoint
kept and with spaced checkpoints."""

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup():
    import torch
    from paper_2211_17028_gb300 import nqs
    torch.cuda.set_device(0)
    nqs.use_torch_allocator()
    yield


@pytest.mark.parametrize("spacing,count", [(0, 3), (3, 2)])
def test_shards_merge_to_the_unsplit_call(spacing, count):
    from paper_2211_17028_gb300 import nqs
    w = W.random_circuit(131, 13, 80, 9, rate_lo=5e-3, rate_hi=5e-2, v_kind="ideal")
    text = W.to_ir_text(w)
    psi, v = nqs.basis(w.psi["bits"]), nqs.ideal()
    level = 3 if spacing == 0 else 2

    def run(rank, cnt):
        c = nqs.NoisyCircuit(text)
        if spacing:
            nqs.nqs_set_option(c.h, nqs.NQS_OPT_CKPT_SPACING, spacing)
        if cnt:
            nqs.nqs_set_option(c.h, nqs.NQS_OPT_SHARD_COUNT, cnt)
            nqs.nqs_set_option(c.h, nqs.NQS_OPT_SHARD_RANK, rank)
        r = c.fidelity(psi, v, level)
        vals = c.term_values()
        mask = nqs.nqs_shard_mask(c.h, level, rank, max(cnt, 1))
        c.close()
        return r, vals, mask

    whole, wvals, _ = run(0, 0)
    parts = []
    for rank in range(count):
        r, vals, mask = run(rank, count)
        assert r["status"] == 0
        assert np.all(vals[~mask] == 0.0)
        assert np.allclose(vals[mask], wvals[mask], rtol=1e-6, atol=1e-12 * abs(whole["F"]))
        parts.append(r["T"])
    T, F = nqs.merge_level_sums(parts)
    for u in range(level + 1):
        assert abs(T[u] - whole["T"][u]) <= 1e-6 * abs(whole["F"]) * 1e-3, (u, T[u], whole["T"][u])
    assert abs(F - whole["F"]) <= 1e-9 * abs(whole["F"])
    with pytest.raises(nqs.NqsError):
        c = nqs.NoisyCircuit(text)
        nqs.nqs_set_option(c.h, nqs.NQS_OPT_SHARD_COUNT, 2)
        nqs.nqs_set_option(c.h, nqs.NQS_OPT_SHARD_RANK, 2)
        try:
            c.fidelity(psi, v, 1)
        finally:
            c.close()
