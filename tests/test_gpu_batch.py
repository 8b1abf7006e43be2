"""Batched evaluation (nqs_batch_fidelity) against the plain per-circuit path
and the FP64 oracle, on seeded circuits of uneven width, depth, noise count
and level (the batched-configuration generator, narrowed to widths the
oracle finishes quickly)."""

import numpy as np
import pytest

import workloads as W

from _gpu_util import compare, oracle_result

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup():
    import torch
    from paper_2211_17028_gb300 import nqs
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    nqs.use_torch_allocator()
    yield
    torch.cuda.synchronize()


def _narrow_batch(count, seed0, n_lo=12, n_hi=15):
    out = []
    for i in range(count):
        w = W.c4_circuit(seed0 + i)
        rng = W.SplitMix64(99 + i)
        # keep the generator's structure but bound the width for the oracle
        n = n_lo + rng.randbelow(n_hi - n_lo + 1)
        w2 = W.random_circuit(5000 + i, n, min(len(w.gates), 60), min(w.n_noise, 8), v_kind="ideal",
                              rate_lo=1e-4, rate_hi=1e-2)
        w2.levels = w.levels
        out.append(w2)
    return out


def _plain(ws):
    from paper_2211_17028_gb300 import nqs
    res = []
    for w in ws:
        c = nqs.NoisyCircuit(W.to_ir_text(w))
        res.append(c.fidelity(nqs.basis(w.psi["bits"]), nqs.ideal(), w.levels[0]))
        c.close()
    return res


def test_batch_equals_plain_path_and_replays():
    from paper_2211_17028_gb300 import nqs
    ws = _narrow_batch(24, 0)
    plain = _plain(ws)
    circs = [nqs.NoisyCircuit(W.to_ir_text(w)) for w in ws]
    hs = [c.h for c in circs]
    psis = [nqs.basis(w.psi["bits"]) for w in ws]
    vs = [nqs.ideal() for _ in ws]
    levels = [w.levels[0] for w in ws]
    for call in range(3):          # first call builds and captures, later calls replay
        outs = nqs.nqs_batch_fidelity(hs, psis, vs, levels)
        for w, p, o in zip(ws, plain, outs):
            d = o.to_dict()
            assert d["status"] == 0
            assert d["F"] == p["F"] and d["T"] == p["T"], (w.name, call, d["F"], p["F"])
            assert d["n_terms"] == p["n_terms"]
    # term values of a batched handle are the plain path's
    t = circs[3].term_values()
    c = nqs.NoisyCircuit(W.to_ir_text(ws[3]))
    c.fidelity(nqs.basis(ws[3].psi["bits"]), nqs.ideal(), levels[3])
    assert np.array_equal(t, c.term_values())
    c.close()
    for c in circs:
        c.close()


def test_batch_matches_oracle():
    from paper_2211_17028_gb300 import nqs
    ws = _narrow_batch(6, 100, 12, 13)
    circs = [nqs.NoisyCircuit(W.to_ir_text(w)) for w in ws]
    outs = nqs.nqs_batch_fidelity([c.h for c in circs], [nqs.basis(w.psi["bits"]) for w in ws],
                                  [nqs.ideal() for _ in ws], [w.levels[0] for w in ws])
    for w, c, o in zip(ws, circs, outs):
        compare(w, w.levels[0], o.to_dict(), c.term_values(), oracle_result(w, w.levels[0]))
        c.close()


def test_batch_rejects_bad_entries():
    from paper_2211_17028_gb300 import nqs
    w = W.random_circuit(7, 12, 30, 3, v_kind="ideal")
    c = nqs.NoisyCircuit(W.to_ir_text(w))
    with pytest.raises(nqs.NqsError) as e:
        nqs.nqs_batch_fidelity([c.h, c.h], [nqs.basis(0)] * 2, [nqs.ideal()] * 2, [1, 1])
    assert e.value.code == nqs.NQS_ERR_ARG
    with pytest.raises(nqs.NqsError) as e:
        nqs.nqs_batch_fidelity([c.h], [nqs.ideal()], [nqs.ideal()], [1])
    assert e.value.code == nqs.NQS_ERR_ARG
    c.close()
