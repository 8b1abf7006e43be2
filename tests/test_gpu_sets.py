"""Site-set weights W(S) (nqs_prepare_sets / nqs_eval_sets) against the FP64
oracle: W(S) is the sum of the oracle's term values over the factor tuples of
the site set S (Algorithm 1's inner loop), compared for every set of sizes
1, 2 and 3 on circuits below and above the 12-qubit tile width."""

import itertools

import numpy as np
import pytest

import workloads as W

from _gpu_util import REL_TOL, oracle_result, site_sets

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup():
    import torch
    from paper_2211_17028_gb300 import nqs
    torch.cuda.set_device(0)
    nqs.use_torch_allocator()
    yield


@pytest.mark.parametrize("n,seed,noise", [(5, 71, 5), (13, 72, 5), (14, 73, 6)])
def test_site_set_weights_match_oracle(n, seed, noise):
    from paper_2211_17028_gb300 import nqs
    w = W.random_circuit(seed, n, 50, noise, v_kind="ideal", rate_lo=1e-3, rate_hi=3e-2)
    ref = oracle_result(w, 3)
    recs = [r for r, _ in ref["terms"]]
    want = site_sets(recs, [x.real for _, x in ref["terms"]])
    F = ref["F"].real
    circ = nqs.NoisyCircuit(W.to_ir_text(w))
    nqs.nqs_prepare_sets(circ.h, nqs.basis(w.psi["bits"]), nqs.ideal())
    N = w.n_noise
    for k in (1, 2, 3):
        sets = np.array(list(itertools.combinations(range(N), k)), dtype=np.int32)
        got = nqs.nqs_eval_sets(circ.h, sets)
        for s, g in zip(sets, got):
            assert abs(g - want[tuple(int(x) for x in s)]) <= REL_TOL * abs(F), (k, s, g, want[tuple(s)])
    circ.close()


def test_site_set_argument_errors():
    from paper_2211_17028_gb300 import nqs
    w = W.random_circuit(74, 4, 20, 3)
    circ = nqs.NoisyCircuit(W.to_ir_text(w))
    with pytest.raises(nqs.NqsError) as e:
        nqs.nqs_eval_sets(circ.h, np.array([[0, 1]]))
    assert e.value.code == nqs.NQS_ERR_ORDER
    nqs.nqs_prepare_sets(circ.h, nqs.basis(w.psi["bits"]), nqs.basis(w.v["bits"]))
    for bad in ([[1, 0]], [[0, 0]], [[0, 5]], [[0, 1, 2, 2]]):
        with pytest.raises(nqs.NqsError) as e:
            nqs.nqs_eval_sets(circ.h, np.array(bad))
        assert e.value.code == nqs.NQS_ERR_ARG
    circ.close()


@pytest.mark.parametrize("spacing", [1, 2, 3])
def test_site_set_weights_with_spaced_checkpoints(spacing):
    """Checkpoints kept every `spacing` sites (chi at block-first, phi at
    block-last sites, the rest recomputed per call) give the same W(S)."""
    from paper_2211_17028_gb300 import nqs
    w = W.random_circuit(75, 13, 60, 7, v_kind="ideal", rate_lo=1e-3, rate_hi=3e-2)
    ref = oracle_result(w, 3)
    want = site_sets([r for r, _ in ref["terms"]], [x.real for _, x in ref["terms"]])
    F = ref["F"].real
    circ = nqs.NoisyCircuit(W.to_ir_text(w))
    nqs.nqs_set_option(circ.h, nqs.NQS_OPT_CKPT_SPACING, spacing)
    nqs.nqs_prepare_sets(circ.h, nqs.basis(w.psi["bits"]), nqs.ideal())
    N = w.n_noise
    for k in (1, 2, 3):
        sets = np.array(list(itertools.combinations(range(N), k)), dtype=np.int32)
        # shuffled order: the evaluation sorts internally and must map values back
        perm = np.random.default_rng(k).permutation(len(sets))
        got = nqs.nqs_eval_sets(circ.h, sets[perm])
        for s, g in zip(sets[perm], got):
            assert abs(g - want[tuple(int(x) for x in s)]) <= REL_TOL * abs(F), (spacing, k, s, g)
    circ.close()
