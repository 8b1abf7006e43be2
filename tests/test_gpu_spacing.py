"""Spaced checkpoints and the execution options (nqs_set_option, nqs_autotune).

With checkpoint spacing k the backward sweep keeps phi only at the last site
of each block of k sites and recomputes a block's phi whenever a sweep enters
it; the expansion it computes is unchanged.  Checked against the FP64 oracle
(F, every T_u, every site-set sum) and against the schedule that keeps every
site, for several k including blocks of one site and a ragged last block."""

import numpy as np
import pytest

import workloads as W

from _gpu_util import REL_TOL, compare, oracle_result

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup():
    import torch
    from paper_2211_17028_gb300 import nqs
    torch.cuda.set_device(0)
    nqs.use_torch_allocator()
    yield


def _spaced_states(N, level, k):
    return -(-N // k) + k + 2 + (3 * k if level >= 2 else 0)


@pytest.mark.parametrize("n,seed,noise", [(13, 91, 10), (8, 92, 7)])
@pytest.mark.parametrize("level", [1, 2])
def test_spaced_checkpoints_match_oracle(n, seed, noise, level):
    from paper_2211_17028_gb300 import nqs
    w = W.random_circuit(seed, n, 60, noise, rate_lo=1e-3, rate_hi=3e-2)
    ref = oracle_result(w, level)
    circ = nqs.NoisyCircuit(W.to_ir_text(w))
    psi, v = nqs.basis(w.psi["bits"]), nqs.basis(w.v["bits"])
    full = circ.fidelity(psi, v, level)
    assert nqs.nqs_get_info(circ.h)["ckpt_spacing"] == 0
    for k in (1, 3, 4):
        nqs.nqs_set_option(circ.h, nqs.NQS_OPT_CKPT_SPACING, k)
        res = circ.fidelity(psi, v, level)
        info = nqs.nqs_get_info(circ.h)
        assert info["ckpt_spacing"] == k
        assert info["n_states"] == _spaced_states(w.n_noise, level, k)
        compare(w, level, res, circ.term_values(), ref)
        assert abs(res["F"] - full["F"]) <= 1e-6 * abs(full["F"])
    nqs.nqs_set_option(circ.h, nqs.NQS_OPT_CKPT_SPACING, 0)
    circ.close()


def test_spacing_option_errors_and_level3():
    from paper_2211_17028_gb300 import nqs
    w = W.random_circuit(93, 6, 30, 5)
    circ = nqs.NoisyCircuit(W.to_ir_text(w))
    psi, v = nqs.basis(w.psi["bits"]), nqs.basis(w.v["bits"])
    nqs.nqs_set_option(circ.h, nqs.NQS_OPT_CKPT_SPACING, 2)
    assert nqs.nqs_get_option(circ.h, nqs.NQS_OPT_CKPT_SPACING) == 2
    with pytest.raises(nqs.NqsError) as e:
        circ.fidelity(psi, v, 3)
    assert e.value.code == nqs.NQS_ERR_UNSUPPORTED
    # k >= N keeps every site
    nqs.nqs_set_option(circ.h, nqs.NQS_OPT_CKPT_SPACING, 5)
    r = circ.fidelity(psi, v, 3)
    assert r["status"] == 0 and nqs.nqs_get_info(circ.h)["ckpt_spacing"] == 0
    for opt, bad in ((nqs.NQS_OPT_SWEEP_RB, 5), (nqs.NQS_OPT_MAX_OPS, 4), (nqs.NQS_OPT_MAX_SITES, 9), (99, 1)):
        with pytest.raises(nqs.NqsError) as e:
            nqs.nqs_set_option(circ.h, opt, bad)
        assert e.value.code == nqs.NQS_ERR_ARG
    circ.close()


def test_segmentation_options_and_autotune_keep_results():
    from paper_2211_17028_gb300 import nqs
    w = W.random_circuit(94, 14, 90, 8, rate_lo=1e-3, rate_hi=3e-2)
    ref = oracle_result(w, 2)
    circ = nqs.NoisyCircuit(W.to_ir_text(w))
    psi, v = nqs.basis(w.psi["bits"]), nqs.basis(w.v["bits"])
    for rb, ops, sites in ((3, 64, 2), (4, 128, 8), (4, 8, 1)):
        nqs.nqs_set_option(circ.h, nqs.NQS_OPT_SWEEP_RB, rb)
        nqs.nqs_set_option(circ.h, nqs.NQS_OPT_MAX_OPS, ops)
        nqs.nqs_set_option(circ.h, nqs.NQS_OPT_MAX_SITES, sites)
        compare(w, 2, circ.fidelity(psi, v, 2), circ.term_values(), ref)
    nqs.nqs_set_option(circ.h, nqs.NQS_OPT_MAX_SITES, 0)
    res = nqs.nqs_autotune(circ.h, psi, v, 2, trials=2)
    assert nqs.nqs_get_option(circ.h, nqs.NQS_OPT_SWEEP_RB) in (3, 4)
    assert nqs.nqs_get_option(circ.h, nqs.NQS_OPT_MAX_OPS) in (64, 96, 128)
    assert abs(res["F"] - ref["F"].real) <= REL_TOL * abs(ref["F"].real)
    compare(w, 2, circ.fidelity(psi, v, 2), circ.term_values(), ref)
    circ.close()
