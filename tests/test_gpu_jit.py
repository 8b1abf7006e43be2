"""Pass-specialised sweep kernels (NQS_OPT_JIT): the generated kernels must
give the oracle's fidelities, level sums and site-set sums within the usual
tolerance, and agree closely with the interpreting kernel on the same
schedule.  Circuits of 12 to 16 qubits run every generated kernel variant
(one and three states, reductions, spawns, checkpoint saves, dense one- and
two-qubit gates, diagonals on register, thread and tile-base qubits)."""

import numpy as np
import pytest

import workloads as W

from _gpu_util import compare, gpu_state, oracle_result

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


def _run(w, level, jit, rb=0):
    from paper_2211_17028_gb300 import nqs
    circ = nqs.NoisyCircuit(W.to_ir_text(w))
    nqs.nqs_set_option(circ.h, nqs.NQS_OPT_JIT, jit)
    if rb:
        nqs.nqs_set_option(circ.h, nqs.NQS_OPT_SWEEP_RB, rb)
    psi, k1 = gpu_state(w.psi, w.n)
    v, k2 = gpu_state(w.v, w.n)
    res = circ.fidelity(psi, v, level)
    terms = circ.term_values()
    info = nqs.nqs_get_info(circ.h)
    launches = nqs.nqs_schedule_launches(circ.h)
    circ.close()
    return res, terms, info, launches


CASES = [
    # (name, workload factory, levels)
    ("random13", lambda: W.random_circuit(41, 13, 90, 6, v_kind="ideal"), (1, 2, 3)),
    ("random14_dense_v", lambda: W.random_circuit(42, 14, 80, 5, v_kind="dense"), (0, 1, 2)),
    ("qaoa16", lambda: W.qaoa_workload(16, 3, 12, 3, "ideal", "qaoa16"), (1, 2)),
    ("grid15", lambda: W.random_circuit(43, 15, 120, 8, noise_kinds=("ad", "pd", "adpd"), v_kind="ideal"), (1, 2)),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_jit_matches_oracle_and_interpreter(case):
    name, make, levels = case
    w = make()
    for level in levels:
        ref = oracle_result(w, level)
        res_j, terms_j, info, launches = _run(w, level, 1)
        assert info["jit_state"] == 1 and info["jit_launches"] > 0, info
        passes = [l for l in launches if l["kind"] == "pass"]
        assert sum(l["jit"] for l in passes) == info["jit_launches"] == len(passes)
        compare(w, level, res_j, terms_j, ref)
        res_i, terms_i, info_i, _ = _run(w, level, 2)
        assert info_i["jit_launches"] == 0
        scale = max(abs(res_i["F"]), 1e-300)
        assert abs(res_j["F"] - res_i["F"]) <= 2e-6 * scale
        assert np.max(np.abs(np.asarray(terms_j) - np.asarray(terms_i))) <= 2e-6 * scale


def test_jit_register_qubits_4_for_three_states():
    w = W.qaoa_workload(16, 5, 10, 3, "ideal", "qaoa16b")
    ref = oracle_result(w, 2)
    res, terms, info, _ = _run(w, 2, 1, rb=4)
    assert info["jit_state"] == 1
    compare(w, 2, res, terms, ref)
