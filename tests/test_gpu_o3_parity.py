"""GPU parity against O3, the checkpointed FP64 oracle (pinned to the
one-sweep-per-term oracle O2 in tests/test_oracle_o3.py), where the term
counts and widths are beyond O2:

* c2 (4x5 grid, n = 20, 20 AD*PD noises, level 2): every one of the 1771
  terms, the level sums and the fidelity;
* the QAOA generator of the 30-qubit bench workload at n = 22 (a state of
  FP64 checkpoints per site fits the host; n = 30 does not): level sums and
  all 191 level-2 site-set sums, through the pass-specialised kernels;
* batched circuits of width 20 to 24 from the 512-circuit set;
* the n = 20 twin of the 200-noise grid circuit at level 3 (35.6 M terms):
  the full enumeration's per-set sums W(S) on the heaviest and on random
  sets against O3's evaluation of those sets.
Tolerances: 1e-5 relative on F, 1e-5 * F absolute on T_u, site-set sums and
terms (the target tolerance); for the level-3 sets, whose W(S) are
~1e-12 of F, 1e-3 relative on sets with W(S) >= 1e-3 max W -- complex64
amplitudes of magnitude |a| carry an absolute error of about 1e-7 * ||phi|| ||w||
summed over ~700 operations, far below 1e-3 |a| for those sets.
"""

import itertools
import math

import numpy as np
import pytest

import workloads as W
from oracle import ir as OIR
from oracle import o3 as O3

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


def _gpu(w, level, jit=0):
    from paper_2211_17028_gb300 import nqs
    circ = nqs.NoisyCircuit(W.to_ir_text(w))
    nqs.nqs_set_option(circ.h, nqs.NQS_OPT_JIT, jit)
    psi, k1 = gpu_state(w.psi, w.n)
    v, k2 = gpu_state(w.v, w.n)
    res = circ.fidelity(psi, v, level)
    terms = circ.term_values()
    info = nqs.nqs_get_info(circ.h)
    circ.close()
    return res, terms, info


def test_grid20_level2_every_term():
    w = W.c2_grid20()
    res, terms, _ = _gpu(w, 2)
    errs = compare(w, 2, res, terms, oracle_result(w, 2), check_terms=True)
    assert errs["term_abs"] <= 1e-5 * abs(res["F"])


def test_qaoa22_level2_all_site_sets_generated_kernels():
    w = W.qaoa_workload(22, 3, 20, 4, "ideal", "qaoa22")
    res, terms, info = _gpu(w, 2, jit=1)
    assert info["jit_state"] == 1 and info["jit_launches"] > 0
    compare(w, 2, res, terms, oracle_result(w, 2))


WIDE = [299, 313, 227, 321, 174, 3]   # widths 20, 20, 21, 22, 23, 24 (levels 1, 2, 1, 1, 1, 1)


def test_batch_wide_circuits_match_o3():
    from paper_2211_17028_gb300 import nqs
    ws = [W.c4_circuit(i) for i in WIDE]
    assert sorted(w.n for w in ws) == [20, 20, 21, 22, 23, 24]
    circs = [nqs.NoisyCircuit(W.to_ir_text(w)) for w in ws]
    outs = nqs.nqs_batch_fidelity([c.h for c in circs], [nqs.basis(w.psi["bits"]) for w in ws],
                                  [nqs.ideal() for _ in ws], [w.levels[0] for w in ws])
    for w, c, o in zip(ws, circs, outs):
        compare(w, w.levels[0], o.to_dict(), c.term_values(), oracle_result(w, w.levels[0]))
        c.close()


def test_twin20_level3_sets_match_o3():
    from paper_2211_17028_gb300 import nqs
    w = W.c5_twin()
    N = w.n_noise
    circ = nqs.NoisyCircuit(W.to_ir_text(w))
    res = circ.fidelity(nqs.basis(w.psi["bits"]), nqs.ideal(), 3)
    assert res["status"] == 0 and res["n_terms"] == 35641501
    vals = circ.term_values()
    circ.close()
    o3 = 1 + 3 * N + 9 * (N * (N - 1) // 2)
    W3 = vals[o3:].reshape(-1, 27).sum(1)
    del vals
    assert abs(W3.sum() - res["T"][3]) <= 1e-9 * abs(res["T"][3])
    sets = list(itertools.combinations(range(N), 3))
    order = np.argsort(-W3)
    heavy = [int(i) for i in order[:4]]
    rng = np.random.default_rng(2211)
    big = np.flatnonzero(W3 >= 1e-3 * W3[order[0]])
    rand = [int(i) for i in rng.choice(big, size=min(4, big.size), replace=False) if int(i) not in heavy]
    pick = heavy + rand
    c = OIR.parse(W.to_ir_text(w))
    want = O3.set_weights(c, w.psi, w.v, np.array([sets[i] for i in pick])).real
    for i, x in zip(pick, want):
        assert abs(W3[i] - x) <= 1e-3 * abs(x), (sets[i], W3[i], x)
