"""Adaptive level selection (nqs_fidelity_adaptive): the level the library
stops at is the one the truncation bound (oracle/bounds.per_site_bound) or
the observed level sums of the oracle predict, and the fidelity is the
oracle's A(l) at that level."""

import pytest

import workloads as W
from oracle import bounds as OB
from oracle import ir as OIR

from _gpu_util import REL_TOL, oracle_result

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup():
    import torch
    from paper_2211_17028_gb300 import nqs
    torch.cuda.set_device(0)
    nqs.use_torch_allocator()
    yield


CASES = [("line6", W.c1_line6), ("random9", lambda: W.random_circuit(91, 9, 60, 6, v_kind="ideal",
                                                                          rate_lo=5e-3, rate_hi=5e-2))]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_bound_criterion_stops_where_the_bound_says(name, make):
    from paper_2211_17028_gb300 import nqs
    w = make()
    c = OIR.parse(W.to_ir_text(w))
    kl = [z[2] for z in c.noises]
    N = len(kl)
    circ = nqs.NoisyCircuit(W.to_ir_text(w))
    psi, v = nqs.basis(w.psi["bits"]), (nqs.ideal() if w.v["kind"] == "ideal" else nqs.basis(w.v["bits"]))
    bounds = [OB.per_site_bound(kl, l) for l in range(N + 1)]
    for l_want in range(0, min(N, 3) + 1):
        # a tolerance between bound(l_want) and bound(l_want - 1)
        hi = bounds[l_want - 1] if l_want > 0 else 1.0
        tol = (bounds[l_want] * hi) ** 0.5 if bounds[l_want] > 0 else 0.5 * hi
        r = nqs.nqs_fidelity_adaptive(circ.h, psi, v, tol, criteria=nqs.NQS_ADAPT_BOUND)
        assert r["level"] == l_want, (name, tol, r["level"], bounds[:4])
        ref = oracle_result(w, l_want, keep_terms=False)
        assert abs(r["F"] - ref["F"].real) <= REL_TOL * abs(ref["F"].real)
    circ.close()


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_observed_criterion_stops_at_the_first_small_level_sum(name, make):
    from paper_2211_17028_gb300 import nqs
    w = make()
    N = w.n_noise
    ref = oracle_result(w, N, keep_terms=False)
    T = [abs(t.real) for t in ref["T"]]
    circ = nqs.NoisyCircuit(W.to_ir_text(w))
    psi, v = nqs.basis(w.psi["bits"]), (nqs.ideal() if w.v["kind"] == "ideal" else nqs.basis(w.v["bits"]))
    for l_want in (1, 2):
        # between |T_l_want| and every earlier |T_l| (l >= 1)
        earlier = min(T[1:l_want]) if l_want > 1 else T[l_want] * 10.0
        tol = (T[l_want] * earlier) ** 0.5
        r = nqs.nqs_fidelity_adaptive(circ.h, psi, v, tol, max_level=N, criteria=nqs.NQS_ADAPT_OBSERVED)
        assert r["level"] == l_want, (name, tol, T[:4], r["level"])
        lvl = oracle_result(w, l_want, keep_terms=False)
        assert abs(r["F"] - lvl["F"].real) <= REL_TOL * abs(lvl["F"].real)
    # both criteria: the earlier stop wins; max_level caps
    r = nqs.nqs_fidelity_adaptive(circ.h, psi, v, 0.0, max_level=1)
    assert r["level"] == 1
    with pytest.raises(nqs.NqsError):
        nqs.nqs_fidelity_adaptive(circ.h, psi, v, 1e-6, criteria=0)
    circ.close()
