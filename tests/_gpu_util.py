"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI
and the oracle on the same seeded workload, then compare."""

import math

import numpy as np

import workloads as W
from oracle import csim
from oracle import expansion as OEX
from oracle import ir as OIR
from oracle import o3 as O3

# tolerance: every fidelity within 1e-5 relative of the FP64 oracle;
# T_u, per-site-set sums and individual terms within 1e-5 * F absolute
REL_TOL = 1e-5


def oracle_result(w, level, keep_terms=True):
    """O2 (one sweep per network per term) up to 10 qubits, O3 (checkpointed,
    pinned to O2) above; the same dict either way."""
    c = OIR.parse(W.to_ir_text(w))
    if w.n <= 10:
        return OEX.approximate(c, w.psi, w.v, level, keep_terms=keep_terms)
    r = O3.approximate(c, w.psi, w.v, level)
    if keep_terms:
        recs = OEX.enumerate_records(len(c.noises), min(level, len(c.noises)))
        r["terms"] = list(zip(recs, r["terms"]))
    else:
        r["terms"] = []
    return r


def gpu_state(spec, n):
    """nqs_state plus the tensor that must stay alive for the call."""
    import torch
    from paper_2211_17028_gb300 import nqs
    if spec["kind"] == "basis":
        return nqs.basis(spec["bits"]), None
    if spec["kind"] == "ideal":
        return nqs.ideal(), None
    t = torch.tensor(np.asarray(spec["amps"], dtype=np.complex64), device="cuda")
    return nqs.dense(t), t


def gpu_result(w, level, flags=0):
    from paper_2211_17028_gb300 import nqs
    circ = nqs.NoisyCircuit(W.to_ir_text(w), None, flags)
    psi, keep1 = gpu_state(w.psi, w.n)
    v, keep2 = gpu_state(w.v, w.n)
    res = circ.fidelity(psi, v, level)
    terms = circ.term_values()
    circ.close()
    return res, terms


def nondegenerate(w, rtol=1e-6):
    """True when every channel's four singular values are pairwise distinct,
    so individual terms do not depend on a basis choice."""
    for z in w.noises:
        d = OEX.svd_factors(z.kraus)[0]
        for i in range(4):
            for j in range(i + 1, 4):
                if abs(d[i] - d[j]) <= rtol * d[0]:
                    return False
    return True


def site_sets(records, values):
    out = {}
    for r, x in zip(records, values):
        k = r & 15
        key = tuple(((r >> (4 + 14 * j)) & 0xFFF) for j in range(k))
        out[key] = out.get(key, 0.0) + x
    return out


def compare(w, level, res, terms, ref, check_terms=None):
    F = ref["F"].real
    scale = max(abs(F), 1e-300)
    errs = {"F_rel": abs(res["F"] - F) / scale}
    assert res["status"] == 0
    assert res["n_terms"] == ref["n_terms"] == len(terms)
    assert errs["F_rel"] <= REL_TOL, (w.name, level, res["F"], F, errs)
    for u, t in enumerate(ref["T"]):
        assert abs(res["T"][u] - t.real) <= REL_TOL * scale, (w.name, level, u, res["T"][u], t)
    recs = [r for r, _ in ref["terms"]]
    want = [x.real for _, x in ref["terms"]]
    got_sets = site_sets(recs, terms)
    want_sets = site_sets(recs, want)
    worst = 0.0
    for key, val in want_sets.items():
        worst = max(worst, abs(got_sets[key] - val))
    errs["site_set_abs"] = worst
    assert worst <= REL_TOL * scale, (w.name, level, worst, scale)
    if check_terms is None:
        check_terms = nondegenerate(w)
    if check_terms:
        d = np.max(np.abs(np.asarray(terms) - np.asarray(want)))
        errs["term_abs"] = float(d)
        assert d <= REL_TOL * scale, (w.name, level, d, scale)
    assert min(terms) >= -1e-7 * scale
    return errs
