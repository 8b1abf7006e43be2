"""Parity at full size: the 30-qubit QAOA workload at level 2, run through
the C ABI in the launch configuration the benchmark times (8 GiB states).

The oracle cannot contract the 1771 networks of 30 qubits in seconds, so it
computes sampled outputs one by one with the help of a property of this
workload: v = U|psi> and every noise is depolarizing, whose dominant factors
are multiples of the identity (Sec. IV: U_0 = c I, V_0 = c' I).  With every
other site on its dominant factor, the two networks of a term with insertions
at sites s < t reduce to

    a = prod_{u not in S} c_u  * <chi_t| U_j  W  U_i |chi_s>
    b = prod_{u not in S} c'_u * conj(<chi_t| conj(V_j) W conj(V_i) |chi_s>)

(chi_s = gates before site s applied to psi, W = gates between s and t), so
the oracle needs only the prefix of the circuit up to the sampled sites,
swept in FP64 by its C state-vector code (one forward pass through the whole
circuit prefix, at 16 GiB per FP64 state).  Checked: T_0, the level-1 sums of
the first six sites, and the level-2 sums of the pairs among them at most 14
operations apart (the oracle sweeps the gap between them for each factor),
each within 1e-5 F and, as these sums are far below F, within 1% of itself;
T_1 equals the sum of all 20 level-1 site sums; F = T_0 + T_1 + T_2."""

import numpy as np
import pytest

import workloads as W
from oracle import csim
from oracle import expansion as OEX
from oracle import gates as G
from oracle import ir as OIR

from _gpu_util import REL_TOL, site_sets

pytestmark = pytest.mark.gpu


def _gate_ops(c, e0, e1):
    """Gates among events [e0, e1) as one op list (noise events skipped)."""
    ops = csim.OpList()
    for e, (kind, idx) in enumerate(OIR.events(c)):
        if e0 <= e < e1 and kind == "gate":
            name, qs, ps = c.gates[idx]
            ops.add(qs, G.gate_matrix(name, ps))
    return ops


def _one(q, m):
    ops = csim.OpList()
    ops.add((q,), m)
    return ops


def _identity_scale(m):
    assert abs(m[0, 1]) < 1e-12 and abs(m[1, 0]) < 1e-12 and abs(m[0, 0] - m[1, 1]) < 1e-12
    return complex(m[0, 0])


def test_qaoa30_level2_sampled_terms():
    import torch
    from paper_2211_17028_gb300 import nqs
    torch.cuda.set_device(0)
    nqs.use_torch_allocator()
    w = W.c3_qaoa30()
    text = W.to_ir_text(w)
    circ = nqs.NoisyCircuit(text)
    res = circ.fidelity(nqs.basis(0), nqs.ideal(), 2)
    recs = nqs.nqs_enumerate_terms(circ.h, 2)
    vals = circ.term_values()
    circ.close()
    torch.cuda.empty_cache()
    assert res["status"] == 0 and res["n_terms"] == 1771
    F = res["F"]
    got = site_sets(recs, vals)
    assert abs(F - sum(res["T"])) <= 1e-12 * F
    assert abs(res["T"][1] - sum(got[(s,)] for s in range(w.n_noise))) <= 1e-9 * F

    c = OIR.parse(text)
    fac = OEX.prepared_factors(c)
    cu = [_identity_scale(f[1][0]) for f in fac]
    cv = [_identity_scale(f[2][0]) for f in fac]
    ev = {idx: e for e, (kind, idx) in enumerate(OIR.events(c)) if kind == "noise"}

    def rest(S):
        a = b = 1.0
        for u in range(len(fac)):
            if u not in S:
                a, b = a * cu[u], b * cv[u]
        return a * b

    T0 = rest(())
    assert abs(res["T"][0] - T0.real) <= REL_TOL * F, (res["T"][0], T0)

    n = c.n
    # the oracle's FP64 sweep costs about a second per operation at n = 30, so the
    # sample stops at the sixth site (the first ~175 operations): level-1 sums of
    # sites 0..5 and level-2 sums of the site pairs among them at most 14
    # operations apart
    N = 6
    pairs = [(s, t) for s in range(N) for t in range(s + 1, N) if ev[t] - ev[s] <= 14]
    assert len(pairs) >= 2
    firsts = {s for s, _ in pairs}
    chi = np.zeros(1 << n, dtype=np.complex128)
    chi[0] = 1.0
    pos = 0
    saved = {}
    for s in range(N):
        csim.apply_ops(n, chi, _gate_ops(c, pos, ev[s]))
        pos = ev[s]
        q = c.noises[s][1]
        W1 = 0.0
        for i in (1, 2, 3):
            x = chi.copy()
            csim.apply_ops(n, x, _one(q, fac[s][1][i]))
            a = csim.inner(n, chi, x)
            x[:] = chi
            csim.apply_ops(n, x, _one(q, fac[s][2][i].conj()))
            b = csim.inner(n, chi, x).conjugate()
            del x
            W1 += (a * b).real
        W1 *= rest((s,)).real
        assert abs(got[(s,)] - W1) <= REL_TOL * F, (s, got[(s,)], W1)
        # the sums are far below F here: also hold each to 1% of itself
        assert abs(got[(s,)] - W1) <= 1e-2 * W1, (s, got[(s,)], W1)
        # level 2: every close pair ending here, from the saved chi of its first site
        for (s0, t) in pairs:
            if t != s:
                continue
            q0 = c.noises[s0][1]
            between = _gate_ops(c, ev[s0], ev[t])
            W2 = 0.0
            for i in (1, 2, 3):
                amps = {}
                for side in (1, 2):
                    y = saved[s0].copy()
                    m0 = fac[s0][side][i] if side == 1 else fac[s0][side][i].conj()
                    csim.apply_ops(n, y, _one(q0, m0))
                    csim.apply_ops(n, y, between)
                    for j in (1, 2, 3):
                        z = y.copy()
                        m1 = fac[t][side][j] if side == 1 else fac[t][side][j].conj()
                        csim.apply_ops(n, z, _one(q, m1))
                        amps[(side, j)] = csim.inner(n, chi, z)
                        del z
                    del y
                for j in (1, 2, 3):
                    W2 += (amps[(1, j)] * amps[(2, j)].conjugate()).real
            W2 *= rest((s0, t)).real
            assert abs(got[(s0, t)] - W2) <= REL_TOL * F, ((s0, t), got[(s0, t)], W2)
            assert abs(got[(s0, t)] - W2) <= 1e-2 * W2, ((s0, t), got[(s0, t)], W2)
        if s in firsts:
            saved[s] = chi.copy()
        for s0 in list(saved):
            if all(t <= s for (a0, t) in pairs if a0 == s0):
                del saved[s0]
    del chi


def test_n31_level1_needs_spaced_checkpoints():
    """A 31-qubit circuit (16 GiB states) with 20 depolarizing noises: keeping
    phi at every site (21 states, 336 GiB) does not fit in HBM, so the engine
    keeps it every k sites and recomputes the rest.  Checked at full size:
    T_0 = prod_s |c_s c'_s| (dominant factors are multiples of the identity
    and v = U|psi>), F = T_0 + T_1, and the level-1 sums of the first two
    sites against the oracle's FP64 prefix sweep."""
    import torch
    from paper_2211_17028_gb300 import nqs
    torch.cuda.set_device(0)
    nqs.use_torch_allocator()
    torch.cuda.empty_cache()
    w = W.random_circuit(131, 31, 240, 20, noise_kinds=("depol",), v_kind="ideal", rate_lo=1e-3, rate_hi=1e-2)
    text = W.to_ir_text(w)
    circ = nqs.NoisyCircuit(text)
    res = circ.fidelity(nqs.basis(w.psi["bits"]), nqs.ideal(), 1)
    info = nqs.nqs_get_info(circ.h)
    recs = nqs.nqs_enumerate_terms(circ.h, 1)
    vals = circ.term_values()
    circ.close()
    torch.cuda.empty_cache()
    assert res["status"] == 0
    assert info["ckpt_spacing"] > 0 and info["n_states"] < 21
    got = site_sets(recs, vals)
    F = res["F"]
    assert abs(F - res["T"][0] - res["T"][1]) <= 1e-12 * F

    c = OIR.parse(text)
    fac = OEX.prepared_factors(c)
    cu = [_identity_scale(f[1][0]) for f in fac]
    cv = [_identity_scale(f[2][0]) for f in fac]
    T0 = np.prod([(a * b).real for a, b in zip(cu, cv)])
    assert abs(res["T"][0] - T0) <= REL_TOL * F, (res["T"][0], T0)
    ev = {idx: e for e, (kind, idx) in enumerate(OIR.events(c)) if kind == "noise"}
    n = c.n
    chi = np.zeros(1 << n, dtype=np.complex128)
    chi[w.psi["bits"]] = 1.0
    pos = 0
    for s in range(2):
        csim.apply_ops(n, chi, _gate_ops(c, pos, ev[s]))
        pos = ev[s]
        q = c.noises[s][1]
        W1 = 0.0
        for i in (1, 2, 3):
            x = chi.copy()
            csim.apply_ops(n, x, _one(q, fac[s][1][i]))
            a = csim.inner(n, chi, x)
            x[:] = chi
            csim.apply_ops(n, x, _one(q, fac[s][2][i].conj()))
            b = csim.inner(n, chi, x).conjugate()
            del x
            W1 += (a * b).real
        W1 *= np.prod([(cu[u] * cv[u]).real for u in range(len(fac)) if u != s])
        assert abs(got[(s,)] - W1) <= REL_TOL * F, (s, got[(s,)], W1)
        assert abs(got[(s,)] - W1) <= 1e-2 * W1 + 1e-12, (s, got[(s,)], W1)
