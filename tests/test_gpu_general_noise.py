"""General noises on the GPU (nqs_load_circuit with noise2 / superop /
superop2 records): two-qubit channels and noises given by a matrix
representation that is not completely positive (two factor sets, each term
the product of two different network amplitudes, Algorithm 1's general
form).  Against the FP64 oracle O2 term by term (canonical order), O3 at a
larger width, the two-qubit depolarizing closed form and the density
matrix; tolerance 1e-5 relative on F, 1e-5 * |F| on T_u, site-set sums and
terms."""

import itertools
import math

import numpy as np
import pytest

import workloads as W
from workloads import channels as ch
from workloads.circuits import Noise
from oracle import density_matrix as DM
from oracle import expansion as OEX
from oracle import ir as OIR
from oracle import o3 as O3

pytestmark = pytest.mark.gpu

REL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _setup():
    import torch
    from paper_2211_17028_gb300 import nqs
    torch.cuda.set_device(0)
    nqs.use_torch_allocator()
    yield


def _mixed(seed, n, gates):
    rng = W.SplitMix64(seed)
    w = W.random_circuit(seed, n, gates, 0, v_kind="ideal")
    g = len(w.gates)
    w.noises = [Noise(g // 6, 1, ch.near_identity_channel2(rng, 0.03, 2), "", 0),
                Noise(g // 3, 0, [], "", -1, ch.perturbed_superop(rng, ch.amplitude_damping(0.05), 0.01)),
                Noise(g // 2, n - 1, ch.depolarizing_paper(0.02), ""),
                Noise(2 * g // 3, n - 2, [], "", n - 3, ch.perturbed_superop(rng, ch.depolarizing2(0.04), 0.005)),
                Noise(5 * g // 6, 0, ch.depolarizing2(0.05), "", n - 1)]
    return w


def _gpu(w, level):
    from paper_2211_17028_gb300 import nqs
    circ = nqs.NoisyCircuit(W.to_ir_text(w))
    psi = nqs.basis(w.psi["bits"])
    v = nqs.ideal() if w.v["kind"] == "ideal" else nqs.basis(w.v["bits"])
    res = circ.fidelity(psi, v, level)
    vals = circ.term_values()
    circ.close()
    return res, vals


def _distinct(d):
    """The nonzero non-dominant singular values are pairwise distinct, so each
    factor (and each term) is independent of a basis choice."""
    nz = [x for x in d[1:] if x > 1e-12 * d[0]]
    return all(abs(a - b) > 1e-9 * d[0] for a, b in itertools.combinations(nz, 2))


def _site_sets(c, level, vals):
    fac = OEX.prepared_factors(c)
    m = [len(f[1]) for f in fac]
    out = {}
    for (k, sites, idx), x in zip(OEX.kept_assignments(len(c.noises), level, m), vals):
        out[sites] = out.get(sites, 0.0) + x
    return out


@pytest.mark.parametrize("seed,n,level", [(101, 4, 1), (102, 5, 2), (103, 6, 3), (104, 8, 2)])
def test_general_noise_matches_o2_term_by_term(seed, n, level):
    w = _mixed(seed, n, 30)
    c = OIR.parse(W.to_ir_text(w))
    ref = OEX.approximate(c, w.psi, w.v, level, keep_terms=True)
    res, vals = _gpu(w, level)
    F = ref["F"].real
    assert res["status"] == 0 and res["n_terms"] == ref["n_terms"] == len(vals)
    assert abs(res["F"] - F) <= REL * abs(F), (res["F"], F)
    for u, t in enumerate(ref["T"]):
        assert abs(res["T"][u] - t.real) <= REL * abs(F), (u, res["T"][u], t)
    want = np.array([x.real for _, x in ref["terms"]])
    # sets carrying a degenerate channel (two-qubit depolarizing) compare as sums
    got_s, want_s = _site_sets(c, level, vals), _site_sets(c, level, want)
    assert max(abs(got_s[k] - want_s[k]) for k in want_s) <= REL * abs(F)
    nondeg = [s for s, (_, q, spec) in enumerate(c.noises) if _distinct(OEX.svd_factors(spec)[0])]
    keys = list(OEX.kept_assignments(len(c.noises), level, [len(f[1]) for f in OEX.prepared_factors(c)]))
    sel = [i for i, (k, sites, idx) in enumerate(keys) if all(s in nondeg for s in sites)]
    assert np.max(np.abs(vals[sel] - want[sel])) <= REL * abs(F)
    # the imaginary parts cancel only in the full sum; the residual is reported
    assert res["imag_residual"] >= 0.0


def test_two_qubit_depolarizing_closed_form_on_gpu():
    p, N = 0.1, 3
    w = W.Workload("dep2", 3, [("h", (2,), ())], [Noise(0, 0, ch.depolarizing2(p), "", 1) for _ in range(N)],
                   {"kind": "basis", "bits": 0}, {"kind": "basis", "bits": 4}, (N,))
    res, vals = _gpu(w, N)
    # qubit 2 in |+>, v = |100>: the (0, 1) pair as on the identity circuit, times |<1|+>|^2 = 1/2
    for u in range(N + 1):
        want = 0.5 * math.comb(N, u) * (1 - p) ** (N - u) * (p / 15) ** u * (15 ** u + 3 * (-1) ** u) / 4
        assert abs(res["T"][u] - want) <= REL * 0.5, (u, res["T"][u], want)
    assert abs(res["F"] - 0.5 * (0.25 + 0.75 * (1 - 16 * p / 15) ** N)) <= REL


def test_general_noise_full_level_is_the_density_matrix():
    w = _mixed(105, 4, 20)
    c = OIR.parse(W.to_ir_text(w))
    res, _ = _gpu(w, 5)
    f = DM.fidelity(c, w.psi, w.v)
    assert abs(res["F"] - f.real) <= REL * abs(f)


def test_general_noise_wider_circuit_against_o3():
    w = _mixed(106, 14, 80)
    c = OIR.parse(W.to_ir_text(w))
    ref = O3.approximate(c, w.psi, w.v, 2)
    res, vals = _gpu(w, 2)
    F = ref["F"].real
    assert abs(res["F"] - F) <= REL * abs(F)
    got_s, want_s = _site_sets(c, 2, vals), _site_sets(c, 2, ref["terms"].real)
    assert max(abs(got_s[k] - want_s[k]) for k in want_s) <= REL * abs(F)


def test_general_noise_entry_points():
    from paper_2211_17028_gb300 import nqs
    w = _mixed(107, 5, 24)
    c = OIR.parse(W.to_ir_text(w))
    circ = nqs.NoisyCircuit(W.to_ir_text(w))
    psi = nqs.basis(w.psi["bits"])
    # adaptive level selection and off-diagonal elements work on the general path
    r = nqs.nqs_fidelity_adaptive(circ.h, psi, nqs.ideal(), 1e-3, criteria=nqs.NQS_ADAPT_OBSERVED)
    assert r["status"] == 0 and r["level"] >= 1
    x = {"kind": "basis", "bits": 3}
    y = {"kind": "basis", "bits": 12}
    got, _ = nqs.nqs_offdiagonal(circ.h, psi, nqs.basis(3), nqs.basis(12), 5)
    want = DM.matrix_element(c, w.psi, x, y)
    assert abs(got - want) <= 1e-5
    for fn in (lambda: nqs.nqs_batch_fidelity([circ.h], [psi], [nqs.ideal()], [1]),
               lambda: nqs.nqs_enumerate_terms(circ.h, 1)):
        with pytest.raises(nqs.NqsError) as e:
            fn()
        assert e.value.code == nqs.NQS_ERR_UNSUPPORTED
    circ.close()
