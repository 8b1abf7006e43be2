"""Host side of the C ABI (no GPU): library exports, circuit reader, noise
factors, canonical enumeration, bounds -- compared with the oracle."""

import ctypes
import os
import re

import numpy as np
import pytest

import workloads as W
from workloads import channels as ch
from oracle import bounds as OB
from oracle import expansion as OEX
from oracle import ir as OIR
from paper_2211_17028_gb300 import nqs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "nqs.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(nqs_[a-z0-9_]+)\s*\(", text)) - {"nqs_alloc_fn", "nqs_free_fn"})


def test_library_exports_every_declared_symbol():
    lib = nqs.library()
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    assert "sm_103a" in nqs.nqs_version()


def test_binding_covers_every_declared_function():
    for name in declared_functions():
        assert hasattr(nqs, name), name


def _handle(w, flags=0):
    h = nqs.nqs_load_circuit(W.to_ir_text(w))
    nqs.nqs_prepare_noise(h, None, flags)
    return h


def test_parse_errors_and_call_order():
    with pytest.raises(nqs.NqsError) as e:
        nqs.nqs_load_circuit("qubits 2\ngate h 0\n")
    assert e.value.code == nqs.NQS_ERR_PARSE
    for bad in ["nqs-ir 1\nqubits 2\ngate h 2\n", "nqs-ir 1\nqubits 2\ngate cz 0 0\n",
                "nqs-ir 1\nqubits 2\ngate rx 0\n", "nqs-ir 1\nqubits 2\ngate foo 0\n",
                "nqs-ir 1\nqubits 2\ngate h 0\nnoise 3 0 1 1 0 0 0 0 0 1 0\n",
                "nqs-ir 1\nqubits 2\ngate h 0\ngate h 1\nnoise 1 0 1 1 0 0 0 0 0 1 0\nnoise 0 0 1 1 0 0 0 0 0 1 0\n"]:
        with pytest.raises(nqs.NqsError) as e:
            nqs.nqs_load_circuit(bad)
        assert e.value.code == nqs.NQS_ERR_PARSE, bad
    with pytest.raises(nqs.NqsError) as e:
        nqs.nqs_load_circuit("nqs-ir 1\nqubits 40\n")
    assert e.value.code == nqs.NQS_ERR_UNSUPPORTED
    h = nqs.nqs_load_circuit("nqs-ir 1\nqubits 2\ngate h 0\n")
    with pytest.raises(nqs.NqsError) as e:
        nqs.nqs_enumerate_terms(h, 1)
    assert e.value.code == nqs.NQS_ERR_ORDER
    nqs.nqs_destroy(h)


def test_noise_validation_errors():
    h = nqs.nqs_load_circuit("nqs-ir 1\nqubits 2\ngate h 0\ngate cx 0 1\n")
    bad = [np.eye(2) * 0.9]
    with pytest.raises(nqs.NqsError) as e:
        nqs.nqs_prepare_noise(h, [(0, 0, bad)])
    assert e.value.code == nqs.NQS_ERR_NOT_CPTP
    with pytest.raises(nqs.NqsError) as e:
        nqs.nqs_prepare_noise(h, [(0, 1, ch.depolarizing_paper(0.75))])
    assert e.value.code == nqs.NQS_ERR_NOT_DOMINANT
    with pytest.raises(nqs.NqsError) as e:
        nqs.nqs_prepare_noise(h, [(0, 2, ch.depolarizing_paper(0.1))])
    assert e.value.code == nqs.NQS_ERR_ARG
    with pytest.raises(nqs.NqsError) as e:
        nqs.nqs_prepare_noise(h, [(1, 0, ch.depolarizing_paper(0.1)), (0, 0, ch.depolarizing_paper(0.1))])
    assert e.value.code == nqs.NQS_ERR_ARG
    nqs.nqs_prepare_noise(h, [(-1, 0, ch.amplitude_damping(0.1)), (1, 1, ch.phase_damping(0.2))])
    assert nqs.nqs_get_info(h)["n_sites"] == 2
    nqs.nqs_destroy(h)


@pytest.mark.parametrize("seed,n,gates,noise", [(1, 3, 20, 4), (2, 5, 30, 6), (3, 4, 10, 9), (4, 6, 40, 0)])
def test_enumeration_is_bit_identical_to_oracle(seed, n, gates, noise):
    w = W.random_circuit(seed, n, gates, noise)
    h = _handle(w)
    N = w.n_noise
    for level in range(0, 5):
        assert nqs.nqs_enumerate_terms(h, level) == OEX.enumerate_records(N, level)
    nqs.nqs_destroy(h)


def test_enumeration_of_configurations():
    for w, levels in ((W.c1_line6(), (1, 4)), (W.c2_grid20(), (1, 2)), (W.c3_qaoa30(), (2,))):
        h = _handle(w)
        for level in levels:
            recs = nqs.nqs_enumerate_terms(h, level)
            assert recs == OEX.enumerate_records(w.n_noise, level)
            assert len(recs) == OEX.term_count(w.n_noise, level)
        nqs.nqs_destroy(h)


CHANNELS = [ch.depolarizing_paper(0.01), ch.amplitude_damping(0.03), ch.phase_damping(0.02),
            ch.ad_pd(1e-3, 1e-3), ch.near_identity_channel(W.SplitMix64(5), 0.02, 3),
            ch.near_identity_channel(W.SplitMix64(6), 0.05, 1), [np.eye(2, dtype=np.complex128)]]


@pytest.mark.parametrize("idx", range(len(CHANNELS)))
def test_noise_factors_match_oracle_svd(idx):
    kraus = CHANNELS[idx]
    h = nqs.nqs_load_circuit("nqs-ir 1\nqubits 1\ngate h 0\n")
    nqs.nqs_prepare_noise(h, [(0, 0, kraus)])
    d, K = nqs.nqs_noise_factors(h, 0)
    do, u, v, _, _ = OEX.svd_factors(kraus)
    assert np.allclose(d, do, atol=1e-14)
    # the factors rebuild the channel: sum_i K_i (x) conj(K_i) = M
    m = OEX.matrix_representation(kraus)
    assert np.allclose(sum(np.kron(K[i], K[i].conj()) for i in range(4)), m, atol=1e-14)
    # per eigenspace the products agree with the oracle's U_i (x) V_i (phase free)
    groups = []
    for i in range(4):
        if groups and abs(d[i] - d[groups[-1][0]]) <= 1e-12 * max(d[0], 1e-300):
            groups[-1].append(i)
        else:
            groups.append([i])
    for g in groups:
        mine = sum(np.kron(K[i], K[i].conj()) for i in g)
        theirs = sum(np.kron(u[i], v[i]) for i in g)
        assert np.allclose(mine, theirs, atol=1e-13)
    nqs.nqs_destroy(h)


def test_truncation_bound_matches_oracle():
    w = W.random_circuit(8, 4, 25, 7, rate_lo=1e-3, rate_hi=3e-2)
    h = _handle(w)
    c = OIR.parse(W.to_ir_text(w))
    kl = [z[2] for z in c.noises]
    for level in range(0, 8):
        assert nqs.nqs_truncation_bound(h, level) == pytest.approx(OB.per_site_bound(kl, level), rel=1e-12,
                                                                   abs=1e-300)
    nqs.nqs_destroy(h)


def test_plan_shapes():
    h = _handle(W.c3_qaoa30())
    info = nqs.nqs_get_info(h)
    assert info["n_qubits"] == 30 and info["n_sites"] == 20 and info["tile_qubits"] == 12
    # CNOT-RZ-CNOT collapses into one diagonal phase: far fewer fused ops than gates
    # (a noise inside a block leaves its two CNOTs, each at most H, diagonal, H)
    assert info["n_ops"] <= 30 + 4 * (45 + 30) + 20 + 4 * 20
    assert info["n_passes"] >= 3
    nqs.nqs_destroy(h)
    h = _handle(W.c1_line6())
    info = nqs.nqs_get_info(h)
    assert info["n_passes"] <= 2 and info["tile_qubits"] == 6
    nqs.nqs_destroy(h)


@pytest.mark.parametrize("make", [
    lambda: W.c1_line6(),
    lambda: W.qaoa_workload(8, 3, 6, 3, "ideal", "qaoa8"),
    lambda: W.qaoa_workload(10, 5, 8, 2, "ideal", "qaoa10"),
    lambda: W.random_circuit(51, 7, 60, 6, noise_kinds=("ad", "pd", "adpd", "depol"), v_kind="ideal"),
    lambda: W.random_circuit(52, 9, 90, 8, v_kind="ideal"),
], ids=["line6", "qaoa8", "qaoa10", "random7", "random9"])
def test_plan_operator_equals_circuit_operator(make):
    # fusion, the Hadamard-diagonal rewrite and the reordering before
    # segmentation keep the product of the operations (K_0 at the sites)
    h = _handle(make())
    assert nqs.nqs_plan_check(h) <= 1e-12
    nqs.nqs_destroy(h)


@pytest.mark.parametrize("seed", range(60, 72))
def test_plan_operator_random_circuits(seed):
    # random widths, depths and noise placements, every gate kind of the reader
    rng = np.random.default_rng(seed)
    n = int(rng.integers(3, 9))
    w = W.random_circuit(seed, n, int(rng.integers(10, 80)), int(rng.integers(1, 12)), v_kind="ideal")
    h = _handle(w)
    assert nqs.nqs_plan_check(h) <= 1e-12
    nqs.nqs_destroy(h)


def test_plan_reordering_cuts_passes():
    # the 30-qubit QAOA workload: 20 passes per sweep in circuit order, 12 after
    # hoisting commuting operations into passes whose tiles are chosen for them
    h = _handle(W.c3_qaoa30())
    assert nqs.nqs_get_info(h)["n_passes"] <= 12
    assert nqs.nqs_plan_check(h) == 0.0      # n > 10: the pass structure only
    # looser segmentation bounds keep the reordering's passes, tighter ones cut in order
    nqs.nqs_set_option(h, nqs.NQS_OPT_MAX_OPS, 128)
    nqs.nqs_set_option(h, nqs.NQS_OPT_MAX_SITES, 8)
    assert nqs.nqs_get_info(h)["n_passes"] <= 12
    nqs.nqs_set_option(h, nqs.NQS_OPT_MAX_OPS, 64)
    nqs.nqs_set_option(h, nqs.NQS_OPT_MAX_SITES, 2)
    assert nqs.nqs_get_info(h)["n_passes"] > 12 and nqs.nqs_plan_check(h) == 0.0
    nqs.nqs_destroy(h)


@pytest.mark.parametrize("make", [lambda: W.c2_grid20(), lambda: W.c5_twin_hot(), lambda: W.c5_grid(),
                                  lambda: W.qaoa_workload(24, 3, 20, 4, "ideal", "qaoa24")],
                         ids=["grid20", "twin20", "c5_28", "qaoa24"])
def test_plan_structure_of_wide_circuits(make):
    # every pass continues the previous one, holds its operations' dense and
    # site qubits in a 12-qubit tile with the low qubits, and keeps the bounds
    h = _handle(make())
    assert nqs.nqs_plan_check(h) == 0.0
    for ops, sites in ((64, 2), (160, 8)):
        nqs.nqs_set_option(h, nqs.NQS_OPT_MAX_OPS, ops)
        nqs.nqs_set_option(h, nqs.NQS_OPT_MAX_SITES, sites)
        assert nqs.nqs_plan_check(h) == 0.0
    nqs.nqs_destroy(h)


def test_prune_flag_drops_zero_rank_factors():
    # amplitude damping has Kraus rank 2: with pruning only factor 1 remains
    h = nqs.nqs_load_circuit("nqs-ir 1\nqubits 2\ngate h 0\ngate cx 0 1\n")
    sites = [(0, 0, ch.amplitude_damping(0.05)), (1, 1, ch.amplitude_damping(0.02)),
             (1, 0, ch.depolarizing_paper(0.01))]
    nqs.nqs_prepare_noise(h, sites, nqs.NQS_PREP_PRUNE_ZERO_RANK)
    recs = nqs.nqs_enumerate_terms(h, 2)
    # per site kept factors: 1, 1, 3 -> level<=2 count = 1 + (1+1+3) + (1*1 + 1*3 + 1*3)
    assert len(recs) == 1 + 5 + 7
    for r in recs:
        k = r & 15
        for j in range(k):
            f = (r >> (4 + 14 * j)) & 0x3FFF
            site, fac = f & 0xFFF, f >> 12
            if site < 2:
                assert fac == 1
    nqs.nqs_destroy(h)


# ----------------------------------------------------------------------------
# general noises (two-qubit channels, superoperators): host factors

def _general_workload(seed):
    from workloads.circuits import Noise
    rng = W.SplitMix64(seed)
    w = W.random_circuit(seed, 4, 20, 0, v_kind="ideal")
    w.noises = [Noise(2, 1, ch.near_identity_channel2(rng, 0.03, 2), "", 3),
                Noise(5, 0, [], "", -1, ch.perturbed_superop(rng, ch.amplitude_damping(0.05), 0.01)),
                Noise(9, 2, ch.depolarizing_paper(0.02), ""),
                Noise(12, 3, [], "", 0, ch.perturbed_superop(rng, ch.depolarizing2(0.04), 0.005)),
                Noise(15, 0, ch.depolarizing2(0.05), "", 2)]
    return w


def test_general_factors_rebuild_the_noise_matrix():
    import numpy as np
    from oracle import expansion as OEX
    from oracle import ir as OIR
    w = _general_workload(7)
    c = OIR.parse(W.to_ir_text(w))
    h = nqs.nqs_load_circuit(W.to_ir_text(w))
    nqs.nqs_prepare_noise(h)
    for s, (_, q, spec) in enumerate(c.noises):
        sv, ka, kb, same = nqs.nqs_general_factors(h, s)
        m = OEX.matrix_representation(spec)
        d_ref = OEX.svd_factors(spec)[0]
        assert np.allclose(sv, d_ref, rtol=1e-10, atol=1e-13)
        # sum_i KA_i (x) conj(KB_i) = M (the factors carry the whole noise)
        rebuilt = sum(np.kron(a, b.conj()) for a, b in zip(ka, kb))
        assert np.allclose(rebuilt, m, atol=1e-12)
        assert same == (not isinstance(spec, OIR.SuperOp))
    with pytest.raises(nqs.NqsError) as e:
        nqs.nqs_noise_factors(h, 0)
    assert e.value.code == nqs.NQS_ERR_UNSUPPORTED
    nqs.nqs_destroy(h)


JIT_CIRCUITS = [
    ("qaoa16", lambda: W.qaoa_workload(16, 3, 12, 3, "ideal", "qaoa16")),
    ("random14", lambda: W.random_circuit(42, 14, 80, 5, v_kind="dense")),
    ("grid15_ad_pd", lambda: W.random_circuit(43, 15, 120, 8, noise_kinds=("ad", "pd", "adpd"), v_kind="ideal")),
]


def _compile_check(make, states, passes=6):
    h = _handle(make())
    try:
        return nqs.nqs_jit_compile_check(h, states, passes)
    except nqs.NqsError as e:
        if e.code == nqs.NQS_ERR_UNSUPPORTED:
            pytest.skip("NVRTC not available")
        raise
    finally:
        nqs.nqs_destroy(h)


@pytest.mark.parametrize("states", [1, 3])
@pytest.mark.parametrize("name,make", JIT_CIRCUITS, ids=[c[0] for c in JIT_CIRCUITS])
def test_generated_kernels_compile(name, make, states):
    # generator output of real passes (dense and diagonal gates on register,
    # lane and tile-base qubits, reductions, spawns) compiles for sm_103a
    assert _compile_check(make, states) >= 1


@pytest.mark.parametrize("env", [{"NQS_JIT_SEQ": "0"}, {"NQS_JIT_RV": "1"}, {"NQS_JIT_HINT": "0"},
                                 {"NQS_JIT_PP": "0"}, {"NQS_JIT_DB": "2"}, {"NQS_JIT_EARLY_PHI": "2"},
                                 {"NQS_JIT_WIDE": "1"}],
                         ids=["seq0", "rv1", "hint0", "pp0", "db2", "early2", "wide"])
def test_generated_kernel_variants_compile(env, monkeypatch):
    # the non-default forms of the generator (kept for comparison runs) still compile
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    assert _compile_check(JIT_CIRCUITS[0][1], 3, 4) >= 1
    assert _compile_check(JIT_CIRCUITS[0][1], 1, 4) >= 1


def test_compile_check_needs_a_prepared_wide_circuit():
    h = nqs.nqs_load_circuit(W.to_ir_text(W.c1_line6()))
    with pytest.raises(nqs.NqsError) as e:
        nqs.nqs_jit_compile_check(h, 1, 1)
    assert e.value.code == nqs.NQS_ERR_ORDER
    nqs.nqs_prepare_noise(h, None, 0)
    with pytest.raises(nqs.NqsError) as e:
        nqs.nqs_jit_compile_check(h, 1, 1)   # 6 qubits: no generated kernels
    assert e.value.code == nqs.NQS_ERR_UNSUPPORTED
    nqs.nqs_destroy(h)
