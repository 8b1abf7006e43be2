"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs.  Tolerance: 1e-5 relative on every fidelity, 1e-5 * F
absolute on T_u, per-site-set sums and (non-degenerate channels) individual
terms; the kept-term list is compared bit for bit on the host side."""

import math

import numpy as np
import pytest

import workloads as W
from workloads import channels as ch

from _gpu_util import compare, gpu_result, oracle_result

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


@pytest.mark.parametrize("level", [0, 1, 2, 4])
def test_line6_depolarizing(level):
    w = W.c1_line6()
    res, terms = gpu_result(w, level)
    compare(w, level, res, terms, oracle_result(w, level))


CASES = [
    # seed, n, gates, noises, v kind, levels
    (11, 1, 6, 3, "basis", (0, 1, 3)),
    (12, 2, 12, 4, "ideal", (1, 2, 4)),
    (13, 3, 25, 5, "basis", (1, 2, 3)),
    (14, 5, 40, 6, "dense", (1, 2, 3)),
    (15, 7, 60, 5, "ideal", (0, 1, 2)),
    (16, 9, 70, 4, "basis", (1, 2, 4)),
    (17, 11, 80, 5, "ideal", (1, 2)),
]


@pytest.mark.parametrize("case", CASES, ids=[f"n{c[1]}_s{c[0]}" for c in CASES])
def test_random_circuits(case):
    seed, n, gates, noise, vkind, levels = case
    w = W.random_circuit(seed, n, gates, noise, v_kind=vkind)
    for level in levels:
        res, terms = gpu_result(w, level)
        compare(w, level, res, terms, oracle_result(w, level))


def test_dense_psi_and_v():
    w = W.random_circuit(21, 6, 40, 4, v_kind="dense")
    w.psi = {"kind": "dense", "amps": W.circuits.random_dense_state(W.SplitMix64(77), 6)}
    for level in (1, 2):
        res, terms = gpu_result(w, level)
        compare(w, level, res, terms, oracle_result(w, level))


@pytest.mark.parametrize("n,seed", [(13, 31), (14, 32), (16, 33)])
def test_several_tiles_and_partial_passes(n, seed):
    # widths above the 12-qubit tile: several tiles per pass, tile sets that
    # change between passes, branches that start inside a pass
    w = W.random_circuit(seed, n, 90, 5, v_kind="ideal", rate_lo=1e-3, rate_hi=2e-2)
    for level in (1, 2):
        res, terms = gpu_result(w, level)
        compare(w, level, res, terms, oracle_result(w, level))


def test_level3_multi_tile():
    w = W.random_circuit(41, 14, 60, 4, noise_kinds=("ad", "adpd", "random"), v_kind="ideal")
    res, terms = gpu_result(w, 3)
    compare(w, 3, res, terms, oracle_result(w, 3))


def test_grid20_level1_full_and_level2_sampled():
    from oracle import csim
    from oracle import expansion as OEX
    from oracle import ir as OIR
    from oracle.density_matrix import state_from_spec
    w = W.c2_grid20()
    res1, terms1 = gpu_result(w, 1)
    compare(w, 1, res1, terms1, oracle_result(w, 1))
    # level 2: every term on the GPU; a seeded sample of terms by the oracle
    res2, terms2 = gpu_result(w, 2)
    assert res2["n_terms"] == 1771
    c = OIR.parse(W.to_ir_text(w))
    psi = state_from_spec(w.psi, w.n)
    v = state_from_spec(w.v, w.n, c, psi)
    fac = OEX.prepared_factors(c)
    recs = list(OEX.kept_assignments(20, 2))
    rng = W.SplitMix64(2024)
    pick = sorted(set([61, 62, 1770] + [61 + rng.randbelow(1710) for _ in range(12)]))
    scale = abs(res1["F"])
    for idx in pick:
        k, sites, fidx = recs[idx]
        x = csim.term_value(c, psi, v, fac, sites, fidx).real
        assert abs(terms2[idx] - x) <= 1e-5 * scale, (idx, terms2[idx], x)
    # the level-2 schedule cuts passes differently, so T_1 agrees to rounding
    assert abs(res2["T"][1] - res1["T"][1]) <= 1e-5 * scale
    assert res2["F"] >= res1["F"] - 1e-12 * scale


def test_amplitude_damping_closed_form_many_sites():
    # identity-like circuit (X X) with 30 AD noises on one qubit: psi = |1>,
    # v = |0>: T_1 = 1 - (1-g)^30, every other level 0
    g = 0.02
    w = W.identity_workload(3, [(1, ch.amplitude_damping(g))] * 30, psi_bits=2, v_bits=0)
    res, terms = gpu_result(w, 2)
    assert abs(res["T"][0]) < 1e-9
    assert abs(res["T"][1] - (1 - (1 - g) ** 30)) <= 1e-5 * res["F"]
    assert abs(res["T"][2]) < 1e-9


def test_depolarizing_closed_form_identity():
    p, N = 0.01, 12
    w = W.identity_workload(2, [(0, ch.depolarizing_paper(p))] * N)
    res, _ = gpu_result(w, 3)
    for u in range(4):
        want = math.comb(N, u) * (1 - p) ** (N - u) * (p / 3) ** u * (3 ** u + (-1) ** u) / 2
        assert abs(res["T"][u] - want) <= 1e-6 * want + 1e-12


def test_results_are_bit_reproducible():
    w = W.random_circuit(51, 15, 80, 6, v_kind="ideal")
    a, ta = gpu_result(w, 2)
    b, tb = gpu_result(w, 2)
    assert a["F"] == b["F"] and a["T"] == b["T"]
    assert np.array_equal(ta, tb)


def test_noiseless_limit():
    w = W.random_circuit(61, 12, 80, 0, v_kind="ideal")
    w.noises = [W.Noise(5, w.gates[5][1][0], [np.eye(2, dtype=np.complex128)]),
                W.Noise(40, w.gates[40][1][0], ch.depolarizing_paper(0.0))]
    res, terms = gpu_result(w, 2)
    assert abs(res["F"] - 1.0) <= 1e-5
    assert all(abs(t) < 1e-10 for t in terms[1:])


def test_reduced_matrix_entry_point():
    import torch
    from paper_2211_17028_gb300 import nqs
    rng = W.SplitMix64(99)
    for n, q in ((1, 0), (5, 3), (13, 0), (17, 16), (20, 7)):
        a = W.circuits.random_dense_state(rng, n) if n <= 13 else None
        if a is None:
            g = torch.Generator().manual_seed(n)
            a = (torch.randn(1 << n, generator=g, dtype=torch.float64) +
                 1j * torch.randn(1 << n, generator=g, dtype=torch.float64)).numpy()
        b = np.roll(a, 3) * (0.5 + 0.1j)
        phi = torch.tensor(a.astype(np.complex64), device="cuda")
        chi = torch.tensor(b.astype(np.complex64), device="cuda")
        nb = nqs.nqs_reduced_matrix_scratch_bytes(n)
        scratch = torch.empty(nb, dtype=torch.uint8, device="cuda")
        out = torch.zeros(8, dtype=torch.float64, device="cuda")
        nqs.nqs_reduced_matrix(phi, chi, n, q, out, scratch, nb)
        got = out.cpu().numpy().view(np.complex128).reshape(2, 2)
        a64 = a.astype(np.complex64).astype(np.complex128).reshape((2,) * n)
        b64 = b.astype(np.complex64).astype(np.complex128).reshape((2,) * n)
        ax = n - 1 - q
        want = np.tensordot(a64.conj(), b64, axes=([i for i in range(n) if i != ax],) * 2)
        assert np.allclose(got, want, rtol=1e-5, atol=1e-5 * np.abs(want).max())
