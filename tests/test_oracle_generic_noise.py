"""Pins of the oracle for two-qubit noise channels and for noises given as a
superoperator whose tensor-permuted matrix is not positive semidefinite
(two different factor sets, so each term is a product of two distinct
network amplitudes -- Algorithm 1's general case)."""

import math

import numpy as np
import pytest

import workloads as W
from workloads import channels as ch
from workloads.circuits import Noise
from oracle import density_matrix as DM
from oracle import expansion as EX
from oracle import ir as IR
from oracle import o3 as O3


def _circ(w):
    return IR.parse(W.to_ir_text(w))


def _ident2(noises, n=2):
    """Identity circuit carrying the given noises (after_gate -1)."""
    return W.Workload("ident", n, [], noises, {"kind": "basis", "bits": 0}, {"kind": "basis", "bits": 0}, (1,))


@pytest.mark.parametrize("p,N", [(0.02, 1), (0.1, 2), (0.3, 3)])
def test_two_qubit_depolarizing_closed_form(p, N):
    # identity circuit, psi = v = |00>, N two-qubit depolarizing noises on (0, 1):
    # a kept term is (p/15)^u (1-p)^(N-u) |<00| P_1 ... P_u |00>|^2 for
    # non-identity Paulis P; the product is diagonal for (15^u + 3 (-1)^u) / 4
    # of the 15^u choices (characters of Z_2^4 over the subgroup {II, IZ, ZI, ZZ}),
    # so T_u = C(N,u) (1-p)^(N-u) (p/15)^u (15^u + 3 (-1)^u) / 4 and
    # F = 1/4 + 3/4 (1 - 16p/15)^N
    w = _ident2([Noise(-1, 0, ch.depolarizing2(p), "", 1) for _ in range(N)])
    c = _circ(w)
    f = DM.fidelity(c, w.psi, w.v).real
    assert math.isclose(f, 0.25 + 0.75 * (1 - 16 * p / 15) ** N, rel_tol=1e-13)
    for r in (EX.approximate(c, w.psi, w.v, N), O3.approximate(c, w.psi, w.v, N)):
        for u in range(N + 1):
            want = math.comb(N, u) * (1 - p) ** (N - u) * (p / 15) ** u * (15 ** u + 3 * (-1) ** u) / 4
            assert math.isclose(r["T"][u].real, want, rel_tol=1e-11, abs_tol=1e-300), (u, r["T"][u], want)
        assert math.isclose(r["F"].real, f, rel_tol=1e-13)
    assert EX.term_count(N, N, [16] * N) == 16 ** N


def test_two_qubit_factors_rebuild_the_channel():
    rng = W.SplitMix64(5)
    k = ch.near_identity_channel2(rng, 0.05, 3)
    d, u, v, _, _ = EX.svd_factors(k)
    assert len(u) == 16 and d[0] > d[1]
    m = EX.matrix_representation(k)
    assert np.allclose(sum(np.kron(a, b) for a, b in zip(u, v)), m, atol=1e-14)
    # CPTP: the tensor-permuted matrix is PSD, U_i proportional to conj(V_i) where d_i > 0
    for i in range(16):
        if d[i] > 1e-12:
            assert np.allclose(u[i], d[i] * v[i].conj(), atol=1e-12)


def test_superop_of_a_channel_equals_its_kraus_form():
    w = W.random_circuit(33, 4, 30, 4, rate_lo=1e-2, rate_hi=5e-2, v_kind="ideal")
    w2 = W.random_circuit(33, 4, 30, 4, rate_lo=1e-2, rate_hi=5e-2, v_kind="ideal")
    for z in w2.noises:
        z.superop = ch.matrix_of(z.kraus)
    c, c2 = _circ(w), _circ(w2)
    assert isinstance(c2.noises[0][2], IR.SuperOp)
    for lvl in (1, 2, 4):
        a = EX.approximate(c, w.psi, w.v, lvl)
        b = EX.approximate(c2, w2.psi, w2.v, lvl)
        assert abs(a["F"] - b["F"]) < 1e-13


def test_superop_closed_form_and_full_level():
    rng = W.SplitMix64(9)
    m = ch.perturbed_superop(rng, ch.depolarizing_paper(0.05), 0.02)
    # not positive semidefinite after the tensor permutation: two factor sets
    t = EX.tensor_permutation(m)
    assert np.min(np.linalg.eigvalsh((t + t.conj().T) / 2)) < -1e-4 or not np.allclose(t, t.conj().T)
    z = Noise(-1, 0, [], "", -1, m)
    w = W.Workload("sop", 1, [], [z], {"kind": "basis", "bits": 0}, {"kind": "basis", "bits": 0}, (1,))
    c = _circ(w)
    # identity circuit, psi = v = |0>: F = <0| M(|0><0|) |0> = M[(0,0), (0,0)]
    r = EX.approximate(c, w.psi, w.v, 1)
    assert abs(r["F"] - m[0, 0]) < 1e-14
    assert abs(DM.fidelity(c, w.psi, w.v) - m[0, 0]) < 1e-14


@pytest.mark.parametrize("seed", [41, 42])
def test_mixed_generic_noise_full_level_equals_density_matrix(seed):
    rng = W.SplitMix64(seed)
    w = W.random_circuit(seed, 4, 24, 0, v_kind="dense")
    gates = len(w.gates)
    w.noises = [Noise(3, 1, ch.near_identity_channel2(rng, 0.03, 2), "", 2),
                Noise(9, 0, [], "", -1, ch.perturbed_superop(rng, ch.amplitude_damping(0.05), 0.01)),
                Noise(15, 3, ch.depolarizing_paper(0.02), ""),
                Noise(min(20, gates - 1), 2, [], "", 0,
                      ch.perturbed_superop(rng, ch.depolarizing2(0.04), 0.005))]
    c = _circ(w)
    f = DM.fidelity(c, w.psi, w.v)
    full = EX.approximate(c, w.psi, w.v, 4)
    assert abs(full["F"] - f) < 1e-13
    # O3 agrees with O2 term by term on the general case
    for lvl in (1, 2, 3):
        r2 = EX.approximate(c, w.psi, w.v, lvl, keep_terms=True)
        r3 = O3.approximate(c, w.psi, w.v, lvl)
        x2 = np.array([x for _, x in r2["terms"]])
        assert r3["n_terms"] == len(x2) == r2["n_terms"]
        assert np.max(np.abs(r3["terms"] - x2)) <= 1e-13 * np.max(np.abs(x2))
