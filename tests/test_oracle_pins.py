"""Pins of the FP64 oracle against values the paper and the mathematics fix.

Nothing here compares the oracle with itself: each check is a closed form,
a worked value printed in the paper, brute force over an independent
definition, or an identity of linear algebra.
"""

import cmath
import itertools
import math

import numpy as np
import pytest

import workloads as W
from workloads import channels as ch
from oracle import bounds as B
from oracle import density_matrix as DM
from oracle import expansion as EX
from oracle import gates as G
from oracle import ir as IR
from oracle import statevector as SV


def _circ(w):
    return IR.parse(W.to_ir_text(w))


def _rng(seed):
    return W.SplitMix64(seed)


def _rand_matrix(rng, r, c):
    return np.array([[ch.gauss(rng) + 1j * ch.gauss(rng) for _ in range(c)] for _ in range(r)])


# ----------------------------------------------------------------------------
# Table I gates and the state-vector step

def test_table1_gates_are_unitary_and_satisfy_pauli_algebra():
    names = [("h", ()), ("x", ()), ("y", ()), ("z", ()), ("t", ()), ("rx", (0.7,)),
             ("ry", (1.3,)), ("rz", (2.1,)), ("u3", (0.3, 1.1, 2.9))]
    for name, ps in names:
        u = G.one_qubit(name, ps)
        assert np.allclose(u.conj().T @ u, np.eye(2), atol=1e-15), name
    X, Y, Z, H, T = (G.one_qubit(k) for k in "xyzht")
    assert np.allclose(X @ Y, 1j * Z)
    assert np.allclose(H @ H, np.eye(2))
    assert np.allclose(H @ X @ H, Z)
    assert np.allclose(np.linalg.matrix_power(T, 8), np.eye(2))
    assert np.allclose(T @ T, np.diag([1, 1j]))                       # T^2 = S
    # rotations are exponentials of Paulis: R_a(t) = cos(t/2) I - i sin(t/2) a
    for a, name in ((X, "rx"), (Y, "ry"), (Z, "rz")):
        t = 0.913
        assert np.allclose(G.one_qubit(name, (t,)),
                           math.cos(t / 2) * np.eye(2) - 1j * math.sin(t / 2) * a)
    # U3 special cases (OpenQASM convention)
    assert np.allclose(G.one_qubit("u3", (0.4, 0.0, 0.0)), G.one_qubit("ry", (0.4,)))
    assert np.allclose(G.one_qubit("u3", (0.4, -math.pi / 2, math.pi / 2)), G.one_qubit("rx", (0.4,)))
    assert np.allclose(G.one_qubit("u3", (math.pi / 2, 0, math.pi)), H)


def test_controlled_gates_act_on_basis_states():
    # CX with control q0=2, target q1=0 on n=3: |x2 x1 x0>
    for bits in range(8):
        out = SV.apply_2q(SV.basis_state(3, bits), 3, 2, 0, G.two_qubit("cx"))
        expect = bits ^ 1 if bits & 4 else bits
        assert np.allclose(out, SV.basis_state(3, expect))
        out = SV.apply_2q(SV.basis_state(3, bits), 3, 0, 2, G.two_qubit("cz"))
        sign = -1 if (bits & 1 and bits & 4) else 1
        assert np.allclose(out, sign * SV.basis_state(3, bits))


def _full_operator(n, qubits, m):
    """Dense 2^n operator built index by index from the definition."""
    d = 1 << n
    out = np.zeros((d, d), dtype=np.complex128)
    k = len(qubits)
    for col in range(d):
        sub_in = 0
        for q in qubits:
            sub_in = (sub_in << 1) | ((col >> q) & 1)
        for sub_out in range(1 << k):
            row = col
            for j, q in enumerate(qubits):
                bit = (sub_out >> (k - 1 - j)) & 1
                row = (row & ~(1 << q)) | (bit << q)
            out[row, col] += m[sub_out, sub_in]
    return out


@pytest.mark.parametrize("qubits", [(0,), (2,), (3,), (0, 3), (3, 1), (2, 1)])
def test_statevector_matches_dense_operator(qubits):
    rng = _rng(11)
    n = 4
    psi = _rand_matrix(rng, 1, 16)[0]
    m = _rand_matrix(rng, 2 ** len(qubits), 2 ** len(qubits))
    got = SV.apply_op(psi, n, qubits, m)
    assert np.allclose(got, _full_operator(n, qubits, m) @ psi, atol=1e-13)


def test_c_state_vector_step_matches_numpy():
    from oracle import csim
    rng = _rng(12)
    n = 7
    psi = _rand_matrix(rng, 1, 1 << n)[0]
    ops = csim.OpList()
    ref = psi.copy()
    for qs in [(0,), (6,), (3, 5), (5, 3), (0, 6), (2,)]:
        m = _rand_matrix(rng, 2 ** len(qs), 2 ** len(qs))
        ops.add(qs, m)
        ref = SV.apply_op(ref, n, qs, m)
    got = csim.apply_ops(n, np.ascontiguousarray(psi.copy()), ops)
    assert np.allclose(got, ref, atol=1e-12)
    ref_ip = np.vdot(psi, got)
    assert abs(csim.inner(n, psi, got) - ref_ip) < 1e-13 * abs(ref_ip)


# ----------------------------------------------------------------------------
# tensor permutation and SVD factors (Sec. IV, Fig. 3, Lemmas 1-2)

def test_identity_tensor_permutation_worked_value(golden):
    want = np.array(golden("identity_tensor_permutation.txt"))
    # M of the identity channel is the 4x4 identity (Sec. III with E = I)
    m = EX.matrix_representation([np.eye(2, dtype=np.complex128)])
    assert np.array_equal(m, np.eye(4))
    assert np.array_equal(EX.tensor_permutation(m).real, want)
    assert np.array_equal(EX.tensor_permutation(np.eye(4)), want)


def test_tensor_permutation_is_an_involution_and_keeps_frobenius_norm():
    rng = _rng(13)
    for _ in range(5):
        a = _rand_matrix(rng, 4, 4)
        assert np.array_equal(EX.tensor_permutation(EX.tensor_permutation(a)), a)
        assert math.isclose(np.linalg.norm(EX.tensor_permutation(a)), np.linalg.norm(a))
    # it is a genuine regrouping: not the identity map and not a transpose
    a = _rand_matrix(rng, 4, 4)
    assert not np.allclose(EX.tensor_permutation(a), a)
    assert not np.allclose(EX.tensor_permutation(a), a.T)


def test_kron_product_permutes_to_outer_product_of_vectorizations():
    rng = _rng(14)
    u, v = _rand_matrix(rng, 2, 2), _rand_matrix(rng, 2, 2)
    # (u (x) v)~ = vec(u) vec(v)^T : a rank-one matrix (Fig. 3c)
    got = EX.tensor_permutation(np.kron(u, v))
    assert np.allclose(got, np.outer(u.reshape(-1), v.reshape(-1)))
    assert np.linalg.matrix_rank(got) == 1


CHANNELS = [
    ("depol", ch.depolarizing_paper(0.02)),
    ("ad", ch.amplitude_damping(0.05)),
    ("pd", ch.phase_damping(0.03)),
    ("adpd", ch.ad_pd(0.01, 0.02)),
    ("rand1", ch.near_identity_channel(_rng(21), 0.03, 1)),
    ("rand3", ch.near_identity_channel(_rng(22), 0.01, 3)),
]


@pytest.mark.parametrize("name,kraus", CHANNELS)
def test_svd_factors_rebuild_the_channel(name, kraus):
    d, u, v, ut, vt = EX.svd_factors(kraus)
    m = EX.matrix_representation(kraus)
    # M = sum_i U_i (x) V_i (Fig. 3c)
    assert np.allclose(sum(np.kron(u[i], v[i]) for i in range(4)), m, atol=1e-14)
    # and the action on a density matrix equals the Kraus form:
    # (A (x) B) vec(rho) = vec(A rho B^T) for row-major vec
    rng = _rng(23)
    a = _rand_matrix(rng, 2, 2)
    rho = a @ a.conj().T
    rho /= np.trace(rho)
    want = sum(e @ rho @ e.conj().T for e in kraus)
    got = sum(u[i] @ rho @ v[i].T for i in range(4))
    assert np.allclose(got, want, atol=1e-14)
    assert np.all(np.diff(d) <= 1e-15) and d[0] > d[1]


@pytest.mark.parametrize("name,kraus", CHANNELS)
def test_realigned_channel_is_psd_so_both_networks_share_factors(name, kraus):
    mt = EX.tensor_permutation(EX.matrix_representation(kraus))
    assert np.allclose(mt, mt.conj().T, atol=1e-15)
    assert np.min(np.linalg.eigvalsh(mt)) > -1e-14
    d, u, v, _, _ = EX.svd_factors(kraus)
    for i in range(4):
        if d[i] > 1e-9:
            # U_i = d_i A_i and V_i = conj(B_i) with A_i = B_i
            assert np.allclose(u[i] / d[i], v[i].conj(), atol=1e-9)


def test_lemma1_norm_inequality():
    rng = _rng(31)
    for _ in range(200):
        a, b = _rand_matrix(rng, 4, 4), _rand_matrix(rng, 4, 4)
        lhs = np.linalg.norm(EX.tensor_permutation(a) - EX.tensor_permutation(b), 2)
        assert lhs <= 2 * np.linalg.norm(a - b, 2) * (1 + 1e-12)


def test_lemma2_dominant_factor_error():
    rng = _rng(32)
    for k in range(100):
        eps = 10 ** (-3 + 2.5 * rng.uniform())
        kraus = ch.near_identity_channel(rng, eps, 1 + k % 3)
        m = EX.matrix_representation(kraus)
        delta = np.linalg.norm(m - np.eye(4), 2)
        m_dom, m_rest = EX.dominant_and_rest(kraus)
        assert np.allclose(m_dom + m_rest, m, atol=1e-14)
        assert np.linalg.norm(m - m_dom, 2) <= 4 * delta * (1 + 1e-12)


def test_depolarizing_noise_rate_readings():
    # the definition ||M - I|| gives 4p/3 for the paper's depolarizing form,
    # while the "2p" of Sec. IV is ||M~ - I~||
    for p in (1e-3, 0.01, 0.2):
        m = EX.matrix_representation(ch.depolarizing_paper(p))
        assert math.isclose(B.noise_rate(ch.depolarizing_paper(p)), 4 * p / 3, rel_tol=1e-12)
        assert math.isclose(np.linalg.norm(EX.tensor_permutation(m) - EX.tensor_permutation(np.eye(4)), 2),
                            2 * p, rel_tol=1e-12)


def test_non_dominant_channel_is_rejected():
    with pytest.raises(EX.NotDominant):
        EX.svd_factors(ch.depolarizing_paper(0.75))   # M~ proportional to identity


# ----------------------------------------------------------------------------
# closed forms

def _poly_closed_form_depol(p_list_per_qubit, x_order):
    """F(x) = prod_q 1/2 [prod_s (1-p_s+p_s x) + prod_s (1-p_s-p_s x/3)];
    returns coefficients T_0..T_x_order."""
    total = np.array([1.0])
    for ps in p_list_per_qubit:
        a = np.array([1.0])
        b = np.array([1.0])
        for p in ps:
            a = np.convolve(a, [1 - p, p])
            b = np.convolve(b, [1 - p, -p / 3])
        total = np.convolve(total, 0.5 * (a + b))
    out = np.zeros(x_order + 1)
    out[:min(len(total), x_order + 1)] = total[:x_order + 1]
    return out


@pytest.mark.parametrize("p,N", [(0.01, 1), (0.05, 3), (0.2, 4)])
def test_depolarizing_identity_circuit_closed_form(p, N):
    w = W.identity_workload(1, [(0, ch.depolarizing_paper(p))] * N)
    c = _circ(w)
    f = DM.fidelity(c, w.psi, w.v)
    assert math.isclose(f.real, 0.5 * (1 + (1 - 4 * p / 3) ** N), rel_tol=1e-13)
    r = EX.approximate(c, w.psi, w.v, N)
    for u in range(N + 1):
        want = math.comb(N, u) * (1 - p) ** (N - u) * (p / 3) ** u * (3 ** u + (-1) ** u) / 2
        assert math.isclose(r["T"][u].real, want, rel_tol=1e-11, abs_tol=1e-300)
    assert math.isclose(r["F"].real, f.real, rel_tol=1e-13)


def test_depolarizing_several_qubits_closed_form():
    ps = [[0.01, 0.03], [0.02], [0.05, 0.01, 0.004]]
    noise = [(q, ch.depolarizing_paper(p)) for q, lst in enumerate(ps) for p in lst]
    w = W.identity_workload(3, noise)
    c = _circ(w)
    N = len(noise)
    coef = _poly_closed_form_depol(ps, N)
    r = EX.approximate(c, w.psi, w.v, N)
    for u in range(N + 1):
        assert abs(r["T"][u].real - coef[u]) < 1e-15 + 1e-12 * abs(coef[u])
    assert math.isclose(DM.fidelity(c, w.psi, w.v).real, sum(coef), rel_tol=1e-13)


@pytest.mark.parametrize("p", [1e-3, 0.1, 0.5])
def test_mixing_form_depolarizing_single_noise(p):
    # rho -> (1-p) rho + p I/2 on |0>: F = 1 - p/2
    w = W.identity_workload(1, [(0, ch.depolarizing_mixing(p))])
    c = _circ(w)
    assert math.isclose(DM.fidelity(c, w.psi, w.v).real, 1 - p / 2, rel_tol=1e-14)
    assert math.isclose(EX.approximate(c, w.psi, w.v, 1)["F"].real, 1 - p / 2, rel_tol=1e-13)


@pytest.mark.parametrize("gamma,N", [(0.01, 3), (0.2, 4)])
def test_amplitude_damping_closed_forms(gamma, N):
    noise = [(0, ch.amplitude_damping(gamma))] * N
    w = W.identity_workload(1, noise, psi_bits=1, v_bits=1)
    c = _circ(w)
    r = EX.approximate(c, w.psi, w.v, N)
    assert math.isclose(r["T"][0].real, (1 - gamma) ** N, rel_tol=1e-13)
    assert all(abs(t) < 1e-15 for t in r["T"][1:])
    assert math.isclose(DM.fidelity(c, w.psi, w.v).real, (1 - gamma) ** N, rel_tol=1e-13)
    w = W.identity_workload(1, noise, psi_bits=1, v_bits=0)
    c = _circ(w)
    r = EX.approximate(c, w.psi, w.v, N)
    assert abs(r["T"][0]) < 1e-15
    assert math.isclose(r["T"][1].real, 1 - (1 - gamma) ** N, rel_tol=1e-12)
    assert all(abs(t) < 1e-15 for t in r["T"][2:])


def test_noiseless_limit_ghz():
    # p = 0: every noise is the identity channel; A(l) = |<v|U|psi>|^2
    w = W.Workload("ghz", 3, [("h", (0,), ()), ("cx", (0, 1), ()), ("cx", (1, 2), ())],
                   [W.Noise(0, 0, [np.eye(2, dtype=np.complex128)]),
                    W.Noise(2, 2, ch.depolarizing_paper(0.0))])
    c = _circ(w)
    for v_bits, want in ((0, 0.5), (7, 0.5), (3, 0.0), (5, 0.0)):
        for lvl in (0, 1, 2):
            r = EX.approximate(c, {"kind": "basis", "bits": 0}, {"kind": "basis", "bits": v_bits}, lvl)
            assert abs(r["F"] - want) < 1e-15
            assert all(abs(t) < 1e-30 for t in r["T"][1:])
        assert abs(DM.fidelity(c, {"kind": "basis", "bits": 0}, {"kind": "basis", "bits": v_bits}) - want) < 1e-15


def test_identity_channel_factors():
    d, u, v, _, _ = EX.svd_factors([np.eye(2, dtype=np.complex128)])
    assert np.allclose(d, [2, 0, 0, 0], atol=1e-15)
    assert np.allclose(np.kron(u[0], v[0]), np.eye(4))


# ----------------------------------------------------------------------------
# full level equals the exact result; O1 against an independent definition

def _trajectory_sum(c, psi_spec, v_spec):
    """F = sum over every Kraus index sequence of |<v| C[E_k1 .. E_kN] |psi>|^2:
    the Kraus decomposition of the composed channel (independent of O1)."""
    n = c.n
    psi = DM.state_from_spec(psi_spec, n)
    v = DM.state_from_spec(v_spec, n, c, psi)
    total = []
    for ks in itertools.product(*[range(len(z[2])) for z in c.noises]):
        s = psi.copy()
        for kind, idx in IR.events(c):
            if kind == "gate":
                name, qs, ps = c.gates[idx]
                s = SV.apply_op(s, n, qs, G.gate_matrix(name, ps))
            else:
                s = SV.apply_1q(s, n, c.noises[idx][1], c.noises[idx][2][ks[idx]])
        total.append(abs(np.vdot(v, s)) ** 2)
    return math.fsum(total)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_density_matrix_oracle_matches_trajectory_sum(seed):
    w = W.random_circuit(seed, 3, 14, 3, rate_lo=0.02, rate_hi=0.2)
    c = _circ(w)
    assert math.isclose(DM.fidelity(c, w.psi, w.v).real, _trajectory_sum(c, w.psi, w.v),
                        rel_tol=1e-12, abs_tol=1e-15)


@pytest.mark.parametrize("seed,n,gates,noise", [(1, 3, 20, 3), (2, 4, 24, 4), (3, 5, 30, 4),
                                                 (4, 2, 10, 5), (5, 4, 18, 3)])
def test_full_level_equals_exact(seed, n, gates, noise):
    w = W.random_circuit(seed, n, gates, noise, rate_lo=0.005, rate_hi=0.1)
    c = _circ(w)
    N = len(c.noises)
    f = DM.fidelity(c, w.psi, w.v)
    r = EX.approximate(c, w.psi, w.v, N)
    assert abs(r["F"] - f) < 1e-12 * max(1.0, abs(f))
    assert abs(f.imag) < 1e-14


def test_full_level_equals_exact_dense_states():
    w = W.random_circuit(9, 3, 16, 3, v_kind="dense")
    w.psi = {"kind": "dense", "amps": W.circuits.random_dense_state(_rng(99), 3)}
    c = _circ(w)
    f = DM.fidelity(c, w.psi, w.v)
    r = EX.approximate(c, w.psi, w.v, 3)
    assert abs(r["F"] - f) < 1e-13


def test_trace_preservation_and_monotone_levels():
    w = W.random_circuit(4, 3, 15, 3, rate_lo=0.01, rate_hi=0.1)
    c = _circ(w)
    N = len(c.noises)
    fs, a_by_level = [], [[] for _ in range(N + 1)]
    for v_bits in range(8):
        v = {"kind": "basis", "bits": v_bits}
        fs.append(DM.fidelity(c, w.psi, v).real)
        r = EX.approximate(c, w.psi, v, N, keep_terms=True)
        assert min(x.real for _, x in r["terms"]) > -1e-15       # every term is PSD
        acc = 0.0
        for lvl in range(N + 1):
            acc += r["T"][lvl].real
            a_by_level[lvl].append(acc)
    assert math.isclose(math.fsum(fs), 1.0, rel_tol=1e-13)
    sums = [math.fsum(a) for a in a_by_level]
    assert math.isclose(sums[-1], 1.0, rel_tol=1e-12)
    assert all(x <= y + 1e-15 for x, y in zip(sums, sums[1:]))
    assert all(x <= 1 + 1e-13 for x in sums)


# ----------------------------------------------------------------------------
# enumeration and counts

def test_kept_assignments_match_brute_force():
    for N in range(0, 6):
        for lvl in range(0, N + 2):
            brute = []
            for sigma in itertools.product(range(4), repeat=N):
                sites = tuple(s for s in range(N) if sigma[s])
                if len(sites) <= lvl:
                    brute.append((len(sites), sites, tuple(sigma[s] for s in sites)))
            brute.sort()
            assert list(EX.kept_assignments(N, lvl)) == brute
            assert len(brute) == EX.term_count(N, lvl)


def test_record_packing_round_trip():
    for k, sites, idx in EX.kept_assignments(9, 4):
        r = EX.pack_record(k, sites, idx)
        assert r & 15 == k
        for j in range(k):
            f = (r >> (4 + 14 * j)) & 0x3FFF
            assert f & 0xFFF == sites[j] and f >> 12 == idx[j]
        assert r >> (4 + 14 * k) == 0


def test_contraction_count_matches_figure4(golden):
    for n_noise, samples in golden("fig4_level1_contractions.txt"):
        assert B.contraction_count(int(n_noise), 1) == int(samples)
    assert B.contraction_count(10, 2) == 2 * (1 + 30 + 45 * 9)
    assert EX.term_count(20, 2) == 1771 and EX.term_count(20, 1) == 61
    assert EX.term_count(4, 4) == 256 and EX.term_count(200, 3) == 35641501


# ----------------------------------------------------------------------------
# error bounds (Theorem 1, level-1 corollary, per-site bound)

@pytest.mark.parametrize("seed", [3, 5, 8])
def test_truncation_error_within_bounds(seed):
    w = W.random_circuit(seed, 4, 30, 5, rate_lo=1e-3, rate_hi=2e-2)
    c = _circ(w)
    N = len(c.noises)
    f = DM.fidelity(c, w.psi, w.v).real
    kl = [z[2] for z in c.noises]
    p = max(B.noise_rate(k) for k in kl)
    r = EX.approximate(c, w.psi, w.v, N)
    acc = 0.0
    for lvl in range(N):
        acc += r["T"][lvl].real
        err = abs(f - acc)
        assert err <= B.per_site_bound(kl, lvl) * (1 + 1e-9) + 1e-15
        assert err <= B.theorem1_bound(N, p, lvl) * (1 + 1e-9) + 1e-15
        if lvl == 1 and p <= 1 / (8 * N):
            assert err <= B.level1_corollary(N, p)
    # Theorem 1 at l = N is zero; at l = 1 it is the tail sum over k >= 2 that
    # the level-1 corollary starts from (the corollary's first line subtracts
    # 1 where the theorem subtracts (1+4p)^N; the tail-sum form is used)
    assert B.theorem1_bound(N, p, N) == pytest.approx(0.0, abs=1e-13)
    tail = math.fsum(math.comb(N, k) * (4 * p) ** k * (1 + 4 * p) ** (N - k) for k in range(2, N + 1))
    assert math.isclose(B.theorem1_bound(N, p, 1), tail, rel_tol=1e-12)


def _per_site_by_subsets(norms, level):
    """Brute force over every site set S with |S| > level of
    prod_{s in S} a_s prod_{s not in S} b_s, with (a_s, b_s) given."""
    N = len(norms)
    tot = []
    for k in range(level + 1, N + 1):
        for S in itertools.combinations(range(N), k):
            term = 1.0
            for s in range(N):
                term *= norms[s][0] if s in S else norms[s][1]
            tot.append(term)
    return math.fsum(tot)


def test_per_site_bound_identical_depolarizing_is_a_binomial_tail():
    # paper-form depolarizing: M' = (1-p) I(x)I and M-bar = p/3 (X(x)X - Y(x)Y + Z(x)Z),
    # whose eigenvalues on the Bell basis are p/3 * {3, -1, -1, -1}: ||M-bar|| = p,
    # ||M'|| = 1 - p, so for N identical sites the bound is P[Binomial(N, p) > l]
    from scipy.stats import binom
    for N, p in ((1, 0.2), (5, 0.03), (12, 0.01), (20, 0.004)):
        kl = [ch.depolarizing_paper(p)] * N
        for lvl in range(0, min(N, 4) + 1):
            want = float(binom.sf(lvl, N, p))
            got = B.per_site_bound(kl, lvl)
            assert math.isclose(got, want, rel_tol=1e-9, abs_tol=1e-300), (N, p, lvl, got, want)
    # the swapped norms would give P[Binomial(N, 1-p) > l], close to 1
    assert B.per_site_bound([ch.depolarizing_paper(0.01)] * 10, 1) < 5e-3


def test_per_site_bound_mixed_channels_brute_force():
    # phase damping: M~ restricted to {|00>, |11>} is [[1, r], [r, 1]] with
    # r = sqrt(1 - lambda); M' = (1 + r)/2 I(x)I, M-bar = (1 - r)/2 Z(x)Z^*
    def pd_norms(lam):
        r = math.sqrt(1.0 - lam)
        return ((1.0 - r) / 2.0, (1.0 + r) / 2.0)
    chans = [("dep", 0.02), ("pd", 0.05), ("dep", 0.001), ("pd", 0.3), ("dep", 0.1), ("pd", 0.01)]
    kl, norms = [], []
    for kind, r in chans:
        if kind == "dep":
            kl.append(ch.depolarizing_paper(r))
            norms.append((r, 1.0 - r))
        else:
            kl.append(ch.phase_damping(r))
            norms.append(pd_norms(r))
    for lvl in range(len(chans)):
        want = _per_site_by_subsets(norms, lvl)
        assert math.isclose(B.per_site_bound(kl, lvl), want, rel_tol=1e-12), lvl
    assert B.per_site_bound(kl, len(chans)) == 0.0


def test_theorem1_bound_hand_values():
    # (1+8p)^N expands binomially as sum_i C(N,i) (4p)^i (1+4p)^(N-i); the bound is its tail.
    # p = 1/100: N=2, l=0: 1.08^2 - 1.04^2 = 0.0848; l=1: (0.04)^2 = 0.0016;
    # N=3, l=1: 3 (0.04)^2 1.04 + 0.04^3 = 0.005056; N=3, l=2: 0.04^3 = 6.4e-5
    assert math.isclose(B.theorem1_bound(2, 0.01, 0), 0.0848, rel_tol=1e-12)
    assert math.isclose(B.theorem1_bound(2, 0.01, 1), 0.0016, rel_tol=1e-12)
    assert math.isclose(B.theorem1_bound(3, 0.01, 1), 0.005056, rel_tol=1e-12)
    assert math.isclose(B.theorem1_bound(3, 0.01, 2), 6.4e-5, rel_tol=1e-9)
    assert B.theorem1_bound(3, 0.01, 5) == 0.0
    # level-1 corollary, hand value: 32 sqrt(e) 10^2 (1e-3)^2 = 0.005275908...
    assert math.isclose(B.level1_corollary(10, 1e-3), 0.0052759080662, rel_tol=1e-10)
    # and it dominates the level-1 tail whenever p <= 1/(8N), as the paper's corollary states
    for N in (1, 2, 5, 20, 100):
        for f in (1.0, 0.5, 0.1, 0.01):
            p = f / (8 * N)
            assert B.theorem1_bound(N, p, 1) <= B.level1_corollary(N, p)


def test_level1_error_grows_quadratically_in_rate():
    # Fig. 6 trend: level-1 error ~ p^2
    errs = []
    for p in (1e-3, 2e-3, 4e-3):
        rng = _rng(77)
        w = W.random_circuit(77, 4, 30, 0)
        pos = sorted(rng.choice_distinct(len(w.gates), 6))
        w.noises = [W.Noise(g, w.gates[g][1][0], ch.depolarizing_paper(p)) for g in pos]
        c = _circ(w)
        f = DM.fidelity(c, w.psi, w.v).real
        errs.append(abs(f - EX.approximate(c, w.psi, w.v, 1)["F"].real))
    assert 3.2 < errs[1] / errs[0] < 4.8 and 3.2 < errs[2] / errs[1] < 4.8


# ----------------------------------------------------------------------------
# planted mistakes: each pin above must catch a plausible error in the oracle

def _pins_pass():
    try:
        test_identity_tensor_permutation_worked_value(lambda n: __import__("conftest").read_golden(n))
        for name, k in CHANNELS:
            test_svd_factors_rebuild_the_channel(name, k)
        test_depolarizing_identity_circuit_closed_form(0.05, 3)
        test_amplitude_damping_closed_forms(0.2, 4)
        test_full_level_equals_exact(2, 4, 24, 4)
    except AssertionError:
        return False
    return True


def test_planted_mistakes_are_caught(monkeypatch):
    assert _pins_pass()
    good_perm = EX.tensor_permutation
    good_mrep = EX.matrix_representation
    good_svd = EX.svd_factors
    good_net = EX._network_amplitude

    # 1. wrong regrouping (transpose instead of the (1,3)(2,4) permutation)
    monkeypatch.setattr(EX, "tensor_permutation",
                        lambda m: np.asarray(m).reshape(2, 2, 2, 2).transpose(0, 3, 1, 2).reshape(4, 4))
    assert not _pins_pass()
    monkeypatch.setattr(EX, "tensor_permutation", good_perm)

    # 2. dropped conjugate in the matrix representation
    monkeypatch.setattr(EX, "matrix_representation",
                        lambda ks: sum(np.kron(e, e) for e in ks))
    assert not _pins_pass()
    monkeypatch.setattr(EX, "matrix_representation", good_mrep)

    # 3. dropped Kraus term
    monkeypatch.setattr(EX, "matrix_representation", lambda ks: good_mrep(ks[:-1] if len(ks) > 1 else ks))
    assert not _pins_pass()
    monkeypatch.setattr(EX, "matrix_representation", good_mrep)

    # 4. V factor without the conjugate
    def bad_svd(kraus):
        d, u, v, ut, vt = good_svd(kraus)
        return d, u, [x.conj() for x in v], ut, vt
    monkeypatch.setattr(EX, "svd_factors", bad_svd)
    assert not _pins_pass()
    monkeypatch.setattr(EX, "svd_factors", good_svd)

    # 5. conjugate network contracted with unconjugated gates
    def bad_net(circuit, psi, v, inserted, conjugate_side):
        return good_net(circuit, psi, v, inserted, False)
    monkeypatch.setattr(EX, "_network_amplitude", bad_net)
    assert not _pins_pass()
    monkeypatch.setattr(EX, "_network_amplitude", good_net)
    assert _pins_pass()

    # 6. per-site bound with ||M'|| and ||M-bar|| swapped, and 7. Theorem 1 with
    # the head summed one level short: the bound pins must fail
    good_dar = B.dominant_and_rest
    monkeypatch.setattr(B, "dominant_and_rest", lambda k: tuple(reversed(good_dar(k))))
    with pytest.raises(AssertionError):
        test_per_site_bound_identical_depolarizing_is_a_binomial_tail()
    with pytest.raises(AssertionError):
        test_per_site_bound_mixed_channels_brute_force()
    monkeypatch.setattr(B, "dominant_and_rest", good_dar)
    good_t1 = B.theorem1_bound
    monkeypatch.setattr(B, "theorem1_bound", lambda N, p, l: good_t1(N, p, max(l - 1, 0)))
    with pytest.raises(AssertionError):
        test_theorem1_bound_hand_values()
    monkeypatch.setattr(B, "theorem1_bound", good_t1)
    test_per_site_bound_identical_depolarizing_is_a_binomial_tail()
    test_theorem1_bound_hand_values()


# ----------------------------------------------------------------------------
# off-diagonal elements <x|rho|y> (Sec. III)

@pytest.mark.parametrize("seed", [61, 62])
def test_offdiagonal_full_level_is_the_density_matrix_element(seed):
    w = W.random_circuit(seed, 3, 20, 3, rate_lo=1e-2, rate_hi=0.1)
    c = _circ(w)
    rng = _rng(seed)
    x = {"kind": "dense", "amps": W.circuits.random_dense_state(rng, 3)}
    y = {"kind": "basis", "bits": 5}
    want = DM.matrix_element(c, w.psi, x, y)
    got = EX.approximate_offdiagonal(c, w.psi, x, y, 3)["value"]
    assert abs(got - want) < 1e-13
    # Hermiticity of the level-l approximation and the x = y reduction
    for lvl in (0, 1, 2):
        a = EX.approximate_offdiagonal(c, w.psi, x, y, lvl)["value"]
        b = EX.approximate_offdiagonal(c, w.psi, y, x, lvl)["value"]
        assert abs(a - b.conjugate()) < 1e-14
        assert abs(EX.approximate_offdiagonal(c, w.psi, x, x, lvl)["value"] -
                   EX.approximate(c, w.psi, x, lvl)["F"]) < 1e-14


def test_offdiagonal_basis_elements_of_a_known_state():
    # identity circuit, one depolarizing noise on |+>: rho = (1-2p/3)|+><+| + (p/3) I ... element <0|rho|1>
    # = (1 - 4p/3) / 2 for the paper-form channel (the coherence shrinks by 1 - 4p/3)
    p = 0.09
    w = W.identity_workload(1, [(0, ch.depolarizing_paper(p))])
    w.psi = {"kind": "dense", "amps": [2 ** -0.5, 2 ** -0.5]}
    c = _circ(w)
    got = EX.approximate_offdiagonal(c, w.psi, {"kind": "basis", "bits": 0}, {"kind": "basis", "bits": 1}, 1)
    assert abs(got["value"] - (1 - 4 * p / 3) / 2) < 1e-15
