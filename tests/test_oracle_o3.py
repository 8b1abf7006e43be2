"""Pins of O3, the checkpointed FP64 evaluator (oracle/o3.py, oracle/csim/o3.c).

O3 must give every kept term of O2 (one sweep per network per term) to
1e-13 relative to the largest term, in both of its parallel modes (narrow
states: insertions spread over threads; wide states, n > 16: passes split
over amplitudes), and reproduce the closed forms on its own.
"""

import math

import numpy as np
import pytest

import workloads as W
from workloads import channels as ch
from oracle import density_matrix as DM
from oracle import expansion as EX
from oracle import ir as IR
from oracle import o3 as O3


def _circ(w):
    return IR.parse(W.to_ir_text(w))


def _o2_terms(c, w, level):
    r = EX.approximate(c, w.psi, w.v, level, keep_terms=True)
    return r, np.array([x for _, x in r["terms"]])


@pytest.mark.parametrize("seed,n,gates,noises,level", [
    (3, 4, 20, 5, 3), (5, 6, 30, 6, 2), (8, 5, 25, 4, 4), (11, 3, 12, 7, 5), (13, 7, 40, 3, 0),
    (17, 2, 10, 2, 1)])
def test_o3_equals_o2_every_term(seed, n, gates, noises, level):
    w = W.random_circuit(seed, n, gates, noises, rate_lo=1e-3, rate_hi=5e-2,
                         v_kind="dense" if seed % 2 else "basis")
    c = _circ(w)
    r2, x2 = _o2_terms(c, w, level)
    r3 = O3.approximate(c, w.psi, w.v, level)
    assert r3["n_terms"] == r2["n_terms"] == len(x2)
    scale = max(np.max(np.abs(x2)), 1e-300)
    assert np.max(np.abs(r3["terms"] - x2)) <= 1e-13 * scale
    for u in range(len(r2["T"])):
        assert abs(r3["T"][u] - r2["T"][u]) <= 1e-13 * scale * max(1, len(x2))


def test_o3_wide_mode_equals_o2():
    # n = 17 runs the amplitude-parallel branch of O3
    w = W.random_circuit(21, 17, 24, 3, rate_lo=1e-2, rate_hi=5e-2)
    c = _circ(w)
    r2, x2 = _o2_terms(c, w, 2)
    r3 = O3.approximate(c, w.psi, w.v, 2)
    assert np.max(np.abs(r3["terms"] - x2)) <= 1e-13 * np.max(np.abs(x2))


def test_o3_no_noise_is_the_plain_amplitude():
    w = W.random_circuit(4, 5, 30, 0)
    c = _circ(w)
    r3 = O3.approximate(c, w.psi, w.v, 2)
    psi = DM.state_from_spec(w.psi, c.n)
    v = DM.state_from_spec(w.v, c.n, c, psi)
    ideal = DM.state_from_spec({"kind": "ideal"}, c.n, c, psi)
    assert r3["n_terms"] == 1
    assert abs(r3["F"] - abs(np.vdot(v, ideal)) ** 2) < 1e-14


@pytest.mark.parametrize("p,N", [(0.01, 1), (0.05, 3), (0.2, 6)])
def test_o3_depolarizing_closed_form(p, N):
    # identity circuit, psi = v = |0>: T_u = C(N,u) (1-p)^(N-u) (p/3)^u (3^u + (-1)^u) / 2
    c = _circ(W.identity_workload(1, [(0, ch.depolarizing_paper(p))] * N))
    w = W.identity_workload(1, [(0, ch.depolarizing_paper(p))] * N)
    r = O3.approximate(c, w.psi, w.v, N)
    for u in range(N + 1):
        want = math.comb(N, u) * (1 - p) ** (N - u) * (p / 3) ** u * (3 ** u + (-1) ** u) / 2
        assert math.isclose(r["T"][u].real, want, rel_tol=1e-11, abs_tol=1e-300)
    assert math.isclose(r["F"].real, 0.5 * (1 + (1 - 4 * p / 3) ** N), rel_tol=1e-13)


def test_o3_full_level_equals_density_matrix():
    w = W.random_circuit(31, 5, 30, 5, rate_lo=1e-2, rate_hi=0.1)
    c = _circ(w)
    f = DM.fidelity(c, w.psi, w.v)
    r = O3.approximate(c, w.psi, w.v, 5)
    assert abs(r["F"] - f) < 1e-13


def test_o3_amplitude_damping_closed_form():
    # identity circuit, psi = v = |1>: every amplitude but level 0 vanishes, F = (1-g)^N
    g, N = 0.2, 4
    w = W.identity_workload(1, [(0, ch.amplitude_damping(g))] * N, psi_bits=1, v_bits=1)
    c = _circ(w)
    r = O3.approximate(c, w.psi, w.v, N)
    assert math.isclose(r["T"][0].real, (1 - g) ** N, rel_tol=1e-13)
    assert all(abs(t) < 1e-15 for t in r["T"][1:])


def test_o3_term_count_and_order():
    # canonical order: level, site tuple lexicographic, factor tuple lexicographic;
    # placing the term of a single inserted factor checks the offsets directly
    assert O3.lib().nqso3_term_count(20, O3._ip(np.full(20, 4, np.int32)), 2) == 1771
    assert O3.lib().nqso3_term_count(200, O3._ip(np.full(200, 4, np.int32)), 3) == 35641501
    m = np.array([4, 2, 3, 4], np.int32)
    # level <= 2 with 3, 1, 2, 3 non-dominant factors: 1 + 9 + (3*1 + 3*2 + 3*3 + 1*2 + 1*3 + 2*3)
    assert O3.lib().nqso3_term_count(4, O3._ip(m), 2) == 1 + 9 + 29
    # a network whose only non-zero factors sit at sites (1, 3) with indices (1, 2)
    n = 2
    ev = [("site", 0, (0,)), ("site", 1, (1,)), ("site", 2, (0,)), ("site", 3, (1,))]
    z = np.zeros((2, 2), complex)
    eye = np.eye(2, dtype=complex)
    facs = [[eye, z, z, z], [eye, eye * 2], [eye, z, z], [eye, z, eye * 3, z]]
    net = O3.Network(n, ev, facs)
    psi = np.zeros(4, complex)
    psi[0] = 1
    amps = net.amplitudes(psi, psi, 2)
    nz = np.flatnonzero(np.abs(amps) > 0)
    # level 0 (1), level 1: site 1 idx 1 at offset 1+3 = 4, site 3 idx 2 at 1+3+1+2+1 = 8;
    # level 2: sets (0,1),(0,2),(0,3),(1,2),(1,3): (1,3) starts at 10+3+6+9+2 = 30, idx (1,2) -> +1
    assert list(nz) == [0, 4, 8, 31]
    assert np.allclose(amps[nz], [1, 2, 3, 6])


@pytest.mark.parametrize("seed,n,k", [(51, 6, 1), (52, 5, 2), (53, 7, 3), (54, 17, 2)])
def test_o3_set_weights_equal_the_full_list(seed, n, k):
    # W(S) of chosen sets = the full level-k list summed per site set
    w = W.random_circuit(seed, n, 30 if n < 10 else 20, 6 if n < 10 else 4, rate_lo=1e-2, rate_hi=5e-2,
                         v_kind="ideal")
    c = _circ(w)
    r = O3.approximate(c, w.psi, w.v, k)
    N = len(c.noises)
    recs = EX.enumerate_records(N, k)
    sums = {}
    for rec, x in zip(recs, r["terms"]):
        u = rec & 15
        if u != k:
            continue
        key = tuple(((rec >> (4 + 14 * j)) & 0xFFF) for j in range(u))
        sums[key] = sums.get(key, 0) + x
    import itertools
    sets = list(itertools.combinations(range(N), k))[::2]
    got = O3.set_weights(c, w.psi, w.v, np.array(sets))
    want = np.array([sums[tuple(s)] for s in sets])
    assert np.max(np.abs(got - want)) <= 1e-13 * max(1e-300, np.max(np.abs(want))) + 1e-300


def test_o3_timed_sample_predicts_the_complete_call():
    # the CPU baseline's method: the first passes of O3's call, timed and scaled
    # by the call's exact pass count, must predict the complete call's time
    import time
    w = W.qaoa_workload(18, 3, 8, 2, "ideal", "qaoa18")
    c = _circ(w)
    t0 = time.perf_counter()
    O3.approximate(c, w.psi, w.v, 2)
    full = time.perf_counter() - t0
    done, total, secs = O3.timed_sample(c, 0, -1, 2, 400)
    assert 0 < done <= total
    pred = secs * total / done
    assert 0.4 * full < pred < 2.5 * full, (pred, full)
    # and the pass count is that of the call: counting twice gives the same
    d2, t2, _ = O3.timed_sample(c, 0, -1, 2, 3, untimed=2)
    assert t2 == total and d2 == 1
