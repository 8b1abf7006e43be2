"""Seeded synthetic workloads: circuits, noise placements and input states.

A workload is plain data: a gate list (name, qubits, angles), a list of noise
sites (after which gate, on which qubit, which Kraus list) and descriptors of
the input state psi and test state v.  The paper's benchmark circuits (ReCirq
QAOA / HF-VQE / supremacy instances) and its decoherence parameters are not
available, so these generators stand in for them with the same structure:
QAOA MaxCut on a random 3-regular graph, grid random circuits of U3 layers and
alternating CZ patterns, and decoherence / depolarizing noise appended after
randomly chosen gates (Sec. V).

Qubit q is bit q of a basis-state index (index = sum_q x_q 2^q).  For a
two-qubit gate the first listed qubit is the control / the more significant
bit of the gate's 4x4 matrix.
"""

from dataclasses import dataclass, field
import math

import numpy as np

from .rng import SplitMix64
from . import channels as ch

GATE_ARITY = {"h": 1, "x": 1, "y": 1, "z": 1, "t": 1, "rx": 1, "ry": 1, "rz": 1,
              "u3": 1, "cz": 2, "cx": 2}
GATE_NPARAM = {"h": 0, "x": 0, "y": 0, "z": 0, "t": 0, "rx": 1, "ry": 1, "rz": 1,
               "u3": 3, "cz": 0, "cx": 0}


@dataclass
class Noise:
    after_gate: int          # index of the gate this noise follows (-1: before all gates)
    qubit: int
    kraus: list              # list of 2x2 (4x4 for two qubits) complex128 arrays
    label: str = ""
    qubit2: int = -1         # second qubit of a two-qubit noise (-1: one qubit)
    superop: object = None   # instead of Kraus operators: the matrix representation M (4x4 or 16x16)


@dataclass
class Workload:
    name: str
    n: int
    gates: list                      # [(name, (q0[, q1]), (params...))]
    noises: list                     # [Noise], ordered by after_gate (stable)
    psi: dict = field(default_factory=lambda: {"kind": "basis", "bits": 0})
    v: dict = field(default_factory=lambda: {"kind": "basis", "bits": 0})
    levels: tuple = (1,)
    meta: dict = field(default_factory=dict)

    @property
    def n_noise(self) -> int:
        return len(self.noises)


# ----------------------------------------------------------------------------
# helpers

def _pick_noise_qubit(rng, gate):
    qs = gate[1]
    return qs[0] if len(qs) == 1 else qs[rng.randbelow(len(qs))]


def _place_noises(rng, gates, n_noise, make_kraus):
    """n_noise noises after distinct seeded gates, sorted by position."""
    pos = sorted(rng.choice_distinct(len(gates), n_noise))
    out = []
    for g in pos:
        q = _pick_noise_qubit(rng, gates[g])
        kraus, label = make_kraus(rng)
        out.append(Noise(g, q, kraus, label))
    return out


def _u3_layer(rng, qubits):
    two_pi = 2.0 * math.pi
    return [("u3", (q,), (rng.uniform_range(0, two_pi), rng.uniform_range(0, two_pi),
                          rng.uniform_range(0, two_pi))) for q in qubits]


def grid_cz_pattern(rows, cols, layer):
    """CZ pairs of a rows x cols grid for the given layer (layer mod 4 cycles
    horizontal-even, horizontal-odd, vertical-even, vertical-odd edges)."""
    k = layer % 4
    pairs = []
    if k in (0, 1):
        for r in range(rows):
            for c in range(k, cols - 1, 2):
                pairs.append((r * cols + c, r * cols + c + 1))
    else:
        for r in range(k - 2, rows - 1, 2):
            for c in range(cols):
                pairs.append((r * cols + c, (r + 1) * cols + c))
    return pairs


def line_cz_pattern(n, layer):
    return [(q, q + 1) for q in range(layer % 2, n - 1, 2)]


def random_bits(rng, n):
    return rng.next_u64() & ((1 << n) - 1)


def random_dense_state(rng, n):
    a = np.array([ch.gauss(rng) + 1j * ch.gauss(rng) for _ in range(1 << n)])
    return a / np.linalg.norm(a)


# ----------------------------------------------------------------------------
# the five configurations

def c1_line6(seed: int = 1) -> Workload:
    """n=6 line, depth 8 (U3 on every qubit then brick CZ), 4 paper-form
    depolarizing noises p=1e-3 after seeded distinct gates, psi=v=|0^6>."""
    rng = SplitMix64(seed)
    n, depth = 6, 8
    gates = []
    for layer in range(depth):
        gates += _u3_layer(rng, range(n))
        gates += [("cz", pr, ()) for pr in line_cz_pattern(n, layer)]
    noises = _place_noises(rng, gates, 4,
                           lambda r: (ch.depolarizing_paper(1e-3), "depol_paper p=1e-3"))
    return Workload("c1_line6", n, gates, noises,
                    {"kind": "basis", "bits": 0}, {"kind": "basis", "bits": 0}, (1, 4))


def grid_random_circuit(rng, rows, cols, depth):
    gates = []
    for layer in range(depth):
        gates += _u3_layer(rng, range(rows * cols))
        gates += [("cz", pr, ()) for pr in grid_cz_pattern(rows, cols, layer)]
    return gates


def c2_grid20(seed: int = 2) -> Workload:
    """4x5 grid, depth 16, 20 noises of amplitude damping gamma=1e-3 composed
    with phase damping lambda=1e-3, v a seeded bitstring."""
    rng = SplitMix64(seed)
    rows, cols, depth = 4, 5, 16
    gates = grid_random_circuit(rng, rows, cols, depth)
    noises = _place_noises(rng, gates, 20,
                           lambda r: (ch.ad_pd(1e-3, 1e-3), "pd(1e-3)*ad(1e-3)"))
    v_bits = random_bits(rng, rows * cols)
    return Workload("c2_grid20", rows * cols, gates, noises,
                    {"kind": "basis", "bits": 0}, {"kind": "basis", "bits": v_bits}, (1, 2))


def random_3_regular_graph(rng, n_vertices):
    """Configuration model with rejection: pair 3 stubs per vertex at random,
    retry until there is no self-loop and no repeated edge."""
    if (3 * n_vertices) % 2:
        raise ValueError("3-regular graph needs an even vertex count")
    while True:
        stubs = [v for v in range(n_vertices) for _ in range(3)]
        rng.shuffle(stubs)
        edges = set()
        ok = True
        for i in range(0, len(stubs), 2):
            a, b = stubs[i], stubs[i + 1]
            e = (min(a, b), max(a, b))
            if a == b or e in edges:
                ok = False
                break
            edges.add(e)
        if ok:
            return sorted(edges)


def qaoa_maxcut_circuit(rng, n, edges, p_layers):
    gates = [("h", (q,), ()) for q in range(n)]
    for _ in range(p_layers):
        gamma = rng.uniform_range(0.0, math.pi)
        beta = rng.uniform_range(0.0, math.pi)
        for a, b in edges:
            gates.append(("cx", (a, b), ()))
            gates.append(("rz", (b,), (2.0 * gamma,)))
            gates.append(("cx", (a, b), ()))
        gates += [("rx", (q,), (2.0 * beta,)) for q in range(n)]
    return gates


def qaoa_workload(n: int, seed: int, n_noise: int = 20, p_layers: int = 4,
                  v_kind: str = "ideal", name: str = None) -> Workload:
    rng = SplitMix64(seed)
    edges = random_3_regular_graph(rng, n)
    gates = qaoa_maxcut_circuit(rng, n, edges, p_layers)

    def mk(r):
        p = r.uniform_range(1e-4, 1e-2)
        return ch.depolarizing_paper(p), "depol_paper p=%.6g" % p

    noises = _place_noises(rng, gates, n_noise, mk)
    v_bits = random_bits(rng, n)
    v = {"kind": "ideal"} if v_kind == "ideal" else {"kind": "basis", "bits": v_bits}
    return Workload(name or "qaoa%d" % n, n, gates, noises, {"kind": "basis", "bits": 0},
                    v, (2,), {"edges": edges})


def c3_qaoa30(seed: int = 3, v_kind: str = "ideal") -> Workload:
    """n=30 QAOA MaxCut, random 3-regular graph, p=4, 20 paper-form
    depolarizing noises p ~ U[1e-4, 1e-2]; v = U|psi> (or a seeded bitstring)."""
    return qaoa_workload(30, seed, 20, 4, v_kind, "c3_qaoa30")


def _grid_dims(n):
    r = int(math.isqrt(n))
    while r >= 2:
        if n % r == 0 and n // r >= 2:
            return r, n // r
        r -= 1
    return None


def mixed_noise_kraus(rng, lo, hi):
    kind = rng.randbelow(3)
    rate = rng.log_uniform(lo, hi)
    if kind == 0:
        return ch.amplitude_damping(rate), "ad g=%.6g" % rate
    if kind == 1:
        return ch.phase_damping(rate), "pd l=%.6g" % rate
    return ch.depolarizing_paper(rate), "depol_paper p=%.6g" % rate


def c4_circuit(idx: int) -> Workload:
    """One of the 512 batched circuits: width U{12..24}, depth U{10..30}, grid
    (when the width factors) or line U3+CZ, 5..40 mixed AD / PD / depolarizing
    noises with log-uniform rates in [1e-4, 1e-2], level U{1, 2}, v = U|psi>."""
    rng = SplitMix64(4000 + idx)
    n = rng.randint(12, 24)
    depth = rng.randint(10, 30)
    dims = _grid_dims(n) if rng.randbelow(2) else None
    if dims:
        gates = grid_random_circuit(rng, dims[0], dims[1], depth)
    else:
        gates = []
        for layer in range(depth):
            gates += _u3_layer(rng, range(n))
            gates += [("cz", pr, ()) for pr in line_cz_pattern(n, layer)]
    n_noise = rng.randint(5, 40)
    noises = _place_noises(rng, gates, n_noise, lambda r: mixed_noise_kraus(r, 1e-4, 1e-2))
    level = rng.randint(1, 2)
    return Workload("c4_%03d" % idx, n, gates, noises, {"kind": "basis", "bits": 0},
                    {"kind": "ideal"}, (level,), {"grid": dims})


def c4_batch(count: int = 512) -> list:
    return [c4_circuit(i) for i in range(count)]


def c5_grid(seed: int = 5, cols: int = 7, rows: int = 4, depth: int = 24,
            n_noise: int = 200, rate_lo: float = 1e-4, rate_hi: float = 5e-3) -> Workload:
    """4 x cols grid random circuit with n_noise mixed noises placed after the
    U3 gate of (layer, qubit) slots whose column is < 5, so the 4x5 twin
    (cols=5) with the same seed carries the identical noise layout.  Rates are
    log-uniform in [rate_lo, rate_hi] (the draws do not depend on the range)."""
    rng = SplitMix64(seed)
    n = rows * cols
    # angles for a 4x7 grid are drawn for every (layer, row, col<7) so that the
    # twin reuses exactly the same angles on its columns
    angles = {}
    for layer in range(depth):
        for r in range(rows):
            for c in range(7):
                angles[(layer, r, c)] = (rng.uniform_range(0, 2 * math.pi),
                                         rng.uniform_range(0, 2 * math.pi),
                                         rng.uniform_range(0, 2 * math.pi))
    slots = [(layer, r, c) for layer in range(depth) for r in range(rows) for c in range(5)]
    chosen = sorted(rng.choice_distinct(len(slots), n_noise))
    noise_spec = {}
    for k in chosen:
        kraus, label = mixed_noise_kraus(rng, rate_lo, rate_hi)
        noise_spec[slots[k]] = (kraus, label)
    gates, noises = [], []
    for layer in range(depth):
        for r in range(rows):
            for c in range(cols):
                gates.append(("u3", (r * cols + c,), angles[(layer, r, c)]))
                if (layer, r, c) in noise_spec:
                    kraus, label = noise_spec[(layer, r, c)]
                    noises.append(Noise(len(gates) - 1, r * cols + c, kraus, label))
        gates += [("cz", pr, ()) for pr in grid_cz_pattern(rows, cols, layer)]
    noises.sort(key=lambda z: z.after_gate)
    return Workload("c5_grid%dx%d" % (rows, cols), n, gates, noises,
                    {"kind": "basis", "bits": 0}, {"kind": "ideal"}, (3,))


def c5_twin(seed: int = 5, rate_lo: float = 1e-4, rate_hi: float = 5e-3) -> Workload:
    return c5_grid(seed, cols=5, rate_lo=rate_lo, rate_hi=rate_hi)


def c5_twin_hot(seed: int = 5) -> Workload:
    """The twin with rates from the upper part of the range, [1e-3, 5e-3]: its
    level-3 sum exceeds 1e-6, so reaching |dF| <= 1e-6 needs level 3."""
    w = c5_twin(seed, 1e-3, 5e-3)
    w.name = "c5_twin_hot"
    return w


# ----------------------------------------------------------------------------
# small random circuits for property and parity tests

ALL_1Q = ["h", "x", "y", "z", "t", "rx", "ry", "rz", "u3"]


def random_circuit(seed: int, n: int, n_gates: int, n_noise: int,
                   noise_kinds=("depol", "ad", "pd", "adpd", "random"),
                   rate_lo: float = 1e-3, rate_hi: float = 5e-2,
                   v_kind: str = "basis") -> Workload:
    rng = SplitMix64(seed)
    gates = []
    for _ in range(n_gates):
        if n >= 2 and rng.randbelow(3) == 0:
            name = "cz" if rng.randbelow(2) else "cx"
            a = rng.randbelow(n)
            b = rng.randbelow(n - 1)
            b = b + 1 if b >= a else b
            gates.append((name, (a, b), ()))
        else:
            name = ALL_1Q[rng.randbelow(len(ALL_1Q))]
            q = rng.randbelow(n)
            params = tuple(rng.uniform_range(0, 2 * math.pi) for _ in range(GATE_NPARAM[name]))
            gates.append((name, (q,), params))

    def mk(r):
        kind = noise_kinds[r.randbelow(len(noise_kinds))]
        rate = r.log_uniform(rate_lo, rate_hi)
        if kind == "depol":
            return ch.depolarizing_paper(rate), "depol_paper p=%g" % rate
        if kind == "ad":
            return ch.amplitude_damping(rate), "ad g=%g" % rate
        if kind == "pd":
            return ch.phase_damping(rate), "pd l=%g" % rate
        if kind == "adpd":
            return ch.ad_pd(rate, 0.5 * rate), "pd*ad"
        return ch.near_identity_channel(r, rate, 1 + r.randbelow(3)), "random eps=%g" % rate

    n_noise = min(n_noise, len(gates))
    noises = _place_noises(rng, gates, n_noise, mk)
    psi = {"kind": "basis", "bits": random_bits(rng, n)}
    if v_kind == "ideal":
        v = {"kind": "ideal"}
    elif v_kind == "dense":
        v = {"kind": "dense", "amps": random_dense_state(rng, n)}
    else:
        v = {"kind": "basis", "bits": random_bits(rng, n)}
    return Workload("rand_n%d_s%d" % (n, seed), n, gates, noises, psi, v, (1, 2))


def identity_workload(n: int, noise_list: list, psi_bits: int = 0, v_bits: int = 0) -> Workload:
    """Circuit of identity-equivalent gates (none) carrying the given noises.

    noise_list: [(qubit, kraus)], all placed before the (empty) gate list in
    the given order (after_gate = -1)."""
    noises = [Noise(-1, q, k, "") for q, k in noise_list]
    return Workload("identity_n%d" % n, n, [], noises, {"kind": "basis", "bits": psi_bits},
                    {"kind": "basis", "bits": v_bits}, (1,))
