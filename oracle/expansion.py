"""O2 / O4: the level-l approximation of Sec. IV in FP64 (oracle; test
infrastructure only).

The oracle first lists the kept assignments, then evaluates each one:

1. matrix representation of each noise, M_E = sum_k E_k (x) E_k^*  (Sec. III);
2. tensor permutation M -> M~: with M's edges (1,2) as row and (3,4) as
   column, M~ takes (1,3) as row and (2,4) as column (Sec. IV, Fig. 3a);
3. SVD M~ = S D T^dagger with d_0 the largest singular value;
   U~_i = d_i S|i>, V~_i = T|i>, so M~ = sum_i U~_i V~_i^dagger (Fig. 3b);
4. tensor permutation back: M = sum_i U_i (x) V_i (Fig. 3c);
5. kept assignments (O4): every level k <= l, every site set p_1 < ... < p_k
   and every choice of a non-dominant factor i in {1,2,3} at those sites,
   the dominant factor U_0 (x) V_0 everywhere else (Algorithm 1);
6. each kept assignment splits the double-size network into the network on
   the original wires (gates U, factors U_i) and the one on the conjugate
   wires (gates U^*, factors V_i); both are contracted -- here by a plain
   state-vector sweep -- and multiplied; T_k sums those products and
   A(l) = sum_{k<=l} T_k.

O4's order is the record format shared with the library's enumerator:
level, then site tuple lexicographic, then factor tuple lexicographic,
packed as 64-bit records: bits 0-3 the level u, then for r = 0..u-1 a 14-bit
field at bit 4 + 14 r holding the site index (12 bits) and, above it, the
factor index (2 bits).
"""

import itertools
import math

import numpy as np

from . import gates as G
from . import ir as IR
from . import statevector as SV
from .density_matrix import state_from_spec

DOMINANCE_RTOL = 1e-12


class NotDominant(ValueError):
    pass


def matrix_representation(kraus):
    """M_E = sum_k E_k (x) E_k^*  (Sec. III); a d^2 x d^2 matrix for d x d
    Kraus operators; a noise given as a SuperOp is its matrix already."""
    if isinstance(kraus, IR.SuperOp):
        return kraus.m.copy()
    d = kraus[0].shape[0]
    m = np.zeros((d * d, d * d), dtype=np.complex128)
    for e in kraus:
        m += np.kron(e, e.conj())
    return m


def tensor_permutation(m):
    """Regroup a d^2 x d^2 matrix with (row edges 1,2 ; column edges 3,4) into
    (row edges 1,3 ; column edges 2,4)  (Sec. IV, Fig. 3a).  An involution.
    Edge 1 is the original wire's output, 2 the conjugate wire's output, 3 and
    4 their inputs; for a two-qubit noise every edge carries both qubits."""
    m = np.asarray(m)
    d = int(round(m.shape[0] ** 0.5))
    t = m.reshape(d, d, d, d)                          # [e1, e2, e3, e4]
    return t.transpose(0, 2, 1, 3).reshape(d * d, d * d)   # [(e1, e3), (e2, e4)]


def svd_factors(kraus):
    """SVD of M~ and the factors of Fig. 3.

    Returns (d, U, V, Ut, Vt): singular values d_0 >= ... >= d_{m-1}
    (m = 4 for a one-qubit noise, 16 for a two-qubit one), d x d factors
    with M_E = sum_i U_i (x) V_i, and the vectors U~_i = d_i S|i>, V~_i = T|i>.
    Raises NotDominant when d_0 does not strictly exceed d_1 (the dominant
    factor would not be unique)."""
    mt = tensor_permutation(matrix_representation(kraus))
    m = mt.shape[0]
    dd = int(round(m ** 0.5))
    s, d, th = np.linalg.svd(mt)
    t = th.conj().T
    if d[0] - d[1] <= DOMINANCE_RTOL * d[0]:
        raise NotDominant("largest singular value is not unique")
    ut = [d[i] * s[:, i] for i in range(m)]
    vt = [t[:, i] for i in range(m)]
    # U~_i V~_i^dagger, permuted back, is U_i (x) V_i with
    # U_i[e1, e3] = U~_i[(e1, e3)] and V_i[e2, e4] = conj(V~_i[(e2, e4)])
    u = [ut[i].reshape(dd, dd) for i in range(m)]
    v = [vt[i].conj().reshape(dd, dd) for i in range(m)]
    return d, u, v, ut, vt


def dominant_and_rest(kraus):
    """M' = U_0 (x) V_0 and M-bar = sum_{i>=1} U_i (x) V_i (Sec. IV)."""
    _, u, v, _, _ = svd_factors(kraus)
    m_dom = np.kron(u[0], v[0])
    m_rest = sum(np.kron(u[i], v[i]) for i in range(1, len(u)))
    return m_dom, m_rest


# ----------------------------------------------------------------------------
# kept assignments (O4)

def kept_assignments(n_noise, level, m=None):
    """(k, sites, factors) in Algorithm 1's loop order; m[s] factors at site s
    (4 for every site when m is None), index 0 the dominant one."""
    level = min(level, n_noise)
    for k in range(level + 1):
        for sites in itertools.combinations(range(n_noise), k):
            ranges = [range(1, 4 if m is None else m[s]) for s in sites]
            for idx in itertools.product(*ranges):
                yield k, sites, idx


def pack_record(k, sites, idx):
    if k > 4:
        raise ValueError("records hold at most 4 insertions")
    r = k
    for j, (s, i) in enumerate(zip(sites, idx)):
        if s >= 4096:
            raise ValueError("site index does not fit the 12-bit record field")
        r |= (s | (i << 12)) << (4 + 14 * j)
    return r


def enumerate_records(n_noise, level):
    return [pack_record(k, s, i) for k, s, i in kept_assignments(n_noise, level)]


def term_count(n_noise, level, m=None):
    level = min(level, n_noise)
    if m is None:
        return sum(math.comb(n_noise, u) * 3 ** u for u in range(level + 1))
    return sum(1 for _ in kept_assignments(n_noise, level, m))


# ----------------------------------------------------------------------------
# contraction of one split network by a state-vector sweep

def _network_amplitude(circuit, psi, v, inserted, conjugate_side):
    """Contract one of the two networks of a substituted double-size network.

    Original side: <v| C[factors] |psi> with the gates U.
    Conjugate side: <v^*| C^*[factors] |psi^*> with the gates U^* (the lower
    half of the double-size network of Sec. III)."""
    n = circuit.n
    s = psi.conj() if conjugate_side else psi.copy()
    for kind, idx in IR.events(circuit):
        if kind == "gate":
            name, qs, ps = circuit.gates[idx]
            g = G.gate_matrix(name, ps)
            s = SV.apply_op(s, n, qs, g.conj() if conjugate_side else g)
        else:
            s = SV.apply_op(s, n, IR.site_qubits(circuit.noises[idx][1]), inserted[idx])
    bra = v.conj() if conjugate_side else v
    return complex(np.vdot(bra, s))


def prepared_factors(circuit):
    return [svd_factors(k) for (_, _, k) in circuit.noises]


def term_value(circuit, psi, v, factors, sites, idx):
    """X of Algorithm 1 for one kept assignment: the product of the two
    contracted networks."""
    n_noise = len(circuit.noises)
    choice = [0] * n_noise
    for s, i in zip(sites, idx):
        choice[s] = i
    ins_u = [factors[s][1][choice[s]] for s in range(n_noise)]
    ins_v = [factors[s][2][choice[s]] for s in range(n_noise)]
    a = _network_amplitude(circuit, psi, v, ins_u, False)
    b = _network_amplitude(circuit, psi, v, ins_v, True)
    return a * b


def _fsum_complex(xs):
    return complex(math.fsum(x.real for x in xs), math.fsum(x.imag for x in xs))


def approximate(circuit, psi_spec, v_spec, level, keep_terms=False, amplitude_fn=None):
    """A(l) of Algorithm 1.

    Returns dict(F=complex A(l), T=[complex T_0..T_l], terms=[(record, X)] if
    keep_terms, n_terms).  Levels above N are clamped to N."""
    n = circuit.n
    psi = state_from_spec(psi_spec, n)
    v = state_from_spec(v_spec, n, circuit, psi)
    factors = prepared_factors(circuit)
    n_noise = len(circuit.noises)
    level = min(level, n_noise)
    m = [len(f[1]) for f in factors]
    per_level = [[] for _ in range(level + 1)]
    terms = []
    for k, sites, idx in kept_assignments(n_noise, level, m):
        if amplitude_fn is None:
            x = term_value(circuit, psi, v, factors, sites, idx)
        else:
            x = amplitude_fn(circuit, psi, v, factors, sites, idx)
        per_level[k].append(x)
        if keep_terms:
            packable = k <= 4 and all(i <= 3 for i in idx) and all(s < 4096 for s in sites)
            terms.append((pack_record(k, sites, idx) if packable else None, x))
    t = [_fsum_complex(xs) for xs in per_level]
    return {"F": _fsum_complex(t), "T": t, "terms": terms,
            "n_terms": term_count(n_noise, level, m)}


def approximate_offdiagonal(circuit, psi_spec, x_spec, y_spec, level):
    """Level-l approximation of one element <x| E(|psi><psi|) |y> (Sec. III).

    The double-size network of Sec. III ends in <x| on the original wires and
    <y^*| on the conjugate wires; substituting the factors of Sec. IV and
    keeping the assignments of Algorithm 1 gives, per kept assignment, the
    product of the original-side network with bra <x| and the conjugate-side
    network with bra <y^*|.  For x = y this is approximate()."""
    n = circuit.n
    psi = state_from_spec(psi_spec, n)
    x = state_from_spec(x_spec, n, circuit, psi)
    y = state_from_spec(y_spec, n, circuit, psi)
    factors = prepared_factors(circuit)
    n_noise = len(circuit.noises)
    level = min(level, n_noise)
    m = [len(f[1]) for f in factors]
    per_level = [[] for _ in range(level + 1)]
    for k, sites, idx in kept_assignments(n_noise, level, m):
        choice = [0] * n_noise
        for s, i in zip(sites, idx):
            choice[s] = i
        ins_u = [factors[s][1][choice[s]] for s in range(n_noise)]
        ins_v = [factors[s][2][choice[s]] for s in range(n_noise)]
        a = _network_amplitude(circuit, psi, x, ins_u, False)
        b = _network_amplitude(circuit, psi, y, ins_v, True)
        per_level[k].append(a * b)
    t = [_fsum_complex(xs) for xs in per_level]
    return {"value": _fsum_complex(t), "T": t, "n_terms": term_count(n_noise, level, m)}


def site_set_sums(terms, n_noise):
    """Sum of term values per site set (basis independent under degenerate
    singular values).  terms: [(record, X)]."""
    out = {}
    for rec, x in terms:
        k = rec & 15
        sites = tuple(((rec >> (4 + 14 * j)) & 0xFFF) for j in range(k))
        out[sites] = out.get(sites, 0) + x
    return out
