"""O3: the level-l expansion by forward/backward FP64 checkpoints, in C with
OpenMP (oracle; test infrastructure only).

Same quantity as ``expansion.approximate`` (Sec. IV, Algorithm 1): every kept
term is the product of two contracted networks, X = a * b, with

* a = <v| C[U_sigma] |psi>     -- gates U, factors U_i at the noise sites,
* b = <v^*| C^*[V_sigma] |psi^*> -- gates U^*, factors V_i (the conjugate wires),

and the factors come from the same SVD of the tensor-permuted matrix
representation (``expansion.svd_factors``).  The C part (csim/o3.c) obtains
all the kept amplitudes of one network at once from backward checkpoints
phi_s and forward states, re-sweeping a level-u assignment only from its
first insertion; it shares no code with the library.  Used for widths and
term counts where the one-sweep-per-term evaluator is too slow.
"""

import ctypes
import os
import subprocess

import numpy as np

from . import expansion as EX
from . import gates as G
from . import ir as IR
from .density_matrix import state_from_spec

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csim", "o3.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "libnqs_oracle_o3.so")
_lib = None


def build(force=False):
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.POINTER
        ip, dp = P(ctypes.c_int), P(ctypes.c_double)
        L.nqso3_amplitudes.argtypes = [ctypes.c_int, ctypes.c_int, ip, ip, ip, ip, ip, dp, ctypes.c_int, ip, dp,
                                       dp, dp, ctypes.c_int, dp, ctypes.c_int64, P(ctypes.c_int64), ctypes.c_int]
        L.nqso3_amplitudes.restype = ctypes.c_int
        L.nqso3_set_amplitudes.argtypes = [ctypes.c_int, ctypes.c_int, ip, ip, ip, ip, ip, dp, ctypes.c_int, ip,
                                           dp, dp, dp, ctypes.c_int, ip, ctypes.c_int64, dp, ctypes.c_int]
        L.nqso3_set_amplitudes.restype = ctypes.c_int
        L.nqso3_timed_passes.argtypes = [ctypes.c_int, ctypes.c_int, ip, ip, ip, ip, ip, dp, ctypes.c_int, ip, dp,
                                         ctypes.c_int64, ctypes.c_int64, dp, ctypes.c_int, ctypes.c_int64,
                                         ctypes.c_int64, ctypes.c_int, P(ctypes.c_double), ctypes.c_int]
        L.nqso3_timed_passes.restype = ctypes.c_int64
        L.nqso3_term_count.argtypes = [ctypes.c_int, ip, ctypes.c_int]
        L.nqso3_term_count.restype = ctypes.c_int64
        _lib = L
    return _lib


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Network:
    """One network of a split double-size network: the event list with its
    gate matrices and the factor list of every noise site."""

    def __init__(self, n, events, site_factors):
        # events: [("gate", qubits, matrix) | ("site", s, qubits)]; site_factors[s] = [F_0, F_1, ...]
        ne = len(events)
        self.n = n
        self.kind = np.zeros(ne, np.int32)
        self.nq = np.zeros(ne, np.int32)
        self.q0 = np.full(ne, -1, np.int32)
        self.q1 = np.full(ne, -1, np.int32)
        self.site = np.full(ne, -1, np.int32)
        self.mat = np.zeros((ne, 16), np.complex128)
        for e, ev in enumerate(events):
            if ev[0] == "gate":
                _, qs, m = ev
                self.mat[e, :m.size] = np.asarray(m).reshape(-1)
            else:
                _, s, qs = ev
                self.kind[e] = 1
                self.site[e] = s
            self.nq[e] = len(qs)
            self.q0[e] = qs[0]
            if len(qs) > 1:
                self.q1[e] = qs[1]
        ns = len(site_factors)
        self.m = np.array([len(f) for f in site_factors], np.int32)
        self.fac = np.zeros((max(ns, 1), 16, 16), np.complex128)
        for s, fl in enumerate(site_factors):
            for j, f in enumerate(fl):
                self.fac[s, j, :f.size] = np.asarray(f).reshape(-1)

    def amplitudes(self, psi, bra, level, threads=0):
        """All kept amplitudes sum_i conj(bra_i) (C[F_sigma] psi)_i in the canonical order."""
        L = lib()
        mat = np.ascontiguousarray(self.mat).view(np.float64)
        fac = np.ascontiguousarray(self.fac).view(np.float64)
        psi = np.ascontiguousarray(psi, np.complex128)
        bra = np.ascontiguousarray(bra, np.complex128)
        count = L.nqso3_term_count(len(self.m), _ip(self.m), level)
        if count < 0:
            raise MemoryError("term table")
        out = np.zeros(count, np.complex128)
        nt = ctypes.c_int64(0)
        rc = L.nqso3_amplitudes(self.n, len(self.kind), _ip(self.kind), _ip(self.nq), _ip(self.q0), _ip(self.q1),
                                _ip(self.site), _dp(mat), len(self.m), _ip(self.m), _dp(fac),
                                _dp(psi.view(np.float64)), _dp(bra.view(np.float64)), level,
                                _dp(out.view(np.float64)), count, ctypes.byref(nt), threads)
        if rc != 0:
            raise RuntimeError("O3 failed (%d)" % rc)
        assert nt.value == count
        return out


    def set_amplitudes(self, psi, bra, sets, threads=0):
        """For each chosen site set (rows of `sets`, ascending sites) the
        amplitudes of every choice of non-dominant factors at its sites, the
        dominant factor elsewhere: a list of arrays in lexicographic order."""
        sets = np.ascontiguousarray(np.asarray(sets, dtype=np.int32))
        m_sets, k = sets.shape
        per = [int(np.prod([self.m[s] - 1 for s in row])) for row in sets]
        out = np.zeros(sum(per), np.complex128)
        mat = np.ascontiguousarray(self.mat).view(np.float64)
        fac = np.ascontiguousarray(self.fac).view(np.float64)
        psi = np.ascontiguousarray(psi, np.complex128)
        bra = np.ascontiguousarray(bra, np.complex128)
        rc = lib().nqso3_set_amplitudes(self.n, len(self.kind), _ip(self.kind), _ip(self.nq), _ip(self.q0),
                                        _ip(self.q1), _ip(self.site), _dp(mat), len(self.m), _ip(self.m), _dp(fac),
                                        _dp(psi.view(np.float64)), _dp(bra.view(np.float64)), k, _ip(sets), m_sets,
                                        _dp(out.view(np.float64)), threads)
        if rc != 0:
            raise RuntimeError("O3 set amplitudes failed (%d)" % rc)
        res, off = [], 0
        for c in per:
            res.append(out[off:off + c])
            off += c
        return res


    def passes(self, psi_bits, v_bits, bra, level, max_passes, dry, threads=0, untimed=0):
        """State passes of this network's wide-state call (see
        nqso3_timed_passes): executed up to max_passes, or only counted.
        bra=None: the bra is |v_bits>, or v = U|psi_bits> when v_bits < 0."""
        mat = np.ascontiguousarray(self.mat).view(np.float64)
        fac = np.ascontiguousarray(self.fac).view(np.float64)
        if bra is None:
            bp = None
        else:
            bra = np.ascontiguousarray(bra, np.complex128)
            bp = _dp(bra.view(np.float64))
        secs = ctypes.c_double(0.0)
        r = lib().nqso3_timed_passes(self.n, len(self.kind), _ip(self.kind), _ip(self.nq), _ip(self.q0),
                                     _ip(self.q1), _ip(self.site), _dp(mat), len(self.m), _ip(self.m), _dp(fac),
                                     int(psi_bits), int(v_bits), bp, level, int(max_passes), int(untimed),
                                     1 if dry else 0, ctypes.byref(secs), threads)
        if r < 0:
            raise MemoryError("O3: a state does not fit in host memory")
        self.last_seconds = secs.value
        return int(r)


def networks(circuit, factors=None):
    """The two networks of Algorithm 1 for a parsed circuit: (gates U, factors
    U_i) and (gates U^*, factors V_i), factors from expansion.svd_factors."""
    if factors is None:
        factors = EX.prepared_factors(circuit)
    ev_a, ev_b = [], []
    for kind, idx in IR.events(circuit):
        if kind == "gate":
            name, qs, ps = circuit.gates[idx]
            g = G.gate_matrix(name, ps)
            ev_a.append(("gate", qs, g))
            ev_b.append(("gate", qs, g.conj()))
        else:
            q = IR.site_qubits(circuit.noises[idx][1])
            ev_a.append(("site", idx, q))
            ev_b.append(("site", idx, q))
    fa = [list(f[1]) for f in factors]
    fb = [list(f[2]) for f in factors]
    return Network(circuit.n, ev_a, fa), Network(circuit.n, ev_b, fb)


def _neumaier(xs):
    s, c = 0.0, 0.0
    for x in xs:
        t = s + x
        c += (s - t) + x if abs(s) >= abs(x) else (x - t) + s
        s = t
    return s + c


def level_sums(terms, n_sites, level, m=None):
    """T_u of a canonical term array (np.complex128): per-level slices."""
    import math
    level = min(level, n_sites)
    if m is None:
        sizes = [math.comb(n_sites, u) * 3 ** u for u in range(level + 1)]
    else:
        sizes = [int(lib().nqso3_term_count(n_sites, _ip(np.asarray(m, np.int32)), u)) for u in range(level + 1)]
        sizes = [sizes[0]] + [sizes[u] - sizes[u - 1] for u in range(1, level + 1)]
    out, off = [], 0
    for sz in sizes:
        seg = terms[off:off + sz]
        out.append(complex(np.sum(seg.real, dtype=np.float64), np.sum(seg.imag, dtype=np.float64)))
        off += sz
    return out


def approximate(circuit, psi_spec, v_spec, level, threads=0, factors=None):
    """A(l) with every term X = a * b; returns dict(F, T, terms, n_terms) like
    expansion.approximate (terms: complex array in the canonical order)."""
    n = circuit.n
    psi = state_from_spec(psi_spec, n)
    v = state_from_spec(v_spec, n, circuit, psi)
    na, nb = networks(circuit, factors)
    level = min(level, len(circuit.noises))
    a = na.amplitudes(psi, v, level, threads)
    b = nb.amplitudes(psi.conj(), v.conj(), level, threads)
    x = a * b
    T = level_sums(x, len(circuit.noises), level, na.m)
    return {"F": sum(T), "T": T, "terms": x, "n_terms": len(x)}


def set_weights(circuit, psi_spec, v_spec, sets, threads=0, factors=None):
    """W(S) = sum over the factor choices at the sites of S of X = a * b
    (Sec. IV: the level-|S| terms of one site set), for each row of `sets`."""
    n = circuit.n
    psi = state_from_spec(psi_spec, n)
    v = state_from_spec(v_spec, n, circuit, psi)
    na, nb = networks(circuit, factors)
    a = na.set_amplitudes(psi, v, sets, threads)
    b = nb.set_amplitudes(psi.conj(), v.conj(), sets, threads)
    return np.array([complex(np.sum(x * y)) for x, y in zip(a, b)])


def timed_sample(circuit, psi_bits, v_bits, level, max_passes, threads=0, untimed=2):
    """Time the first `max_passes` state passes of O3's complete call
    (psi = |psi_bits>, v = |v_bits> or, for v_bits < 0, U|psi> computed in C;
    both networks), and count
    the passes of the complete call.  Returns (passes_done, passes_total,
    seconds of the passes after the first `untimed` -- the set-up of psi and
    v -- allocation and first touch of states excluded):
    the call's time is seconds * passes_total / passes_done when every pass
    sweeps the full state, as here."""
    na, nb = networks(circuit)
    level = min(level, len(circuit.noises))
    dummy = np.zeros(1, np.complex128)
    total = (na.passes(psi_bits, v_bits, None, level, 1 << 62, True) +
             nb.passes(psi_bits, v_bits, dummy, level, 1 << 62, True) + 1)
    done = na.passes(psi_bits, v_bits, None, level, max_passes, False, threads, untimed)
    return max(done - untimed, 0), total, na.last_seconds
