"""ctypes wrapper of oracle/csim/sv.c (oracle; test infrastructure only).

``build()`` compiles the C file with gcc into oracle/_build/; the functions
below run Algorithm 1's per-network contraction (a plain state-vector sweep)
in C for widths where numpy is too slow.  The arithmetic is identical to
oracle.statevector: one pass per operation, in circuit order.
"""

import ctypes
import os
import subprocess

import numpy as np

from . import gates as G
from . import ir as IR

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csim", "sv.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "libnqs_oracle_sv.so")
_lib = None


def build(force=False):
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.POINTER
        L.nqso_apply_ops.argtypes = [ctypes.c_int, P(ctypes.c_double), ctypes.c_int,
                                     P(ctypes.c_int), P(ctypes.c_int), P(ctypes.c_int),
                                     P(ctypes.c_double), ctypes.c_int]
        L.nqso_apply_ops.restype = None
        L.nqso_inner.argtypes = [ctypes.c_int, P(ctypes.c_double), P(ctypes.c_double),
                                 P(ctypes.c_double)]
        L.nqso_inner.restype = None
        L.nqso_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


class OpList:
    """A flat list of (qubits, matrix) operations for the C sweep."""

    def __init__(self):
        self.arity, self.q0, self.q1, self.mats = [], [], [], []

    def add(self, qubits, m):
        buf = np.zeros(16, dtype=np.complex128)
        buf[:m.size] = np.asarray(m, dtype=np.complex128).reshape(-1)
        self.arity.append(len(qubits))
        self.q0.append(qubits[0])
        self.q1.append(qubits[1] if len(qubits) > 1 else -1)
        self.mats.append(buf)

    def arrays(self):
        return (np.array(self.arity, dtype=np.int32), np.array(self.q0, dtype=np.int32),
                np.array(self.q1, dtype=np.int32),
                np.ascontiguousarray(np.concatenate(self.mats).view(np.float64))
                if self.mats else np.zeros(32, dtype=np.float64))


def apply_ops(n, state, ops: OpList, threads=0):
    """In place on a complex128 array of length 2^n."""
    assert state.dtype == np.complex128 and state.flags.c_contiguous and state.size == 1 << n
    ar, q0, q1, mats = ops.arrays()
    lib().nqso_apply_ops(n, _dp(state.view(np.float64)), len(ops.arity), _ip(ar), _ip(q0),
                         _ip(q1), _dp(mats), threads)
    return state


def inner(n, a, b):
    out = np.zeros(2, dtype=np.float64)
    lib().nqso_inner(n, _dp(a.view(np.float64)), _dp(b.view(np.float64)), _dp(out))
    return complex(out[0], out[1])


def circuit_ops(circuit, inserted=None, conjugate=False, upto_event=None):
    """The circuit's event sequence as an OpList; noise site s contributes
    inserted[s] (or nothing when inserted is None)."""
    ops = OpList()
    for e, (kind, idx) in enumerate(IR.events(circuit)):
        if upto_event is not None and e >= upto_event:
            break
        if kind == "gate":
            name, qs, ps = circuit.gates[idx]
            g = G.gate_matrix(name, ps)
            ops.add(qs, g.conj() if conjugate else g)
        elif inserted is not None:
            ops.add(IR.site_qubits(circuit.noises[idx][1]), inserted[idx])
    return ops


def network_amplitude(circuit, psi, v, inserted, conjugate_side, threads=0):
    """Same contraction as expansion._network_amplitude, swept in C."""
    n = circuit.n
    s = np.ascontiguousarray(psi.conj() if conjugate_side else psi.copy())
    apply_ops(n, s, circuit_ops(circuit, inserted, conjugate_side), threads)
    bra = np.ascontiguousarray(v.conj() if conjugate_side else v)
    return inner(n, bra, s)


def term_value(circuit, psi, v, factors, sites, idx, threads=0):
    """Drop-in amplitude_fn for expansion.approximate: X = product of the two
    contracted networks, each swept in C."""
    n_noise = len(circuit.noises)
    choice = [0] * n_noise
    for s, i in zip(sites, idx):
        choice[s] = i
    ins_u = [factors[s][1][choice[s]] for s in range(n_noise)]
    ins_v = [factors[s][2][choice[s]] for s in range(n_noise)]
    a = network_amplitude(circuit, psi, v, ins_u, False, threads)
    b = network_amplitude(circuit, psi, v, ins_v, True, threads)
    return a * b


def ideal_state(circuit, psi, threads=0):
    s = np.ascontiguousarray(psi.copy())
    apply_ops(circuit.n, s, circuit_ops(circuit, None, False), threads)
    return s
