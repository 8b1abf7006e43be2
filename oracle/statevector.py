"""Plain FP64 state vectors with numpy (oracle; test infrastructure only).

Qubit q is bit q of the basis index, so in a C-order reshape to (2,)*n it is
axis n-1-q.  Gate application is a tensordot of the gate's matrix with the
state tensor -- the textbook definition of applying a local operator.
"""

import numpy as np


def basis_state(n, bits):
    s = np.zeros(1 << n, dtype=np.complex128)
    s[bits] = 1.0
    return s


def apply_1q(state, n, q, m):
    t = state.reshape((2,) * n)
    ax = n - 1 - q
    t = np.tensordot(m, t, axes=([1], [ax]))          # new axis 0 = output of m
    t = np.moveaxis(t, 0, ax)
    return t.reshape(-1)


def apply_2q(state, n, q0, q1, m):
    """m is 4x4 with row index 2*b(q0) + b(q1)."""
    t = state.reshape((2,) * n)
    a0, a1 = n - 1 - q0, n - 1 - q1
    g = m.reshape(2, 2, 2, 2)                          # [o0, o1, i0, i1]
    t = np.tensordot(g, t, axes=([2, 3], [a0, a1]))    # [o0, o1, rest...]
    t = np.moveaxis(t, [0, 1], [a0, a1])
    return t.reshape(-1)


def apply_op(state, n, qubits, m):
    if len(qubits) == 1:
        return apply_1q(state, n, qubits[0], m)
    return apply_2q(state, n, qubits[0], qubits[1], m)


def inner(a, b):
    """<a|b>."""
    return complex(np.vdot(a, b))
