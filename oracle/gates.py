"""Gate matrices, FP64 (oracle; test infrastructure only).

Single-qubit gates follow Table I of the paper (H, X, Y, Z, T, Rx, Ry, Rz).
Two-qubit gates follow the controlled-U construction of Sec. II: the first
qubit is the control and the more significant index bit of the 4x4 matrix.
U3 is not in the paper; it uses the OpenQASM convention
U3(t, f, l) = [[cos t/2, -e^{il} sin t/2], [e^{if} sin t/2, e^{i(f+l)} cos t/2]].
"""

import cmath
import math

import numpy as np


def one_qubit(name, params=()):
    if name == "h":
        s = 1.0 / math.sqrt(2.0)
        return np.array([[s, s], [s, -s]], dtype=np.complex128)
    if name == "x":
        return np.array([[0, 1], [1, 0]], dtype=np.complex128)
    if name == "y":
        return np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
    if name == "z":
        return np.array([[1, 0], [0, -1]], dtype=np.complex128)
    if name == "t":
        return np.array([[1, 0], [0, cmath.exp(1j * math.pi / 4)]], dtype=np.complex128)
    if name == "rx":
        (th,) = params
        c, s = math.cos(th / 2), math.sin(th / 2)
        return np.array([[c, -1j * s], [-1j * s, c]], dtype=np.complex128)
    if name == "ry":
        (th,) = params
        c, s = math.cos(th / 2), math.sin(th / 2)
        return np.array([[c, -s], [s, c]], dtype=np.complex128)
    if name == "rz":
        (th,) = params
        return np.array([[cmath.exp(-1j * th / 2), 0], [0, cmath.exp(1j * th / 2)]],
                        dtype=np.complex128)
    if name == "u3":
        th, ph, la = params
        c, s = math.cos(th / 2), math.sin(th / 2)
        return np.array([[c, -cmath.exp(1j * la) * s],
                         [cmath.exp(1j * ph) * s, cmath.exp(1j * (ph + la)) * c]],
                        dtype=np.complex128)
    raise KeyError(name)


def controlled(u):
    """Controlled-U on (control, target): block diag(I, U) (Sec. II)."""
    m = np.eye(4, dtype=np.complex128)
    m[2:, 2:] = u
    return m


def two_qubit(name, params=()):
    if name == "cz":
        return controlled(one_qubit("z"))
    if name == "cx":
        return controlled(one_qubit("x"))
    raise KeyError(name)


def gate_matrix(name, params=()):
    try:
        return one_qubit(name, params)
    except KeyError:
        return two_qubit(name, params)
