"""Reader of the circuit/noise text format (oracle; test infrastructure only).

Line records: ``nqs-ir 1``, ``qubits n``, ``gate name q0 [q1] [params]``,
``noise after_gate qubit n_kraus re im ...`` (row-major 2x2 Kraus matrices),
``noise2 after_gate q0 q1 n_kraus re im ...`` (4x4, index 2*b(q0) + b(q1)),
``superop after_gate qubit re im ...`` and ``superop2 after_gate q0 q1 re im
...`` (the matrix representation M directly, 4x4 / 16x16).
Written independently of the library's own reader.

A noise entry is (after_gate, qubits, spec): qubits an int for one qubit and
a pair for two, spec a list of Kraus matrices or a SuperOp.
"""

from dataclasses import dataclass

import numpy as np

ARITY = {"h": 1, "x": 1, "y": 1, "z": 1, "t": 1, "rx": 1, "ry": 1, "rz": 1, "u3": 1,
         "cz": 2, "cx": 2}
NPARAM = {"h": 0, "x": 0, "y": 0, "z": 0, "t": 0, "rx": 1, "ry": 1, "rz": 1, "u3": 3,
          "cz": 0, "cx": 0}


class SuperOp:
    """A noise given by its matrix representation M (Sec. III) instead of
    Kraus operators."""

    def __init__(self, m):
        self.m = np.asarray(m, dtype=np.complex128)


def site_qubits(q):
    """The qubits of a noise entry as a tuple."""
    return tuple(q) if isinstance(q, tuple) else (q,)


@dataclass
class Circuit:
    n: int
    gates: list      # [(name, (qubits...), (params...))]
    noises: list     # [(after_gate, qubit, [2x2 arrays])]


def parse(text: str) -> Circuit:
    n = None
    gates, noises = [], []
    seen_header = False
    for raw in text.splitlines():
        line = raw.split("#", 1)[0].strip()
        if not line:
            continue
        tok = line.split()
        if tok[0] == "nqs-ir":
            if tok[1] != "1":
                raise ValueError("unsupported IR version")
            seen_header = True
        elif tok[0] == "qubits":
            n = int(tok[1])
        elif tok[0] == "gate":
            name = tok[1]
            a = ARITY[name]
            qs = tuple(int(x) for x in tok[2:2 + a])
            ps = tuple(float(x) for x in tok[2 + a:])
            if len(ps) != NPARAM[name]:
                raise ValueError("wrong parameter count for " + name)
            gates.append((name, qs, ps))
        elif tok[0] in ("noise", "noise2"):
            two = tok[0] == "noise2"
            g = int(tok[1])
            q = (int(tok[2]), int(tok[3])) if two else int(tok[2])
            k = int(tok[4] if two else tok[3])
            vals = [float(x) for x in tok[(5 if two else 4):]]
            d = 4 if two else 2
            if len(vals) != 2 * d * d * k:
                raise ValueError("wrong Kraus value count")
            mats = []
            for j in range(k):
                v = vals[2 * d * d * j:2 * d * d * (j + 1)]
                mats.append(np.array([v[2 * e] + 1j * v[2 * e + 1] for e in range(d * d)],
                                     dtype=np.complex128).reshape(d, d))
            noises.append((g, q, mats))
        elif tok[0] in ("superop", "superop2"):
            two = tok[0] == "superop2"
            g = int(tok[1])
            q = (int(tok[2]), int(tok[3])) if two else int(tok[2])
            vals = [float(x) for x in tok[(4 if two else 3):]]
            d2 = 16 if two else 4
            if len(vals) != 2 * d2 * d2:
                raise ValueError("wrong superoperator value count")
            m = np.array([vals[2 * e] + 1j * vals[2 * e + 1] for e in range(d2 * d2)]).reshape(d2, d2)
            noises.append((g, q, SuperOp(m)))
        else:
            raise ValueError("unknown record " + tok[0])
    if not seen_header or n is None:
        raise ValueError("missing header or qubit count")
    return Circuit(n, gates, noises)


def events(c: Circuit):
    """The circuit as one ordered sequence: ('gate', g) and ('noise', s).

    Noise s with after_gate g acts right after gate g (g = -1: before gate 0);
    the noise sites are numbered s = 0..N-1 in that order, which is the
    i_1, ..., i_N order of the noise channels in Sec. IV."""
    by_gate = {}
    for s, (g, _, _) in enumerate(c.noises):
        by_gate.setdefault(g, []).append(s)
    prev = -2
    for g, _, _ in c.noises:
        if g < prev or g < -1 or g >= len(c.gates):
            raise ValueError("noise sites must be ordered by after_gate and in range")
        prev = g
    out = [("noise", s) for s in by_gate.get(-1, [])]
    for g in range(len(c.gates)):
        out.append(("gate", g))
        out += [("noise", s) for s in by_gate.get(g, [])]
    return out
