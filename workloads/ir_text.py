"""Text form of a workload's circuit and noise sites (the shared data file).

Format, one record per line, '#' starts a comment:

    nqs-ir 1
    qubits <n>
    gate <name> <q0> [<q1>] [<param> ...]
    noise <after_gate> <qubit> <n_kraus> <re im> x (4 * n_kraus)
    noise2 <after_gate> <q0> <q1> <n_kraus> <re im> x (16 * n_kraus)
    superop <after_gate> <qubit> <re im> x 16
    superop2 <after_gate> <q0> <q1> <re im> x 256

Gate names: h x y z t rx ry rz u3 cz cx.  Gates are numbered 0.. in file
order; a noise with after_gate = g acts right after gate g (g = -1: before
the first gate).  Noise lines must be ordered by after_gate; several noises
after the same gate act in file order.  Kraus matrices are row-major 2x2
(4x4 for two qubits, indexed 2*b(q0) + b(q1)).  A superoperator record gives
the noise's matrix representation M = sum_k E_k (x) E_k^* directly (row
index (out, out'), column (in, in'), each pair with the original-wire index
first), so maps that are not completely positive can be written too.
Floats are written with Python's shortest round-trip repr, so both readers
recover the exact doubles.
"""

from .circuits import GATE_ARITY, GATE_NPARAM


def to_ir_text(w) -> str:
    lines = ["nqs-ir 1", "# %s" % w.name, "qubits %d" % w.n]
    for name, qs, params in w.gates:
        assert len(qs) == GATE_ARITY[name] and len(params) == GATE_NPARAM[name]
        lines.append("gate %s %s%s" % (name, " ".join(str(q) for q in qs),
                                       "".join(" " + repr(float(x)) for x in params)))
    prev = -2
    for z in w.noises:
        if z.after_gate < prev:
            raise ValueError("noise sites must be ordered by after_gate")
        prev = z.after_gate
        vals = []

        def put(c):
            c = complex(c)
            vals.append(repr(c.real))
            vals.append(repr(c.imag))
        two = getattr(z, "qubit2", -1) >= 0
        sop = getattr(z, "superop", None)
        if sop is not None:
            for c in sop.reshape(-1):
                put(c)
            if two:
                lines.append("superop2 %d %d %d %s" % (z.after_gate, z.qubit, z.qubit2, " ".join(vals)))
            else:
                lines.append("superop %d %d %s" % (z.after_gate, z.qubit, " ".join(vals)))
            continue
        for k in z.kraus:
            for c in k.reshape(-1):
                put(c)
        if two:
            lines.append("noise2 %d %d %d %d %s" % (z.after_gate, z.qubit, z.qubit2, len(z.kraus), " ".join(vals)))
        else:
            lines.append("noise %d %d %d %s" % (z.after_gate, z.qubit, len(z.kraus), " ".join(vals)))
    return "\n".join(lines) + "\n"
