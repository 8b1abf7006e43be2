"""Text form of a workload's circuit and noise sites (the shared data file).

Format, one record per line, '#' starts a comment:

    nqs-ir 1
    qubits <n>
    gate <name> <q0> [<q1>] [<param> ...]
    noise <after_gate> <qubit> <n_kraus> <re im> x (4 * n_kraus)

Gate names: h x y z t rx ry rz u3 cz cx.  Gates are numbered 0.. in file
order; a noise with after_gate = g acts right after gate g (g = -1: before
the first gate).  Noise lines must be ordered by after_gate; several noises
after the same gate act in file order.  Kraus matrices are row-major 2x2.
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
        for k in z.kraus:
            for a in range(2):
                for b in range(2):
                    c = complex(k[a, b])
                    vals.append(repr(c.real))
                    vals.append(repr(c.imag))
        lines.append("noise %d %d %d %s" % (z.after_gate, z.qubit, len(z.kraus), " ".join(vals)))
    return "\n".join(lines) + "\n"
