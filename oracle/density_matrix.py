"""O1: exact noisy fidelity by density matrices, FP64 (oracle; test infrastructure only).

Follows the definitions of Sec. II and Problem 1 directly:
rho <- |psi><psi|; every gate U acts as rho -> U rho U^dagger, every noise
channel as rho -> sum_k E_k rho E_k^dagger (Kraus form), in circuit order;
F = <v| rho |v>.  Memory is 16 * 4^n bytes, so n <= 12.
"""

import numpy as np

from . import gates as G
from . import ir as IR
from . import ir as IR
from . import statevector as SV


def _left_right(rho, n, qubits, left, right):
    """rho -> left rho right^dagger for operators acting on `qubits`.

    rho[i, j] is held as the 2n-qubit tensor of index i * 2^n + j, so row
    qubit q is index bit n+q and column qubit q is index bit q; multiplying by
    `left` on the row index and by conj(right) on the column index is the
    index form of left . rho . right^dagger."""
    d = 1 << n
    flat = rho.reshape(-1)
    flat = SV.apply_op(flat, 2 * n, tuple(n + q for q in qubits), left)
    flat = SV.apply_op(flat, 2 * n, tuple(qubits), right.conj())
    return flat.reshape(d, d)


def apply_channel(rho, n, qubits, kraus):
    """sum_k E_k rho E_k^dagger (Kraus form, Sec. II)."""
    acc = np.zeros_like(rho)
    for e in kraus:
        acc += _left_right(rho, n, qubits, e, e)
    return acc


def apply_superop(rho, n, qubits, m):
    """rho -> the linear map whose matrix representation is M (Sec. III), on
    `qubits`, by its definition: vec(rho')[(o, o')] = sum_{i, i'} M[(o, o'),
    (i, i')] vec(rho)[(i, i')], where o, i index the site's qubits on the row
    (original) side and o', i' on the column (conjugate) side, each as
    2*b(q0) + b(q1).  For M = sum_k E_k (x) E_k^* this is sum_k E_k rho E_k^dagger."""
    k = len(qubits)
    t = rho.reshape((2,) * (2 * n))        # axis j: row qubit n-1-j; axis n+j: column qubit n-1-j
    rows = [n - 1 - q for q in qubits]
    cols = [2 * n - 1 - q for q in qubits]
    mt = np.asarray(m).reshape((2,) * (4 * k))   # [o..., o'..., i..., i'...]
    out = np.tensordot(mt, t, axes=(list(range(2 * k, 4 * k)), rows + cols))
    # out axes: o (k), o' (k), then the remaining axes of t in order
    rest = [a for a in range(2 * n) if a not in rows + cols]
    order = rows + cols + rest
    res = np.empty_like(t)
    res = np.moveaxis(out, list(range(2 * k + len(rest))), order)
    return res.reshape(rho.shape)


def state_from_spec(spec, n, circuit=None, psi=None):
    kind = spec["kind"]
    if kind == "basis":
        return SV.basis_state(n, spec["bits"])
    if kind == "dense":
        return np.asarray(spec["amps"], dtype=np.complex128).copy()
    if kind == "ideal":
        # v = U |psi>: the noiseless circuit applied to psi
        s = psi.copy()
        for name, qs, ps in circuit.gates:
            s = SV.apply_op(s, n, qs, G.gate_matrix(name, ps))
        return s
    raise ValueError(kind)


def final_density_matrix(circuit, psi_vec):
    n = circuit.n
    rho = np.outer(psi_vec, psi_vec.conj())
    for kind, idx in IR.events(circuit):
        if kind == "gate":
            name, qs, ps = circuit.gates[idx]
            u = G.gate_matrix(name, ps)
            rho = _left_right(rho, n, qs, u, u)
        else:
            _, q, spec = circuit.noises[idx]
            if isinstance(spec, IR.SuperOp):
                rho = apply_superop(rho, n, IR.site_qubits(q), spec.m)
            else:
                rho = apply_channel(rho, n, IR.site_qubits(q), spec)
    return rho


def matrix_element(circuit, psi_spec, x_spec, y_spec):
    """<x| E(|psi><psi|) |y>, one element of the output density matrix
    (Sec. III: every element can be estimated on its own)."""
    n = circuit.n
    if n > 12:
        raise ValueError("density-matrix oracle limited to n <= 12")
    psi = state_from_spec(psi_spec, n)
    x = state_from_spec(x_spec, n, circuit, psi)
    y = state_from_spec(y_spec, n, circuit, psi)
    rho = final_density_matrix(circuit, psi)
    return complex(np.vdot(x, rho @ y))


def fidelity(circuit, psi_spec, v_spec):
    """Exact F = <v| E(|psi><psi|) |v> (Problem 1)."""
    n = circuit.n
    if n > 12:
        raise ValueError("density-matrix oracle limited to n <= 12")
    psi = state_from_spec(psi_spec, n)
    v = state_from_spec(v_spec, n, circuit, psi)
    rho = final_density_matrix(circuit, psi)
    return complex(np.vdot(v, rho @ v))
