"""Kraus lists of the single-qubit noise channels used by the synthetic workloads.

These are problem inputs (the channel a user hands to the simulator), written
from their textbook definitions:

* depolarizing in the paper's form (Sec. II and Sec. IV): Kraus operators
  sqrt(1-p) I, sqrt(p/3) X, sqrt(p/3) Y, sqrt(p/3) Z, i.e.
  rho -> (1-p) rho + p/3 (X rho X + Y rho Y + Z rho Z);
* depolarizing in the "mix towards I/2" form rho -> (1-p) rho + p I/2, which is
  the paper form with p' = 3p/4 (kept separate and labelled, never mixed up);
* amplitude damping with decay probability gamma (T1 noise);
* phase damping with parameter lambda (T2 noise);
* compositions of the above, and seeded random CPTP channels.

Every function returns a list of 2x2 complex128 numpy arrays.
"""

import numpy as np

_I = np.eye(2, dtype=np.complex128)
_X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
_Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
_Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)


def depolarizing_paper(p: float) -> list:
    """rho -> (1-p) rho + p/3 (X rho X + Y rho Y + Z rho Z)."""
    if not 0.0 <= p <= 1.0:
        raise ValueError("p must lie in [0, 1]")
    a = np.sqrt(1.0 - p)
    b = np.sqrt(p / 3.0)
    return [a * _I, b * _X, b * _Y, b * _Z]


def depolarizing_mixing(p: float) -> list:
    """rho -> (1-p) rho + p I/2; equal to depolarizing_paper(3p/4)."""
    return depolarizing_paper(0.75 * p)


def amplitude_damping(gamma: float) -> list:
    if not 0.0 <= gamma <= 1.0:
        raise ValueError("gamma must lie in [0, 1]")
    e0 = np.array([[1, 0], [0, np.sqrt(1.0 - gamma)]], dtype=np.complex128)
    e1 = np.array([[0, np.sqrt(gamma)], [0, 0]], dtype=np.complex128)
    return [e0, e1]


def phase_damping(lam: float) -> list:
    if not 0.0 <= lam <= 1.0:
        raise ValueError("lambda must lie in [0, 1]")
    e0 = np.array([[1, 0], [0, np.sqrt(1.0 - lam)]], dtype=np.complex128)
    e1 = np.array([[0, 0], [0, np.sqrt(lam)]], dtype=np.complex128)
    return [e0, e1]


def compose(after: list, before: list) -> list:
    """Kraus list of the channel 'after o before' (before acts first).

    Products that are exactly the zero matrix are dropped.
    """
    out = []
    for a in after:
        for b in before:
            m = a @ b
            if np.any(m != 0):
                out.append(m)
    return out


def ad_pd(gamma: float, lam: float) -> list:
    """Phase damping applied after amplitude damping (the two commute)."""
    return compose(phase_damping(lam), amplitude_damping(gamma))


def random_channel(rng, n_kraus: int) -> list:
    """Seeded random CPTP channel: blocks of a random 2k x 2 isometry."""
    g = np.empty((2 * n_kraus, 2), dtype=np.complex128)
    for i in range(2 * n_kraus):
        for j in range(2):
            g[i, j] = _gauss(rng) + 1j * _gauss(rng)
    q, r = np.linalg.qr(g)
    # fix the QR phase freedom so the result depends only on the seed
    d = np.diag(r)
    q = q * (d / np.abs(d))[None, :]
    return [q[2 * k:2 * k + 2, :].copy() for k in range(n_kraus)]


def near_identity_channel(rng, eps: float, n_kraus: int = 2) -> list:
    """(1-eps) identity channel mixed with eps of a random channel."""
    rest = random_channel(rng, n_kraus)
    return [np.sqrt(1.0 - eps) * _I] + [np.sqrt(eps) * e for e in rest]


def depolarizing2(p: float) -> list:
    """Two-qubit depolarizing: rho -> (1-p) rho + p/15 sum_{P != II} P rho P,
    P over the two-qubit Paulis; 4x4 Kraus operators indexed 2*b(q0) + b(q1)."""
    if not 0.0 <= p <= 1.0:
        raise ValueError("p must lie in [0, 1]")
    paulis = [_I, _X, _Y, _Z]
    out = [np.sqrt(1.0 - p) * np.kron(_I, _I)]
    for a in range(4):
        for b in range(4):
            if a or b:
                out.append(np.sqrt(p / 15.0) * np.kron(paulis[a], paulis[b]))
    return out


def random_channel2(rng, n_kraus: int) -> list:
    """Seeded random two-qubit CPTP channel: blocks of a random 4k x 4 isometry."""
    g = np.empty((4 * n_kraus, 4), dtype=np.complex128)
    for i in range(4 * n_kraus):
        for j in range(4):
            g[i, j] = _gauss(rng) + 1j * _gauss(rng)
    q, r = np.linalg.qr(g)
    d = np.diag(r)
    q = q * (d / np.abs(d))[None, :]
    return [q[4 * k:4 * k + 4, :].copy() for k in range(n_kraus)]


def near_identity_channel2(rng, eps: float, n_kraus: int = 2) -> list:
    """(1-eps) two-qubit identity channel mixed with eps of a random one."""
    rest = random_channel2(rng, n_kraus)
    return [np.sqrt(1.0 - eps) * np.eye(4, dtype=np.complex128)] + [np.sqrt(eps) * e for e in rest]


def matrix_of(kraus: list) -> np.ndarray:
    """M = sum_k E_k (x) E_k^* (the input form of a noise given as a superoperator)."""
    return sum(np.kron(e, e.conj()) for e in kraus)


def perturbed_superop(rng, kraus: list, eps: float) -> np.ndarray:
    """The matrix of a channel plus eps times a seeded random complex matrix:
    a linear map on density matrices that is in general neither completely
    positive nor Hermiticity preserving (its tensor-permuted matrix is not
    positive semidefinite, so the two factor sets of the SVD differ)."""
    m = matrix_of(kraus)
    d = m.shape[0]
    r = np.array([[_gauss(rng) + 1j * _gauss(rng) for _ in range(d)] for _ in range(d)])
    return m + eps * r


def _gauss(rng) -> float:
    # Box-Muller from two uniforms of the seeded generator
    u1 = max(rng.uniform(), 1e-300)
    u2 = rng.uniform()
    return float(np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2))


def gauss(rng) -> float:
    return _gauss(rng)
