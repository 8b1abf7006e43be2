"""Off-diagonal elements <x|rho|y> through the polarization identity
(nqs_offdiagonal, Sec. III): against the oracle's direct level-l evaluation
(both boundary vectors in one double-size network) and, at the full level,
against the density matrix element."""

import numpy as np
import pytest

import workloads as W
from oracle import density_matrix as DM
from oracle import expansion as OEX
from oracle import ir as OIR

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup():
    import torch
    from paper_2211_17028_gb300 import nqs
    torch.cuda.set_device(0)
    nqs.use_torch_allocator()
    yield


def _dense(amps):
    import torch
    return torch.tensor(np.asarray(amps, dtype=np.complex64), device="cuda")


@pytest.mark.parametrize("seed,n,level", [(71, 4, 1), (72, 6, 2), (73, 8, 1), (74, 5, 6)])
def test_offdiagonal_matches_oracle(seed, n, level):
    from paper_2211_17028_gb300 import nqs
    w = W.random_circuit(seed, n, 40, 6, rate_lo=5e-3, rate_hi=5e-2)
    c = OIR.parse(W.to_ir_text(w))
    rng = W.SplitMix64(seed)
    x_amps = W.circuits.random_dense_state(rng, n)
    x_spec = {"kind": "dense", "amps": x_amps}
    y_spec = {"kind": "basis", "bits": w.v["bits"]}
    want = OEX.approximate_offdiagonal(c, w.psi, x_spec, y_spec, level)["value"]
    xt = _dense(x_amps)
    circ = nqs.NoisyCircuit(W.to_ir_text(w))
    got, parts = nqs.nqs_offdiagonal(circ.h, nqs.basis(w.psi["bits"]), nqs.dense(xt), nqs.basis(w.v["bits"]), level)
    circ.close()
    scale = max(abs(p["F"]) for p in parts)
    assert all(p["status"] == 0 for p in parts)
    assert abs(got - want) <= 1e-5 * scale, (got, want, scale)
    if level >= w.n_noise and n <= 8:
        exact = DM.matrix_element(c, w.psi, x_spec, y_spec)
        assert abs(got - exact) <= 1e-5 * scale


def test_offdiagonal_hermitian_and_diagonal():
    from paper_2211_17028_gb300 import nqs
    w = W.random_circuit(75, 5, 30, 4, rate_lo=1e-2, rate_hi=5e-2)
    circ = nqs.NoisyCircuit(W.to_ir_text(w))
    psi = nqs.basis(w.psi["bits"])
    a, _ = nqs.nqs_offdiagonal(circ.h, psi, nqs.basis(3), nqs.basis(17), 2)
    b, _ = nqs.nqs_offdiagonal(circ.h, psi, nqs.basis(17), nqs.basis(3), 2)
    assert abs(a - b.conjugate()) <= 1e-6
    d, _ = nqs.nqs_offdiagonal(circ.h, psi, nqs.basis(3), nqs.basis(3), 2)
    f = circ.fidelity(psi, nqs.basis(3), 2)["F"]
    assert abs(d.real - f) <= 1e-5 * abs(f) + 1e-9 and abs(d.imag) <= 1e-6
    with pytest.raises(nqs.NqsError):
        nqs.nqs_offdiagonal(circ.h, psi, nqs.ideal(), nqs.basis(3), 1)
    circ.close()
