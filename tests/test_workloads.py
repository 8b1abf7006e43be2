"""Seeded input generators: SplitMix64 test vectors and workload shapes."""

import numpy as np

import workloads as W
from workloads import channels as ch


def test_splitmix64_published_vectors():
    assert W.SplitMix64(0).next_u64() == 0xE220A8397B1DCDAF
    r = W.SplitMix64(1234567)
    assert [r.next_u64() for _ in range(3)] == [6457827717110365317, 3203168211198807973,
                                                9817491932198370423]


def test_channels_are_trace_preserving():
    rng = W.SplitMix64(3)
    for k in [ch.depolarizing_paper(0.1), ch.depolarizing_mixing(0.3), ch.amplitude_damping(0.2),
              ch.phase_damping(0.4), ch.ad_pd(0.1, 0.2), ch.random_channel(rng, 3),
              ch.near_identity_channel(rng, 0.05, 2)]:
        assert np.allclose(sum(e.conj().T @ e for e in k), np.eye(2), atol=1e-14)


def test_config_shapes():
    c1, c2, c3 = W.c1_line6(), W.c2_grid20(), W.c3_qaoa30()
    assert (c1.n, len(c1.gates), c1.n_noise) == (6, 68, 4)
    assert (c2.n, len(c2.gates), c2.n_noise) == (20, 444, 20)
    assert (c3.n, len(c3.gates), c3.n_noise) == (30, 690, 20)
    assert sum(1 for g in c2.gates if g[0] == "cz") == 124
    edges = c3.meta["edges"]
    deg = [0] * 30
    for a, b in edges:
        deg[a] += 1
        deg[b] += 1
    assert len(edges) == 45 and set(deg) == {3} and len(set(edges)) == 45
    c5, tw = W.c5_grid(), W.c5_twin()
    assert (c5.n, c5.n_noise, tw.n, tw.n_noise) == (28, 200, 20, 200)
    for a, b in zip(c5.noises, tw.noises):
        ra, ca = divmod(a.qubit, 7)
        rb, cb = divmod(b.qubit, 5)
        assert (ra, ca) == (rb, cb) and a.label == b.label


def test_generators_are_deterministic():
    assert W.to_ir_text(W.c2_grid20()) == W.to_ir_text(W.c2_grid20())
    b = W.c4_circuit(17)
    assert 12 <= b.n <= 24 and 5 <= b.n_noise <= 40 and b.levels[0] in (1, 2)
