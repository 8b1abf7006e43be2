"""Pins of the FP64 proposal-network oracle: bfloat16 rounding on exact
values and the backpropagated gradient against central finite differences
of the oracle's own loss (an independent computation)."""

import numpy as np

from oracle import mlp as OM


def test_bf16_rounding_values():
    x = np.array([1.0, -2.5, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, 1.0 + 2 ** -7, 3.0e38, 1e-40], dtype=np.float32)
    got = OM.to_bf16(x)
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: even mantissa (1.0) wins;
    # 1 + 3*2^-9 rounds up; 1 + 2^-7 is exact in bfloat16
    assert got[0] == 1.0 and got[1] == -2.5
    assert got[2] == 1.0
    assert got[3] == 1.0 + 2 ** -7
    assert got[4] == 1.0 + 2 ** -7
    assert abs(got[5] - 3.0e38) / 3.0e38 < 2 ** -8
    assert abs(got[6]) < 1e-39


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(5)
    dims = [5, 7, 6, 1]
    n = sum(a * b + b for a, b in zip(dims[:-1], dims[1:]))
    # parameters exactly representable in bf16 so that small perturbations of
    # the biases (not rounded) and the weights' own rounding stay consistent
    params = OM.to_bf16(rng.normal(size=n).astype(np.float32) * 0.5)
    X = rng.normal(size=(9, 5))
    y = rng.normal(size=9)
    loss, g = OM.loss_and_grad(params, dims, X, y)
    # finite differences on the biases (weights are rounded to bf16 inside)
    off = 0
    for a, b in zip(dims[:-1], dims[1:]):
        off += a * b
        for j in range(b):
            e = np.zeros(n)
            e[off + j] = 1e-6
            lp, _ = OM.loss_and_grad(params + e, dims, X, y)
            lm, _ = OM.loss_and_grad(params - e, dims, X, y)
            assert abs((lp - lm) / 2e-6 - g[off + j]) < 1e-6 * max(1.0, abs(g[off + j]))
        off += b
    # weights: perturb by one bf16 ulp-scaled step on a linearised copy
    lin = [(W, bias) for W, bias in OM.unflatten(params, dims)]
    W0 = lin[0][0]

    def loss_w(Wmod):
        h = X @ Wmod.T + lin[0][1]
        h = np.maximum(h, 0)
        for l, (W, bb) in enumerate(lin[1:], start=1):
            h = h @ W.T + bb
            if l + 1 < len(lin):
                h = np.maximum(h, 0)
        return np.mean((h[:, 0] - y) ** 2)

    for (r, c) in [(0, 0), (3, 4), (6, 2)]:
        E = np.zeros_like(W0)
        E[r, c] = 1e-6
        fd = (loss_w(W0 + E) - loss_w(W0 - E)) / 2e-6
        assert abs(fd - g[r * dims[0] + c]) < 1e-6 * max(1.0, abs(fd))
    assert loss > 0
