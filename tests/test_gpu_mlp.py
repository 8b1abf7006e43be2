"""Proposal-network kernels (bf16 weights, fp32 accumulation) against the FP64
oracle: forward outputs, loss and gradients; training lowers the loss."""

import numpy as np
import pytest

from oracle import mlp as OM

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup():
    import torch
    from paper_2211_17028_gb300 import nqs
    torch.cuda.set_device(0)
    nqs.use_torch_allocator()
    yield


def _data(rng, B, n_in):
    import torch
    X = rng.normal(size=(B, n_in)).astype(np.float32)
    y = (np.sin(X[:, 0]) + 0.5 * X[:, 1] * X[:, 2 % n_in]).astype(np.float32)
    return X, y, torch.tensor(X, device="cuda"), torch.tensor(y, device="cuda")


def test_forward_loss_and_gradient_match_oracle():
    import torch
    from paper_2211_17028_gb300 import nqs
    rng = np.random.default_rng(1)
    n_in, hidden, layers = 8, 256, 3
    m = nqs.nqs_mlp_create(n_in, hidden, layers, seed=11)
    dims = [n_in] + [hidden] * layers + [1]
    params = nqs.nqs_mlp_get_params(m)
    assert params.size == sum(a * b + b for a, b in zip(dims[:-1], dims[1:]))
    X, y, Xd, yd = _data(rng, 96, n_in)
    out = torch.zeros(96, device="cuda")
    nqs.nqs_mlp_forward(m, Xd, out)
    want = OM.forward(params, dims, X)[-1][:, 0]
    got = out.cpu().numpy()
    assert np.allclose(got, want, rtol=1e-4, atol=1e-5 * np.abs(want).max())
    loss, g = nqs.nqs_mlp_loss_grad(m, Xd, yd)
    lo, go = OM.loss_and_grad(params, dims, X, y)
    assert abs(loss - lo) <= 1e-5 * lo
    scale = np.abs(go).max()
    assert np.allclose(g, go, rtol=1e-3, atol=1e-4 * scale), float(np.abs(g - go).max() / scale)
    nqs.nqs_mlp_destroy(m)


def test_training_lowers_the_loss():
    from paper_2211_17028_gb300 import nqs
    rng = np.random.default_rng(2)
    m = nqs.nqs_mlp_create(8, 256, 3, seed=3)
    X, y, Xd, yd = _data(rng, 4096, 8)
    l0, _ = nqs.nqs_mlp_loss_grad(m, Xd[:512], yd[:512])
    nqs.nqs_mlp_train(m, Xd, yd, batch=512, steps=400, lr=1e-3, seed=7)
    l1, _ = nqs.nqs_mlp_loss_grad(m, Xd[:512], yd[:512])
    assert l1 < 0.1 * l0, (l0, l1)
    nqs.nqs_mlp_destroy(m)
