"""FP64 reference of the proposal network (oracle; test infrastructure only).

Forward: h_0 = x; h_l = relu(h_{l-1} W_l^T + b_l) for hidden layers; output
linear.  The weights are taken as the GPU uses them -- rounded to bfloat16
(round to nearest, ties to even, on the fp32 bit pattern) -- and everything
else is computed in FP64.  Loss = mean (pred - y)^2; the gradient is the
textbook backpropagation of that loss with respect to every W_l and b_l.
"""

import numpy as np


def to_bf16(w):
    """fp32 -> bfloat16 -> fp64, round to nearest even."""
    b = np.asarray(w, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    b = (b + 0x7FFF + lsb) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def unflatten(params, dims):
    out, off = [], 0
    for a, b in zip(dims[:-1], dims[1:]):
        W = np.asarray(params[off:off + a * b], dtype=np.float64).reshape(b, a)
        off += a * b
        bias = np.asarray(params[off:off + b], dtype=np.float64)
        off += b
        out.append((W, bias))
    assert off == len(params)
    return out


def forward(params, dims, X):
    layers = unflatten(params, dims)
    h = [np.asarray(X, dtype=np.float64)]
    for l, (W, b) in enumerate(layers):
        z = h[-1] @ to_bf16(W).T + b
        h.append(np.maximum(z, 0.0) if l + 1 < len(layers) else z)
    return h


def loss_and_grad(params, dims, X, y):
    layers = unflatten(params, dims)
    h = forward(params, dims, X)
    B = X.shape[0]
    pred = h[-1][:, 0]
    err = pred - np.asarray(y, dtype=np.float64)
    loss = float(np.mean(err ** 2))
    d = (2.0 * err / B)[:, None]
    grads = []
    for l in range(len(layers) - 1, -1, -1):
        W, b = layers[l]
        if l + 1 < len(layers):
            d = d * (h[l + 1] > 0)
        gW = d.T @ h[l]
        gb = d.sum(axis=0)
        grads.append((gW, gb))
        d = d @ to_bf16(W)
    grads.reverse()
    flat = []
    for gW, gb in grads:
        flat.append(gW.reshape(-1))
        flat.append(gb)
    return loss, np.concatenate(flat)
