"""Plain float64 multilayer perceptron: forward, backward, Adam (oracle).

The learned parameter predictor is a project extension (the paper chooses a,
K and n by hand, Sec. III). Its network is a stack of affine layers with ReLU
between them and a linear output; the loss is half the mean squared error
over the batch and the outputs:

    z_l = W_l a_{l-1} + b_l,   a_l = relu(z_l) (hidden),   y = z_L
    loss = sum_{batch, out} (y - t)^2 / (2 B)

Backward pass by the chain rule; Adam as published by Kingma & Ba (2015):
m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2, theta <- theta - lr mhat /
(sqrt(vhat) + eps) with mhat = m / (1 - b1^t), vhat = v / (1 - b2^t).

Weights are stored as W_l with shape (out, in), row-major, like the CUDA side.
The analytic gradient is pinned against central finite differences in the
tests.
"""

from __future__ import annotations

import numpy as np


def init(sizes, seed: int = 0):
    """He-uniform weights and zero biases for layer sizes [n_in, h, ..., n_out]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    params = []
    for fan_in, fan_out in zip(sizes[:-1], sizes[1:]):
        lim = np.sqrt(6.0 / fan_in)
        params.append((rng.uniform(-lim, lim, size=(fan_out, fan_in)), np.zeros(fan_out)))
    return params


def forward(params, x):
    """Returns (y, cache). x has shape (B, n_in)."""
    a = np.asarray(x, dtype=np.float64)
    cache = [a]
    L = len(params)
    for l, (W, b) in enumerate(params):
        z = a @ W.T + b
        a = np.maximum(z, 0.0) if l < L - 1 else z
        cache.append(z)
        if l < L - 1:
            cache.append(a)
    return a, cache


def loss(params, x, t):
    y, _ = forward(params, x)
    return float(((y - t) ** 2).sum() / (2.0 * len(x)))


def backward(params, x, t):
    """Gradients [(dW, db), ...] of the loss, and the loss."""
    y, cache = forward(params, x)
    B = len(x)
    L = len(params)
    acts = [cache[0]] + [cache[2 * l + 2] for l in range(L - 1)]   # inputs to each layer
    zs = [cache[2 * l + 1] for l in range(L)]
    delta = (y - t) / B                                          # d loss / d z_L
    grads = [None] * L
    for l in reversed(range(L)):
        W, _ = params[l]
        grads[l] = (delta.T @ acts[l], delta.sum(axis=0))
        if l > 0:
            delta = (delta @ W) * (zs[l - 1] > 0.0)
    return grads, float(((y - t) ** 2).sum() / (2.0 * B))


def adam_step(params, grads, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update in place; state = {'t': int, 'm': [...], 'v': [...]}."""
    if not state:
        state.update(t=0, m=[(np.zeros_like(W), np.zeros_like(b)) for W, b in params],
                     v=[(np.zeros_like(W), np.zeros_like(b)) for W, b in params])
    state["t"] += 1
    t = state["t"]
    new = []
    for l, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
        out = []
        for i, (p, g) in enumerate(((W, gW), (b, gb))):
            m = b1 * state["m"][l][i] + (1 - b1) * g
            v = b2 * state["v"][l][i] + (1 - b2) * g * g
            state["m"][l] = tuple(m if j == i else state["m"][l][j] for j in range(2))
            state["v"][l] = tuple(v if j == i else state["v"][l][j] for j in range(2))
            mh = m / (1 - b1 ** t)
            vh = v / (1 - b2 ** t)
            out.append(p - lr * mh / (np.sqrt(vh) + eps))
        new.append((out[0], out[1]))
    params[:] = new
    return params


def flatten(params):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in params])


def unflatten(vec, sizes):
    out, o = [], 0
    for fan_in, fan_out in zip(sizes[:-1], sizes[1:]):
        W = vec[o:o + fan_in * fan_out].reshape(fan_out, fan_in)
        o += fan_in * fan_out
        b = vec[o:o + fan_out]
        o += fan_out
        out.append((W.copy(), b.copy()))
    return out
