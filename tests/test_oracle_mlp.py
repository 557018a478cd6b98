"""Pins for the MLP oracle: finite differences, a closed-form tiny network, Adam's first step."""

import numpy as np

from oracle import mlp as M


def test_gradient_matches_central_differences():
    sizes = [5, 7, 6, 3]
    params = M.init(sizes, seed=1)
    rng = np.random.default_rng(0)
    x = rng.standard_normal((9, 5))
    t = rng.standard_normal((9, 3))
    grads, _ = M.backward(params, x, t)
    g = M.flatten([(gw, gb) for gw, gb in grads])
    theta = M.flatten(params)
    h = 1e-6
    num = np.zeros_like(theta)
    for i in range(len(theta)):
        tp = theta.copy(); tp[i] += h
        tm = theta.copy(); tm[i] -= h
        num[i] = (M.loss(M.unflatten(tp, sizes), x, t) - M.loss(M.unflatten(tm, sizes), x, t)) / (2 * h)
    assert np.abs(g - num).max() < 1e-7 * max(1.0, np.abs(num).max())


def test_closed_form_tiny_network():
    # 1 -> 2 -> 1: y = w2 . relu(w1 x + b1) + b2
    params = [(np.array([[2.0], [-1.0]]), np.array([0.5, 0.25])), (np.array([[3.0, 4.0]]), np.array([-1.0]))]
    x = np.array([[1.0], [-2.0]])
    y, _ = M.forward(params, x)
    # x=1: h = relu(2.5, -0.75) = (2.5, 0) -> 7.5 - 1 = 6.5 ; x=-2: h = relu(-3.5, 2.25) -> 9 - 1 = 8
    assert np.allclose(y.ravel(), [6.5, 8.0])
    grads, L = M.backward(params, x, np.array([[6.0], [8.0]]))
    assert abs(L - 0.25 / 4) < 1e-15                       # ((0.5)^2 + 0) / (2*2)
    assert np.allclose(grads[1][1], [0.25])                # d/db2 = mean residual = 0.5/2


def test_adam_first_step_moves_by_lr():
    params = [(np.array([[1.0, -2.0]]), np.array([0.5]))]
    grads = [(np.array([[0.3, -4.0]]), np.array([1e-3]))]
    state = {}
    M.adam_step(params, grads, state, lr=0.01)
    # first step: mhat = g, vhat = g^2 -> update = lr * sign(g) (up to eps)
    assert np.allclose(params[0][0], [[0.99, -1.99]], atol=1e-7)
    assert np.allclose(params[0][1], [0.49], atol=1e-6)
