"""Pins for the float64 learned-predictor reference (forward, gradient, Adam)
and for the float64 interpolation reference."""
import numpy as np

import oracle
from oracle import mlp


def _random_theta(g, scale=0.5):
    return g.normal(0, scale, mlp.N_PARAMS)


def test_gradient_matches_central_differences():
    g = np.random.default_rng(1)
    theta = _random_theta(g)
    u = g.uniform(0, 1, 64)
    y = g.uniform(0, 1, 64)
    _, grad = mlp.loss_and_grad(theta, u, y)
    h = 1e-6
    num = np.empty_like(theta)
    for k in range(theta.size):
        e = np.zeros_like(theta); e[k] = h
        num[k] = (mlp.loss_only(theta + e, u, y) - mlp.loss_only(theta - e, u, y)) / (2 * h)
    assert np.max(np.abs(num - grad)) <= 1e-7 * max(1.0, np.max(np.abs(grad)))


def test_forward_closed_form():
    # A net that computes 2*relu(u - 0.25) + 0.5 through one active path.
    W1 = np.zeros(32); b1 = np.zeros(32); W2 = np.zeros((32, 32)); b2 = np.zeros(32)
    w3 = np.zeros(32)
    W1[3], b1[3] = 1.0, -0.25
    W2[7, 3] = 2.0
    w3[7] = 1.0
    theta = mlp.pack(W1, b1, W2, b2, w3, 0.5)
    u = np.array([0.0, 0.25, 0.5, 1.0])
    assert np.allclose(mlp.forward(theta, u), [0.5, 0.5, 1.0, 2.0], rtol=0, atol=1e-15)
    loss, g = mlp.loss_and_grad(theta, u, np.zeros(4))
    assert np.isclose(loss, np.mean(np.array([0.5, 0.5, 1.0, 2.0]) ** 2))
    # only the active path and the output bias get gradient
    W1g, b1g, W2g, b2g, w3g, b3g = mlp.unpack(g)
    assert np.isclose(b3g, 2 * np.mean([0.5, 0.5, 1.0, 2.0]))
    assert np.count_nonzero(W2g) == 1 and W2g[7, 3] != 0


def test_adam_first_step_closed_form():
    # From zero moments the bias-corrected first step is -lr * g / (|g| + eps).
    g = np.random.default_rng(2)
    theta = _random_theta(g)
    grad = g.normal(size=theta.size)
    lr = 1e-3
    new, m, v = mlp.adam_step(theta, np.zeros_like(theta), np.zeros_like(theta), grad, 1, lr)
    assert np.allclose(new - theta, -lr * grad / (np.abs(grad) + mlp.ADAM_EPS), rtol=1e-12, atol=0)
    # a constant gradient keeps the bias-corrected moments at g and g^2
    t2, m, v = mlp.adam_step(new, m, v, grad, 2, lr)
    assert np.allclose(t2 - new, -lr * grad / (np.abs(grad) + mlp.ADAM_EPS), rtol=1e-9, atol=1e-15)


def test_interp_reference():
    g = np.random.default_rng(3)
    X = np.sort(g.uniform(-10, 10, 1000)).astype(np.float32)
    X = np.unique(X)
    Y = g.standard_normal(X.size).astype(np.float32)
    # at a knot the interpolant is exactly the knot value
    I, y = oracle.interp(X, Y, X[:-1])
    assert np.array_equal(I, np.arange(X.size - 1)) and np.array_equal(y, Y[:-1].astype(np.float64))
    # linear data is reproduced up to float64 rounding
    a, b = 0.75, -2.0
    Yl = (a * X.astype(np.float64) + b).astype(np.float32)
    Z = g.uniform(float(X[0]), float(X[-1]), 5000).astype(np.float32)
    I, y = oracle.interp(X, Yl, Z)
    yl0, yl1 = Yl[I].astype(np.float64), Yl[I + 1].astype(np.float64)
    t = (Z.astype(np.float64) - X[I]) / (X[I + 1].astype(np.float64) - X[I])
    assert np.all((t >= 0) & (t < 1))
    assert np.allclose(y, yl0 + (yl1 - yl0) * t, rtol=0, atol=1e-12)
    # midpoints give the mean of the two knot values
    Xd = np.array([0.0, 2.0, 4.0, 8.0], dtype=np.float32)
    Yd = np.array([1.0, 3.0, -1.0, 5.0], dtype=np.float32)
    I, y = oracle.interp(Xd, Yd, np.array([1.0, 3.0, 6.0], dtype=np.float32))
    assert list(I) == [0, 1, 2] and list(y) == [2.0, 1.0, 2.0]
