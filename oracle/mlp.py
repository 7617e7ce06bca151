"""Float64 reference of the learned CDF predictor (test infrastructure only).

The paper has no learned model; this follows the predictor the library
implements: a 1 -> 32 -> 32 -> 1 ReLU network on the normalised query
u = (z - X_0) / (X_N - X_0), trained by mean squared error against i / N and
updated with Adam (Kingma & Ba, "Adam: A Method for Stochastic Optimization",
ICLR 2015, Algorithm 1).

Flat parameter layout (1153 values):
    W1[32] | b1[32] | W2[32][32] (row = output unit) | b2[32] | w3[32] | b3[1]
ReLU'(a) is taken as 1 for a > 0 and 0 otherwise (also at a == 0).
"""
import numpy as np

HID = 32
N_PARAMS = HID + HID + HID * HID + HID + HID + 1

ADAM_B1 = 0.9
ADAM_B2 = 0.999
ADAM_EPS = 1e-8


def unpack(theta):
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.shape == (N_PARAMS,)
    o = 0
    W1 = theta[o:o + HID]; o += HID
    b1 = theta[o:o + HID]; o += HID
    W2 = theta[o:o + HID * HID].reshape(HID, HID); o += HID * HID
    b2 = theta[o:o + HID]; o += HID
    w3 = theta[o:o + HID]; o += HID
    b3 = theta[o]
    return W1, b1, W2, b2, w3, b3


def pack(W1, b1, W2, b2, w3, b3):
    return np.concatenate([W1, b1, W2.reshape(-1), b2, w3, np.array([b3], dtype=np.float64)])


def forward(theta, u):
    """Network output for each input u (float64)."""
    W1, b1, W2, b2, w3, b3 = unpack(theta)
    u = np.asarray(u, dtype=np.float64)
    h1 = np.maximum(np.outer(u, W1) + b1, 0.0)
    h2 = np.maximum(h1 @ W2.T + b2, 0.0)
    return h2 @ w3 + b3


def loss_and_grad(theta, u, y):
    """Mean squared error over the batch and its gradient (reverse mode)."""
    W1, b1, W2, b2, w3, b3 = unpack(theta)
    u = np.asarray(u, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    B = u.shape[0]
    a1 = np.outer(u, W1) + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0.0)
    out = h2 @ w3 + b3
    r = out - y
    loss = float(np.mean(r * r))
    d_out = 2.0 * r / B
    g_w3 = h2.T @ d_out
    g_b3 = float(np.sum(d_out))
    d_a2 = np.outer(d_out, w3) * (a2 > 0.0)
    g_W2 = d_a2.T @ h1
    g_b2 = np.sum(d_a2, axis=0)
    d_a1 = (d_a2 @ W2) * (a1 > 0.0)
    g_W1 = d_a1.T @ u
    g_b1 = np.sum(d_a1, axis=0)
    return loss, pack(g_W1, g_b1, g_W2, g_b2, g_w3, g_b3)


def loss_only(theta, u, y):
    r = forward(theta, u) - np.asarray(y, dtype=np.float64)
    return float(np.mean(r * r))


def adam_step(theta, m, v, g, t, lr):
    """One Adam update at step t (1-based).  Returns new (theta, m, v)."""
    m = ADAM_B1 * m + (1.0 - ADAM_B1) * g
    v = ADAM_B2 * v + (1.0 - ADAM_B2) * g * g
    mhat = m / (1.0 - ADAM_B1 ** t)
    vhat = v / (1.0 - ADAM_B2 ** t)
    theta = theta - lr * mhat / (np.sqrt(vhat) + ADAM_EPS)
    return theta, m, v
