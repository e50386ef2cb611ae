"""Three-layer perceptron used as a learned PCG initial guess (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Not from the paper: the learned-guess pattern layered on the element PCG of
Section 7.1.  For an element's u_t system (S_c2 + w w^T) y = r_u the network
maps features x = [c^2 / mean(c^2) at the 81 nodes, r_u / ||r_u||] (162
numbers) to a guess of y / ||r_u|| (81 numbers); the system is linear, so the
guess is rescaled by ||r_u||.

  h1 = tanh(W1 x + b1)      W1: 64 x 162
  h2 = tanh(W2 h1 + b2)     W2: 64 x 64
  yhat = W3 h2 + b3         W3: 81 x 64
  loss = (1/B) sum_b ||yhat_b - y_b||^2

Plain FP64 forward and backward (chain rule written out), plus the
feature map.  The GPU kernels keep BF16 weights and accumulate in FP32; the
tests feed this oracle the same BF16-rounded weights.
"""
import numpy as np

SIZES = (162, 64, 64, 81)


def init_params(seed, sizes=SIZES):
    """Glorot-uniform weights, zero biases."""
    rng = np.random.default_rng(seed)
    params = []
    for fan_in, fan_out in zip(sizes[:-1], sizes[1:]):
        lim = np.sqrt(6.0 / (fan_in + fan_out))
        params.append(rng.uniform(-lim, lim, size=(fan_out, fan_in)))
        params.append(np.zeros(fan_out))
    return params


def features(c2, r):
    """x = [c2 / mean(c2), r / ||r||] per row; returns (x, ||r||)."""
    c2 = np.atleast_2d(c2)
    r = np.atleast_2d(r)
    nr = np.linalg.norm(r, axis=1)
    safe = np.where(nr > 0, nr, 1.0)
    x = np.concatenate([c2 / c2.mean(axis=1, keepdims=True), r / safe[:, None]], axis=1)
    return x, nr


def forward(params, x):
    """Returns yhat and the cache needed by backward."""
    W1, b1, W2, b2, W3, b3 = params
    z1 = x @ W1.T + b1
    h1 = np.tanh(z1)
    z2 = h1 @ W2.T + b2
    h2 = np.tanh(z2)
    yhat = h2 @ W3.T + b3
    return yhat, (x, h1, h2)


def loss(params, x, y):
    yhat, _ = forward(params, x)
    return np.sum((yhat - y) ** 2) / x.shape[0]


def backward(params, x, y):
    """Gradients of loss with respect to (W1, b1, W2, b2, W3, b3)."""
    W1, b1, W2, b2, W3, b3 = params
    yhat, (x, h1, h2) = forward(params, x)
    B = x.shape[0]
    g3 = 2.0 * (yhat - y) / B              # d loss / d yhat
    dW3 = g3.T @ h2
    db3 = g3.sum(axis=0)
    gh2 = g3 @ W3
    g2 = gh2 * (1.0 - h2 ** 2)             # tanh'
    dW2 = g2.T @ h1
    db2 = g2.sum(axis=0)
    gh1 = g2 @ W2
    g1 = gh1 * (1.0 - h1 ** 2)
    dW1 = g1.T @ x
    db1 = g1.sum(axis=0)
    return [dW1, db1, dW2, db2, dW3, db3]


def bf16_round(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    a32 = np.asarray(a, dtype=np.float32)
    bits = a32.view(np.uint32).astype(np.uint64)
    lsb = (bits >> 16) & 1
    bits = ((bits + 0x7FFF + lsb) >> 16) << 16
    return bits.astype(np.uint32).view(np.float32).astype(np.float64)
