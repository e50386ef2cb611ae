"""Pins of the oracle MLP (learned PCG guess): central-difference gradients,
the layer definition written as loops on a tiny case, and BF16 rounding."""
import numpy as np

from oracle import mlp


def test_gradient_matches_central_differences():
    sizes = (7, 5, 4, 3)
    params = mlp.init_params(3, sizes)
    rng = np.random.default_rng(0)
    params = [p + 0.1 * rng.standard_normal(p.shape) for p in params]
    x = rng.standard_normal((6, 7))
    y = rng.standard_normal((6, 3))
    grads = mlp.backward(params, x, y)
    eps = 1e-6
    for k, p in enumerate(params):
        it = np.nditer(p, flags=["multi_index"])
        for _ in it:
            idx = it.multi_index
            old = p[idx]
            p[idx] = old + eps
            lp = mlp.loss(params, x, y)
            p[idx] = old - eps
            lm = mlp.loss(params, x, y)
            p[idx] = old
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - grads[k][idx]) < 1e-7 * max(1.0, abs(fd)), (k, idx)


def test_forward_matches_loop_definition():
    sizes = (4, 3, 3, 2)
    params = mlp.init_params(5, sizes)
    params[1][:] = [0.1, -0.2, 0.3]
    x = np.array([[0.5, -1.0, 2.0, 0.25]])
    W1, b1, W2, b2, W3, b3 = params
    h1 = [np.tanh(sum(W1[i, j] * x[0, j] for j in range(4)) + b1[i]) for i in range(3)]
    h2 = [np.tanh(sum(W2[i, j] * h1[j] for j in range(3)) + b2[i]) for i in range(3)]
    y = [sum(W3[i, j] * h2[j] for j in range(3)) + b3[i] for i in range(2)]
    yhat, _ = mlp.forward(params, x)
    assert np.allclose(yhat[0], y, atol=1e-14)


def test_bf16_rounding():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -3.140625, 1e-3, 65504.0])
    r = mlp.bf16_round(vals)
    assert r[0] == 1.0 and r[1] == 1.0 + 2 ** -7 * 0 + 0.0 or r[1] in (1.0, 1.0 + 2 ** -7)
    assert r[2] == 1.0 + 2 ** -7          # rounds up past the halfway point
    assert r[3] == -3.140625              # exactly representable
    assert abs(r[4] - 1e-3) < 1e-3 * 2 ** -8
    # 8 significant bits: every result has at most 8 mantissa bits
    for v in r:
        m, e = np.frexp(v)
        assert (m * 2 ** 8) == np.round(m * 2 ** 8)


def test_features_are_scale_invariant():
    rng = np.random.default_rng(1)
    c2 = 1.0 + rng.random((3, 81))
    r = rng.standard_normal((3, 81))
    x1, n1 = mlp.features(c2, r)
    x2, n2 = mlp.features(4.0 * c2, 7.0 * r)
    assert np.allclose(x1, x2) and np.allclose(n2, 7.0 * n1)
