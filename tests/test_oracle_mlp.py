"""Pins of the oracle's surrogate network: finite differences and closed forms."""
import numpy as np
from scipy.special import erf

from oracle import mlp


def small_net(rng, sizes=(4, 7, 6, 3)):
    params = []
    for a, b in zip(sizes[:-1], sizes[1:]):
        params.append((rng.standard_normal((b, a)) / np.sqrt(a), 0.1 * rng.standard_normal(b)))
    return params


def test_gelu_closed_forms():
    x = np.array([-3.0, -1.0, 0.0, 0.5, 2.0])
    # x * Phi(x) with Phi the standard normal CDF
    phi = 0.5 * (1.0 + erf(x / np.sqrt(2.0)))
    np.testing.assert_allclose(mlp.gelu(x), x * phi, rtol=1e-15)
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    # derivative against central differences
    h = 1e-6
    fd = (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h)
    np.testing.assert_allclose(mlp.gelu_grad(x), fd, rtol=1e-8, atol=1e-10)


def test_gradients_match_central_differences():
    rng = np.random.default_rng(0)
    params = small_net(rng)
    X = rng.standard_normal((5, 4))
    Y = rng.standard_normal((5, 3))
    loss, grads = mlp.loss_and_grads(params, X, Y)
    h = 1e-6
    for li in range(len(params)):
        for k in range(2):
            P = params[li][k]
            G = grads[li][k]
            it = np.nditer(P, flags=["multi_index"])
            for _ in it:
                idx = it.multi_index
                def f(delta):
                    pp = [tuple(a.copy() for a in layer) for layer in params]
                    pp[li][k][idx] += delta
                    return mlp.loss_and_grads(pp, X, Y)[0]
                fd = (f(h) - f(-h)) / (2 * h)
                assert abs(fd - G[idx]) <= 1e-7 * max(1.0, abs(fd)), (li, k, idx, fd, G[idx])


def test_adam_first_step_closed_form():
    """After one step with bias correction, each weight moves by lr * sign(g) (up to eps)."""
    rng = np.random.default_rng(1)
    params = small_net(rng)
    X = rng.standard_normal((8, 4))
    Y = rng.standard_normal((8, 3))
    _, grads = mlp.loss_and_grads(params, X, Y)
    state = mlp.adam_init(params)
    new = mlp.adam_step(params, grads, state, lr=1e-3)
    for (W, b), (W2, b2), (gW, gb) in zip(params, new, grads):
        np.testing.assert_allclose(W - W2, 1e-3 * gW / (np.abs(gW) + 1e-8), rtol=1e-12)
        np.testing.assert_allclose(b - b2, 1e-3 * gb / (np.abs(gb) + 1e-8), rtol=1e-12)


def test_linear_network_reduces_to_least_squares_gradient():
    """With one linear layer the gradient is the least-squares normal-equation residual."""
    rng = np.random.default_rng(2)
    W = rng.standard_normal((3, 4))
    b = rng.standard_normal(3)
    X = rng.standard_normal((10, 4))
    Y = rng.standard_normal((10, 3))
    loss, grads = mlp.loss_and_grads([(W, b)], X, Y)
    R = X @ W.T + b - Y
    np.testing.assert_allclose(grads[0][0], 2 * R.T @ X / 30, rtol=1e-13)
    np.testing.assert_allclose(loss, (R * R).sum() / 30, rtol=1e-13)
