"""Float64 reference of the learned surrogate network (test infrastructure).

The network has no counterpart in the paper: it is the learned p -> y(p) map
that predicts the coefficient vector of Alg. 1 step 4, and whose predictions
are accepted only when the subsampled residual ||M(p) y - b_J|| / ||b_J||
(Sec. 4.3.1) passes a threshold.  Architecture: d_in -> 256 -> 256 -> r with
the exact GELU, x * Phi(x) = 0.5 x (1 + erf(x / sqrt 2)), after each hidden
layer and a linear output.  Loss: mean over batch and components of the
squared error.  Optimiser: Adam with bias correction.

The device kernels compute with bfloat16 weights and float32 accumulation;
the checks feed this float64 code the same (rounded) weights.  Gradients here
are pinned by central finite differences (tests/test_oracle_mlp.py); the
place of the network in the method is not from the paper.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

SQRT2 = np.sqrt(2.0)
INV_SQRT_2PI = 1.0 / np.sqrt(2.0 * np.pi)


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / SQRT2))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / SQRT2)) + x * np.exp(-0.5 * x * x) * INV_SQRT_2PI


def forward(params, X):
    """params = [(W1, b1), (W2, b2), (W3, b3)] with W_l of shape (out, in).

    Returns the output and the cache of pre-activations and activations.
    """
    H = X
    cache = [(None, X)]
    for li, (W, b) in enumerate(params):
        Z = H @ W.T + b
        H = gelu(Z) if li < len(params) - 1 else Z
        cache.append((Z, H))
    return H, cache


def loss_and_grads(params, X, Y):
    """Mean squared error over batch and components, and its gradients."""
    out, cache = forward(params, X)
    B, r = Y.shape
    diff = out - Y
    loss = float((diff * diff).sum() / (B * r))
    dH = 2.0 * diff / (B * r)
    grads = [None] * len(params)
    for li in range(len(params) - 1, -1, -1):
        Z, H = cache[li + 1]
        dZ = dH if li == len(params) - 1 else dH * gelu_grad(Z)
        Hprev = cache[li][1]
        W, _ = params[li]
        grads[li] = (dZ.T @ Hprev, dZ.sum(axis=0))
        dH = dZ @ W
    return loss, grads


def adam_step(params, grads, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update in place; state = {"t": int, "m": [...], "v": [...]}."""
    state["t"] += 1
    t = state["t"]
    new = []
    for li, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
        out = []
        for k, (p, g) in enumerate(((W, gW), (b, gb))):
            m = state["m"][2 * li + k] = beta1 * state["m"][2 * li + k] + (1 - beta1) * g
            v = state["v"][2 * li + k] = beta2 * state["v"][2 * li + k] + (1 - beta2) * g * g
            mh = m / (1 - beta1 ** t)
            vh = v / (1 - beta2 ** t)
            out.append(p - lr * mh / (np.sqrt(vh) + eps))
        new.append(tuple(out))
    return new


def adam_init(params):
    zeros = []
    for W, b in params:
        zeros += [np.zeros_like(W), np.zeros_like(b)]
    return {"t": 0, "m": [z.copy() for z in zeros], "v": [z.copy() for z in zeros]}
