"""FP64 reference of the cost-model MLP.  TEST INFRASTRUCTURE ONLY.

Network: x (16) -> dense 64 -> ReLU -> dense 64 -> ReLU -> dense 64 -> ReLU -> dense 1, trained on
the mean squared error 1/B * sum_b (y_b - t_b)^2 with Adam (Kingma & Ba, 2015: m = b1 m + (1-b1) g,
v = b2 v + (1-b2) g^2, p -= lr * (m / (1 - b1^s)) / (sqrt(v / (1 - b2^s)) + eps)).

Parameter vector order (shared with the library's flat parameter buffer): for each layer l = 1..4,
the weight matrix W_l (out x in, row-major) followed by its bias b_l.
"""
from __future__ import annotations

import numpy as np

SIZES = (16, 64, 64, 64, 1)


def n_params(sizes=SIZES) -> int:
    return sum(sizes[i + 1] * sizes[i] + sizes[i + 1] for i in range(len(sizes) - 1))


def unpack(theta: np.ndarray, sizes=SIZES):
    layers, o = [], 0
    for i in range(len(sizes) - 1):
        fin, fout = sizes[i], sizes[i + 1]
        W = theta[o:o + fout * fin].reshape(fout, fin)
        o += fout * fin
        b = theta[o:o + fout]
        o += fout
        layers.append((W, b))
    assert o == theta.size
    return layers


def forward(theta: np.ndarray, X: np.ndarray, sizes=SIZES):
    """Returns (predictions (B,), list of layer inputs, list of pre-activations)."""
    h = np.asarray(X, dtype=np.float64)
    inputs, pre = [], []
    layers = unpack(np.asarray(theta, dtype=np.float64), sizes)
    for li, (W, b) in enumerate(layers):
        inputs.append(h)
        z = h @ W.T + b
        pre.append(z)
        h = np.maximum(z, 0.0) if li < len(layers) - 1 else z
    return h[:, 0], inputs, pre


def loss(theta, X, t, sizes=SIZES) -> float:
    y, _, _ = forward(theta, X, sizes)
    return float(np.mean((y - np.asarray(t, dtype=np.float64)) ** 2))


def gradient(theta, X, t, sizes=SIZES):
    """(loss, dloss/dtheta) by backpropagation, fp64."""
    y, inputs, pre = forward(theta, X, sizes)
    B = y.size
    layers = unpack(np.asarray(theta, dtype=np.float64), sizes)
    delta = (2.0 / B) * (y - np.asarray(t, dtype=np.float64))[:, None]   # dL/dz of the output layer
    grads = [None] * len(layers)
    for li in range(len(layers) - 1, -1, -1):
        W, _ = layers[li]
        grads[li] = (delta.T @ inputs[li], delta.sum(axis=0))
        if li > 0:
            delta = (delta @ W) * (pre[li - 1] > 0)
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return float(np.mean((y - t) ** 2)), flat


def adam_step(theta, m, v, g, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def finite_difference(theta, X, t, idx, h=1e-6, sizes=SIZES) -> np.ndarray:
    """Central differences of the loss along the coordinates `idx`."""
    out = np.zeros(len(idx))
    for n, i in enumerate(idx):
        tp = np.array(theta, dtype=np.float64)
        tm = np.array(theta, dtype=np.float64)
        tp[i] += h
        tm[i] -= h
        out[n] = (loss(tp, X, t, sizes) - loss(tm, X, t, sizes)) / (2 * h)
    return out
