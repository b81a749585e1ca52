"""Reference for the run-time / memory predictor: the MLP 8 -> 64 -> 64 -> 2
(ReLU) in numpy float64, written from its definition (test infrastructure).

Parameters are one flat vector: W1[64][8] b1[64] W2[64][64] b2[64] W3[2][64]
b3[2].  Loss L = 1/(2B) sum_b sum_o (y_bo - t_bo)^2.  ``grad`` is analytic
backpropagation (the chain rule layer by layer); ``numgrad`` is the central
finite difference that pins it.
"""
from __future__ import annotations

import numpy as np

IN, HID, OUT = 8, 64, 2
SHAPES = [("W1", (HID, IN)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)),
          ("W3", (OUT, HID)), ("b3", (OUT,))]
NPARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta: np.ndarray) -> dict:
    out, k = {}, 0
    for name, shape in SHAPES:
        size = int(np.prod(shape))
        out[name] = theta[k:k + size].reshape(shape)
        k += size
    return out


def forward(theta: np.ndarray, X: np.ndarray):
    p = unpack(np.asarray(theta, dtype=np.float64))
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ p["W1"].T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ p["W3"].T + p["b3"]
    return y, (X, z1, h1, z2, h2)


def loss(theta, X, T) -> float:
    y, _ = forward(theta, X)
    return float(((y - T) ** 2).sum() / (2 * len(X)))


def grad(theta, X, T) -> np.ndarray:
    p = unpack(np.asarray(theta, dtype=np.float64))
    y, (X, z1, h1, z2, h2) = forward(theta, X)
    B = len(X)
    dy = (y - np.asarray(T, dtype=np.float64)) / B
    g = {"W3": dy.T @ h2, "b3": dy.sum(0)}
    dz2 = (dy @ p["W3"]) * (z2 > 0)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(0)
    dz1 = (dz2 @ p["W2"]) * (z1 > 0)
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(0)
    return np.concatenate([g[name].ravel() for name, _ in SHAPES])


def numgrad(theta, X, T, idx, h: float = 1e-6) -> np.ndarray:
    theta = np.asarray(theta, dtype=np.float64)
    out = np.empty(len(idx))
    for j, k in enumerate(idx):
        e = np.zeros_like(theta)
        e[k] = h
        out[j] = (loss(theta + e, X, T) - loss(theta - e, X, T)) / (2 * h)
    return out


def adam_step(theta, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8, wd=0.0):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return theta - lr * (mh / (np.sqrt(vh) + eps) + wd * theta), m, v
