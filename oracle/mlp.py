"""CPU reference of the support-prediction network, in float64 (TEST INFRASTRUCTURE ONLY).

The network is 32 -> 64 -> 64 -> 1 with ReLU after the two hidden layers; inputs are
standardised, x' = (x - mean) / stdev; the loss is the mean squared error of the output against
the target (log MNI support).  Forward and backward are written from these definitions with
numpy matrix products as the only library step; the GPU kernels are checked against them.

Parameter vector layout (6337 values): W1[32][64] (input i, unit j), b1[64], W2[64][64], b2[64],
w3[64], b3.  ``bf16_round`` rounds float32 values to the nearest bfloat16 (ties to even), the
precision in which the GPU multiplies by the weights.
"""
from __future__ import annotations

import numpy as np

NIN, NH = 32, 64
SHAPES = [("W1", (NIN, NH)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)), ("w3", (NH,)), ("b3", (1,))]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta):
    theta = np.asarray(theta, dtype=np.float64)
    out, o = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = theta[o:o + n].reshape(shape)
        o += n
    return out


def pack(parts) -> np.ndarray:
    return np.concatenate([np.asarray(parts[name], np.float64).reshape(-1) for name, _ in SHAPES])


def bf16_round(x) -> np.ndarray:
    """Nearest bfloat16 value (round half to even) of each float32, returned as float64."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    r = ((b + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def gpu_weights(theta):
    """The weights the GPU multiplies with: W1, W2, w3 rounded to bfloat16, biases in FP32."""
    p = unpack(np.asarray(theta, np.float32).astype(np.float64))
    for name in ("W1", "W2", "w3"):
        p[name] = bf16_round(p[name])
    return p


def forward(p, X, mean, stdev):
    x = (np.asarray(X, np.float64) - np.asarray(mean, np.float64)) / np.asarray(stdev, np.float64)
    z1 = x @ p["W1"] + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"] + p["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ p["w3"] + p["b3"][0]
    return y, (x, z1, h1, z2, h2)


def loss_and_grad(p, X, Y, mean, stdev):
    """Mean squared error and its gradient with respect to every parameter (chain rule)."""
    y, (x, z1, h1, z2, h2) = forward(p, X, mean, stdev)
    n = len(y)
    e = y - np.asarray(Y, np.float64)
    loss = float(np.mean(e * e))
    dy = 2.0 * e / n
    g = {"w3": h2.T @ dy, "b3": np.array([dy.sum()])}
    dz2 = np.outer(dy, p["w3"]) * (z2 > 0)
    g["W2"] = h1.T @ dz2
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ p["W2"].T) * (z1 > 0)
    g["W1"] = x.T @ dz1
    g["b1"] = dz1.sum(axis=0)
    return loss, pack(g)


def adam_step(theta, m, v, g, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba 2015) with bias correction; returns new (theta, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
