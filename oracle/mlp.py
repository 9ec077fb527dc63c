"""FP64 oracle of the learned face-flux correction network.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The network (not part of arXiv 2302.09005; it is the learned correction the
build adds on top of the paper's Rusanov flux, Eq. 4): a multilayer
perceptron 16 -> 64 -> 64 -> 4 with GELU activations,
    z1 = W1 x + b1, h1 = gelu(z1), z2 = W2 h1 + b2, h2 = gelu(z2),
    y  = W3 h2 + b3,
gelu(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2, and the mean squared error
loss L = mean((y - t)^2) over the batch and the 4 outputs.  Gradients are the
chain rule written out layer by layer (reverse mode).

Parameters are one flat vector in the order W1 (64x16, row-major: output
index major), b1 (64), W2 (64x64), b2 (64), W3 (4x64), b3 (4).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

N_IN, N_HID, N_OUT = 16, 64, 4
SHAPES = [("W1", (N_HID, N_IN)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
          ("W3", (N_OUT, N_HID)), ("b3", (N_OUT,))]
N_PARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta):
    """Flat parameter vector -> dict of arrays (views)."""
    theta = np.asarray(theta, dtype=np.float64)
    out, i = {}, 0
    for name, shape in SHAPES:
        k = int(np.prod(shape))
        out[name] = theta[i:i + k].reshape(shape)
        i += k
    return out


def pack(params) -> np.ndarray:
    return np.concatenate([np.asarray(params[name], dtype=np.float64).reshape(-1)
                           for name, _ in SHAPES])


def init_params(seed: int = 0) -> np.ndarray:
    """Seeded initial parameters: weights ~ N(0, 1/fan_in), biases 0, and the
    last layer scaled by 0.1 so the initial correction is small."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shape in SHAPES:
        if name.startswith("b"):
            p[name] = np.zeros(shape)
        else:
            p[name] = rng.standard_normal(shape) / math.sqrt(shape[1])
    p["W3"] *= 0.1
    return pack(p)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_prime(z):
    """d gelu / dz = Phi(z) + z phi(z)."""
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2 * math.pi)


def forward(theta, X):
    """X: (B, 16).  Returns (y (B, 4), cache)."""
    p = unpack(theta)
    z1 = X @ p["W1"].T + p["b1"]
    h1 = gelu(z1)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = gelu(z2)
    y = h2 @ p["W3"].T + p["b3"]
    return y, (X, z1, h1, z2, h2)


def loss_and_grad(theta, X, T):
    """Mean squared error over the batch and outputs, and its gradient with
    respect to the flat parameter vector (reverse mode)."""
    p = unpack(theta)
    y, (X, z1, h1, z2, h2) = forward(theta, X)
    B = X.shape[0]
    r = y - T
    loss = float(np.mean(r * r))
    dy = 2.0 * r / (B * N_OUT)
    g = {"W3": dy.T @ h2, "b3": dy.sum(0)}
    dh2 = dy @ p["W3"]
    dz2 = dh2 * gelu_prime(z2)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(0)
    dh1 = dz2 @ p["W2"]
    dz1 = dh1 * gelu_prime(z1)
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(0)
    return loss, pack(g)


def adam_step(theta, grad, m, v, step: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1) on flat vectors;
    step counts from 1.  Returns (theta, m, v)."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mhat = m / (1 - beta1 ** step)
    vhat = v / (1 - beta2 ** step)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


def bf16_round(a) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    a32 = np.asarray(a, dtype=np.float32)
    b = a32.view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    b = (b + 0x7FFF + lsb) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)
