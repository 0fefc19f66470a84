"""FP64 reference of the learned cost model's network -- test infrastructure.

A three-layer perceptron y = W3 relu(W2 relu(W1 x + b1) + b2) + b3 (hidden
width H), trained on the mean squared error of log run time with Adam
(Kingma and Ba, 2015: m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2,
p <- p - lr * mhat / (sqrt(vhat) + eps), mhat = m / (1-b1^t),
vhat = v / (1-b2^t)).  Everything here is float64 numpy, written from those
definitions; the GPU kernels are checked against it.

Parameter layout (shared with the C ABI's flat parameter vector):
W1 [F x H], b1 [H], W2 [H x H], b2 [H], W3 [H], b3 [1], row-major, so that
layer l computes x @ W_l.
"""
from __future__ import annotations

import numpy as np


def param_shapes(F: int, H: int):
    return [("W1", (F, H)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H,)), ("b3", (1,))]


def num_params(F: int, H: int) -> int:
    return sum(int(np.prod(s)) for _, s in param_shapes(F, H))


def unpack(theta: np.ndarray, F: int, H: int) -> dict:
    out, at = {}, 0
    for name, shape in param_shapes(F, H):
        size = int(np.prod(shape))
        out[name] = theta[at:at + size].reshape(shape)
        at += size
    return out


def pack(p: dict, F: int, H: int) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in param_shapes(F, H)])


def forward(theta, x, F, H):
    p = unpack(np.asarray(theta, dtype=np.float64), F, H)
    x = np.asarray(x, dtype=np.float64)
    z1 = x @ p["W1"] + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"] + p["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ p["W3"] + p["b3"][0]
    return y, (x, z1, h1, z2, h2)


def loss(theta, x, t, F, H) -> float:
    y, _ = forward(theta, x, F, H)
    return float(np.mean((y - np.asarray(t, dtype=np.float64)) ** 2))


def gradient(theta, x, t, F, H, tau=0.5):
    """Backpropagation of the expectile loss mean(w (y - t)^2), w = 2 tau
    where y < t and 2 (1 - tau) elsewhere (tau = 0.5: the mean squared
    error); returns (loss, grad)."""
    p = unpack(np.asarray(theta, dtype=np.float64), F, H)
    y, (x, z1, h1, z2, h2) = forward(theta, x, F, H)
    B = x.shape[0]
    d = y - np.asarray(t, dtype=np.float64)
    w = np.where(d < 0, 2.0 * tau, 2.0 * (1.0 - tau))
    dy = 2.0 * w * d / B
    g = {}
    g["W3"] = h2.T @ dy
    g["b3"] = np.array([dy.sum()])
    dh2 = np.outer(dy, p["W3"]) * (z2 > 0)
    g["W2"] = h1.T @ dh2
    g["b2"] = dh2.sum(axis=0)
    dh1 = (dh2 @ p["W2"].T) * (z1 > 0)
    g["W1"] = x.T @ dh1
    g["b1"] = dh1.sum(axis=0)
    return float(np.mean(w * d ** 2)), pack(g, F, H)


class Adam:
    def __init__(self, n, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.m = np.zeros(n)
        self.v = np.zeros(n)
        self.t = 0
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps

    def step(self, theta, g):
        self.t += 1
        self.m = self.b1 * self.m + (1 - self.b1) * g
        self.v = self.b2 * self.v + (1 - self.b2) * g * g
        mhat = self.m / (1 - self.b1 ** self.t)
        vhat = self.v / (1 - self.b2 ** self.t)
        return theta - self.lr * mhat / (np.sqrt(vhat) + self.eps)


def init_params(F, H, seed=0):
    """He-uniform weights, zero biases (the initialisation the library uses
    is checked only through these shapes; values come from the library)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shape in param_shapes(F, H):
        if name.startswith("b"):
            p[name] = np.zeros(shape)
        else:
            fan_in = shape[0]
            lim = np.sqrt(6.0 / fan_in)
            p[name] = rng.uniform(-lim, lim, size=shape)
    return pack(p, F, H)
