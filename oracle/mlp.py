"""FP64 oracle of the boid-force surrogate -- TEST INFRASTRUCTURE ONLY.

The surrogate is not in the paper (it is the learned growth item of this
project): an MLP from a boid's local flow features to the fluid force the
SPH coupling puts on it (section "Boid Motion and Agent Fluid Interaction":
the force F_b that v_b += sph_factor dt F_b applies).

Network (rows = samples):
    x  in R^272  (256 stencil features, 3 boid-velocity features, 13 zeros)
    h1 = gelu(x  W1^T + b1)   W1: 256 x 272
    h2 = gelu(h1 W2^T + b2)   W2: 256 x 256
    h3 = gelu(h2 W3^T + b3)   W3: 256 x 256
    y  = h3 W4^T + b4         W4: 16 x 256; y[:, 0:3] = F / F_scale,
                              y[:, 3] = error head (log10 relative error)
gelu(z) = z/2 (1 + erf(z / sqrt 2)) (the exact form).
Force loss: mean over samples of 1/2 |y[:, :3] - t|^2.

Plain numpy in float64; matrix products use numpy's matmul.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

D_IN, D_H, D_OUT = 272, 256, 16
LAYERS = (("W1", "b1", D_H, D_IN), ("W2", "b2", D_H, D_H), ("W3", "b3", D_H, D_H), ("W4", "b4", D_OUT, D_H))


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    """d gelu / dz = Phi(z) + z phi(z)."""
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def init_params(seed: int = 0) -> dict:
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases."""
    rng = np.random.default_rng(seed)
    p = {}
    for w, b, n_out, n_in in LAYERS:
        lim = 1.0 / math.sqrt(n_in)
        p[w] = rng.uniform(-lim, lim, size=(n_out, n_in))
        p[b] = np.zeros(n_out)
    return p


def forward(p: dict, x: np.ndarray) -> dict:
    x = np.asarray(x, np.float64)
    c = {"x": x}
    h = x
    for k, (w, b, _, _) in enumerate(LAYERS, start=1):
        z = h @ p[w].T + p[b]
        c[f"z{k}"] = z
        h = gelu(z) if k < 4 else z
        c[f"h{k}"] = h
    c["y"] = h
    return c


def force_loss(y: np.ndarray, t: np.ndarray) -> float:
    d = y[:, :3] - t
    return 0.5 * float(np.sum(d * d)) / len(y)


def backward(p: dict, c: dict, dy: np.ndarray) -> dict:
    """Gradients of sum(dy * y) with respect to every weight and bias."""
    g = {}
    delta = np.asarray(dy, np.float64)
    for k in range(4, 0, -1):
        w, b, _, _ = LAYERS[k - 1]
        h_in = c["x"] if k == 1 else c[f"h{k - 1}"]
        g[w] = delta.T @ h_in
        g[b] = delta.sum(axis=0)
        if k > 1:
            delta = (delta @ p[w]) * gelu_grad(c[f"z{k - 1}"])
    return g


def force_loss_grad_y(y: np.ndarray, t: np.ndarray) -> np.ndarray:
    """d force_loss / d y (zero outside the three force columns)."""
    dy = np.zeros_like(y)
    dy[:, :3] = (y[:, :3] - t) / len(y)
    return dy


def error_loss_grad_y(y: np.ndarray, t: np.ndarray) -> np.ndarray:
    """d/dy of the error-head loss mean over samples of 1/2 (y[:, 3] - t)^2
    (zero outside column 3)."""
    dy = np.zeros_like(y)
    dy[:, 3] = (y[:, 3] - t) / len(y)
    return dy


def adam_update(w, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba): returns the new (w, m, v)."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v
