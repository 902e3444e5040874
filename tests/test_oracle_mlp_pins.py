"""Pins of the FP64 surrogate MLP oracle (CPU): the GELU values and
derivative, the backward pass against finite differences of the forward
pass, and the closed form of a first Adam step."""
import math

import numpy as np

from oracle import mlp


def test_gelu_values_and_derivative():
    # gelu(1) = Phi(1) (standard normal CDF at 1)
    assert mlp.gelu(np.array(1.0)) == np.float64(0.8413447460685429)
    assert mlp.gelu(np.array(0.0)) == 0.0
    assert abs(mlp.gelu(np.array(8.0)) - 8.0) < 1e-12
    z = np.linspace(-4, 4, 41)
    e = 1e-6
    fd = (mlp.gelu(z + e) - mlp.gelu(z - e)) / (2 * e)
    assert np.allclose(mlp.gelu_grad(z), fd, rtol=1e-7, atol=1e-9)


def test_backward_matches_finite_differences():
    p = mlp.init_params(3)
    rng = np.random.default_rng(4)
    x = rng.normal(size=(5, mlp.D_IN))
    x[:, 259:] = 0
    t = rng.normal(size=(5, 3))
    c = mlp.forward(p, x)
    g = mlp.backward(p, c, mlp.force_loss_grad_y(c["y"], t))
    e = 1e-6
    for name, idx in (("W1", (7, 11)), ("b1", (3,)), ("W2", (100, 5)), ("b3", (250,)), ("W4", (1, 17)),
                      ("b4", (2,)), ("W3", (0, 0))):
        q = {k: v.copy() for k, v in p.items()}
        q[name][idx] += e
        lp = mlp.force_loss(mlp.forward(q, x)["y"], t)
        q[name][idx] -= 2 * e
        lm = mlp.force_loss(mlp.forward(q, x)["y"], t)
        fd = (lp - lm) / (2 * e)
        assert abs(g[name][idx] - fd) <= 1e-6 * max(1.0, abs(fd)), (name, g[name][idx], fd)
    # the unused outputs 4..15 receive no gradient from the force loss
    assert np.all(g["W4"][4:] == 0) and np.all(g["b4"][3:] == 0)


def test_first_adam_step_closed_form():
    w = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 0.0])
    lr = 1e-3
    w1, m, v = mlp.adam_update(w, g, np.zeros(3), np.zeros(3), 1, lr)
    # bias-corrected moments equal g and g^2 after one step
    assert np.allclose(w1, w - lr * g / (np.abs(g) + 1e-8))
    assert math.isclose(m[0], 0.1 * 0.3) and math.isclose(v[1], 0.001 * 16.0)
