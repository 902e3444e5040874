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


def test_stencil_features_by_hand():
    """h = 0.25: a boid at cell coordinate 8.5 of the feature grid (cells of
    size h) has its stencil start at cell 7 per axis (floor(8.5 - 1.5)) and
    sits 0.5 cells below the stencil's centre; fluid particles placed in
    stencil cells (0,0,0), (3,1,2) and (2,1,1) and one outside; only the
    last lies within h of the boid (r = h/2, q = 1/2)."""
    from oracle.features import stencil_features
    from paper_2311_15088_gb300 import scenes

    h = 0.25
    p = scenes.default_params(mass=0.01, h=h, cell_size=h / 2, box_max=(4.0, 4.0, 4.0))
    boid = np.array([[8.5 * h, 8.5 * h, 8.5 * h, 0]], np.float32)
    bvel = np.array([[0.1, -0.2, 0.3, 0]], np.float32)
    pts = [[7.5 * h, 7.5 * h, 7.5 * h], [7.2 * h, 7.9 * h, 7.1 * h],   # cell (7,7,7): stencil (0,0,0)
           [10.5 * h, 8.5 * h, 9.5 * h],                              # cell (10,8,9): stencil (3,1,2)
           [12.5 * h, 8.5 * h, 8.5 * h],                              # outside the stencil
           [9.0 * h, 8.5 * h, 8.5 * h]]                               # cell (9,8,8): stencil (2,1,1)
    vel = [[1, 0, 0], [0, 2, 0], [0, 0, 3], [5, 5, 5], [0, 0, 1]]
    fp = np.zeros((5, 4), np.float32)
    fp[:, :3] = pts
    fv = np.zeros((5, 4), np.float32)
    fv[:, :3] = vel
    x = stencil_features(p, fp, fv, boid, bvel)
    unit = p["mass"] / (h ** 3 * 1000.0)
    q0, q1, q2 = 0, (2 * 4 + 1) * 4 + 3, (1 * 4 + 1) * 4 + 2
    assert math.isclose(x[0, 4 * q0], 2 * unit) and np.allclose(x[0, 4 * q0 + 1:4 * q0 + 4], [0.5, 1.0, 0.0])
    assert math.isclose(x[0, 4 * q1], unit) and np.allclose(x[0, 4 * q1 + 1:4 * q1 + 4], [0, 0, 3])
    assert math.isclose(x[0, 4 * q2], unit) and np.allclose(x[0, 4 * q2 + 1:4 * q2 + 4], [0, 0, 1])
    others = np.delete(np.arange(64), [q0, q1, q2])
    assert np.all(x[0, 4 * others] == 0)
    assert np.allclose(x[0, 256:259], [0.1, -0.2, 0.3]) and np.all(x[0, 270:] == 0)
    assert np.all(x[0, 259:262] == -0.5)
    # moments: the one neighbour at r = h/2 has weight 1 - q = 1/2
    kn = p["mass"] / (1000.0 * h ** 3)
    c6 = p["mass"] * 315.0 / (64.0 * math.pi * h ** 9)
    assert math.isclose(x[0, 262], c6 * h ** 6 * (1.0 + 0.75 ** 3) / 1000.0, rel_tol=1e-6)
    assert math.isclose(x[0, 263], 0.5 * kn, rel_tol=1e-6)
    assert np.allclose(x[0, 264:267], 0.5 * kn * np.array([-0.1, 0.2, 0.7]), rtol=1e-6)
    assert np.allclose(x[0, 267:270], 0.25 * kn * np.array([-1.0, 0.0, 0.0]), rtol=1e-6, atol=1e-12)


def test_stencil_offset_moves_with_the_boid():
    """The offset column follows the boid across a cell: at cell coordinate
    9.25 the stencil starts at 7 (floor(7.75)) and the offset is +0.25; at
    9.5 the stencil starts at 8 and the offset is -0.5."""
    from oracle.features import stencil_features
    from paper_2311_15088_gb300 import scenes

    h = 0.25
    p = scenes.default_params(mass=0.01, h=h, cell_size=h / 2, box_max=(4.0, 4.0, 4.0))
    boid = np.array([[9.25 * h, 9.5 * h, 8.0 * h, 0], [0.1 * h, 0.6 * h, 2.0 * h, 0]], np.float32)
    z = np.zeros((0, 4), np.float32)
    x = stencil_features(p, z, z, boid, np.zeros_like(boid))
    assert np.allclose(x[0, 259:262], [0.25, -0.5, 0.0])
    # near the minimum wall the stencil starts outside the grid (c0 = -2)
    assert np.allclose(x[1, 259:262], [0.1, 0.6 - 1.0, 0.0], atol=1e-6)
    assert np.all(x[:, :256] == 0)
