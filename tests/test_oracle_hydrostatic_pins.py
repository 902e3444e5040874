"""Hydrostatics of the method's discretisation, on the oracle (CPU).

The pressure term of section "Pressure and Viscosity" is symmetrised as
(p_i + p_j) / 2 with the spiky gradient.  For a particle inside the fluid
the p_i half sums to zero (sum_j m/rho_j grad W_ij ~ grad 1 = 0), so in the
continuum limit the term carries HALF of the pressure gradient:
a_i = -(1 / (2 rho_i)) grad p + g.  The hydrostatic balance of the method is
therefore (k / 2) d(rho)/dy = -rho g, rho ~ exp(2 g depth / k), not the
exp(g depth / k) of the equation of state alone.  These checks use static
blocks far from every wall and from the free surface, so no boundary effect
enters; lattice spacing h/4 (about 250 neighbours) makes the lattice sums
close to their continuum integrals."""
import math

import numpy as np
import pytest

import oracle
from paper_2311_15088_gb300 import scenes


def _block(profile, frac=0.25, n=40):
    """A block of n x n x n particles at x, z spacing s = frac h whose layer
    spacing follows profile(y - y_c) (the relative spacing, 1 at the centre
    layer): density ~ 1 / layer spacing.  Returns (params, positions, index
    of the centre particle, layer heights)."""
    p = scenes.default_params(mass=scenes.f32(1.0))
    h = float(np.float32(p["h"]))
    s = h * frac
    ys = [0.0]
    yc = s * n / 2
    for _ in range(n - 1):
        ys.append(ys[-1] + s * profile(ys[-1] - yc))
    ys = np.array(ys) + 0.2
    xs = 0.2 + s * np.arange(n)
    X, Y, Z = np.meshgrid(xs, ys, xs, indexing="ij")
    pos = np.zeros((X.size, 4), np.float32)
    pos[:, 0], pos[:, 1], pos[:, 2] = X.ravel(), Y.ravel(), Z.ravel()
    q = dict(p, mu=0.0, cell_size=scenes.f32(h / 2), mass=scenes.f32(1000.0 * s ** 3))
    ic = int(np.argmin(np.sum((pos[:, :3] - pos[:, :3].mean(0)) ** 2, axis=1)))
    return q, pos, ic, ys


def _step(q, pos):
    z = np.zeros((0, 4), np.float32)
    return oracle.step(q, pos, np.zeros_like(pos), z, z)


def _centre_rho0(q, pos, ic):
    """rho0 set to the centre particle's density: p = 0 there."""
    q = dict(q, rho0=float(np.float32(_step(q, pos)["rho"][ic])))
    return q


def test_pressure_term_carries_half_the_gradient():
    """Density varying linearly by about 20 % across the block, no gravity
    or viscosity, at rest: the centre particle's acceleration is
    -(1/2)(1/rho) dp/dy (ratio within 1 % of 1/2), with dp/dy the central
    difference of the layer-mean pressures; and nothing sideways."""
    q, pos, ic, ys = _block(lambda dy: 1.0 / (1.0 + 0.4 * dy))
    q = _centre_rho0(dict(q, gx=0.0, gy=0.0, gz=0.0), pos, ic)
    o = _step(q, pos)
    h = float(q["h"])
    inner = (np.abs(pos[:, 0] - pos[ic, 0]) < 3 * h) & (np.abs(pos[:, 2] - pos[ic, 2]) < 3 * h)
    j = int(np.argmin(np.abs(ys - pos[ic, 1])))
    layer = lambda k: o["pressure"][inner & (np.abs(pos[:, 1] - np.float32(ys[k])) < 1e-6)].mean()
    dpdy = (layer(j + 1) - layer(j - 1)) / (np.float32(ys[j + 1]) - np.float32(ys[j - 1]))
    a = o["acc"][ic]
    ratio = a[1] / (-dpdy / o["rho"][ic])
    assert abs(ratio - 0.5) <= 0.01, ratio
    assert abs(a[0]) <= 1e-3 * abs(a[1]) and abs(a[2]) <= 1e-3 * abs(a[1])


@pytest.mark.parametrize("factor,expect", [(2.0, 0.0), (1.0, -0.5)])
def test_hydrostatic_profile_of_the_method(factor, expect):
    """Gravity on, layers spaced so that rho ~ exp(factor g depth / k): with
    factor 2 (the method's balance) the centre particle's acceleration is
    within 3 % of g of zero; with factor 1 (the equation of state's
    continuum profile) half of g is left unbalanced, a_y = -g/2 within 3 %
    of g."""
    p = scenes.default_params()
    g, k = abs(float(np.float32(p["gy"]))), float(np.float32(p["k"]))
    lam = factor * g / k
    q, pos, ic, _ = _block(lambda dy: math.exp(lam * dy))
    q = _centre_rho0(q, pos, ic)
    a = _step(q, pos)["acc"][ic]
    assert abs(a[1] / g - expect) <= 0.03, a[1] / g
