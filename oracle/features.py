"""Oracle of the surrogate's input features -- TEST INFRASTRUCTURE ONLY.

Row b of the features (272 columns), for boid b at p_b with velocity v_b:

* 0 .. 255: the 4 x 4 x 4 cells of size h of a feature grid anchored at the
  box minimum m, starting at c0 = floor(t - 1.5) per axis with
  t = (p_b - m) * inv_h in float32 (inv_h = fl(1/h)); cell
  q = (iz * 4 + iy) * 4 + ix gives columns 4q .. 4q+3 = (fluid particles in
  the cell * mass / (h^3 rho0), their mean velocity).  A fluid particle's
  feature cell is floor((x - m) * inv_h) in float32, like the binning of
  section "Neighborhood Search" (not clamped).
* 256 .. 258: v_b.
* 259 .. 261: t - c0 - 2 (float32): the boid's offset from the stencil's
  centre, in [-0.5, 0.5).
* 262: rho_b / rho0, the SPH density of the boid's attached particle: the
  poly6 sum of section "Smoothed Particle Hydrodynamics" over itself and
  the fluid particles within h (attached pairs excluded, as in the step).
* 263: S0 = m / (rho0 h^3) sum_j (1 - q_j).
* 264 .. 266: S1 = m / (rho0 h^3) sum_j (1 - q_j) (v_j - v_b).
* 267 .. 269: S2 = m / (rho0 h^3) sum_j (1 - q_j)^2 (p_b - x_j) / r_j.
* 270, 271: zero.

j runs over the fluid particles with r_j = |x_j - p_b| < h (float64 here),
q_j = r_j / h.  Counts and sums in float64.  ``with_scale=True`` also
returns, per feature, the magnitude its float32 evaluation rounds against
(the same sums or means of absolute values for the velocity means and the
moments, |feature| elsewhere).
"""
from __future__ import annotations

import math

import numpy as np

D_IN = 272


def stencil_features(p: dict, fluid_pos, fluid_vel, boid_pos, boid_vel, with_scale: bool = False):
    fp = np.asarray(fluid_pos, np.float32)[:, :3]
    fv = np.asarray(fluid_vel, np.float32)[:, :3].astype(np.float64)
    bp = np.asarray(boid_pos, np.float32)[:, :3]
    bv = np.asarray(boid_vel, np.float32)[:, :3].astype(np.float64)
    h32 = np.float32(p["h"])
    inv_h = np.float32(1.0 / float(h32))
    mn = np.asarray(p["box_min"], np.float32)
    h = float(h32)
    mass, rho0 = float(np.float32(p["mass"])), float(np.float32(p["rho0"]))
    # feature cell of every fluid particle (float32, two roundings, floor)
    fcell = np.floor((fp - mn) * inv_h).astype(np.int64)
    t = (bp - mn) * inv_h
    c0 = np.floor(t - np.float32(1.5))
    x = np.zeros((len(bp), D_IN))
    scale = np.zeros((len(bp), D_IN))
    dens_unit = mass / (h ** 3 * rho0)
    kn = mass / (rho0 * h ** 3)
    c6 = mass * 315.0 / (64.0 * math.pi * h ** 9)
    for b in range(len(bp)):
        rel = fcell - c0[b].astype(np.int64)
        inside = np.all((rel >= 0) & (rel < 4), axis=1)
        q = rel[inside, 0] + 4 * (rel[inside, 1] + 4 * rel[inside, 2])
        cnt = np.bincount(q, minlength=64).astype(np.float64)
        vs = np.stack([np.bincount(q, weights=fv[inside, a], minlength=64) for a in range(3)], 1)
        vabs = np.stack([np.bincount(q, weights=np.abs(fv[inside, a]), minlength=64) for a in range(3)], 1)
        x[b, 0:256:4] = cnt * dens_unit
        safe = np.maximum(cnt, 1.0)
        for a in range(3):
            x[b, 1 + a:256:4] = np.where(cnt > 0, vs[:, a] / safe, 0.0)
        x[b, 256:259] = bv[b]
        x[b, 259:262] = (t[b] - c0[b]) - np.float32(2.0)
        # kernel moments over the fluid within h
        d = fp.astype(np.float64) - bp[b].astype(np.float64)
        r = np.sqrt((d * d).sum(1))
        near = r < h
        w = 1.0 - r[near] / h
        dv = fv[near] - bv[b]
        x[b, 262] = c6 * (np.sum((h * h - r[near] ** 2) ** 3) + (h * h) ** 3) / rho0
        x[b, 263] = kn * w.sum()
        x[b, 264:267] = kn * (w[:, None] * dv).sum(0)
        dn, rn = d[near], r[near]
        unit = np.zeros_like(dn)
        pos_r = rn > 0
        unit[pos_r] = -dn[pos_r] / rn[pos_r, None]
        x[b, 267:270] = kn * ((w ** 2)[:, None] * unit).sum(0)
        scale[b] = np.abs(x[b])
        for a in range(3):
            scale[b, 1 + a:256:4] = np.where(cnt > 0, vabs[:, a] / safe, 0.0)
        scale[b, 264:267] = kn * (w[:, None] * np.abs(dv)).sum(0)
        scale[b, 267:270] = kn * (w ** 2).sum()
    return (x, scale) if with_scale else x
