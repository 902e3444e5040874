"""Oracle of the surrogate's stencil features -- TEST INFRASTRUCTURE ONLY.

Row b of the features: the 4 x 4 x 4 cells of the particle grid starting at
c0 = floor((p_b - m) / d - 1.5) per axis (float32, like the grid's own cell
function); cell q = (iz * 4 + iy) * 4 + ix gives columns 4q .. 4q+3 =
(fluid particles in the cell * mass / (d^3 rho0), their mean velocity);
columns 256 .. 258 hold the boid's velocity, 259 .. 271 are zero.  A fluid
particle's cell is floor((x - m) * inv_d) in float32, clamped to the grid
(the binning of section "Neighborhood Search").  Counts and sums in float64.
"""
from __future__ import annotations

import numpy as np

from oracle import grid_dims

D_IN = 272


def _f32(v):
    return np.float32(v)


def _cells(p, xyz):
    dims = grid_dims(p, 0)
    mn = np.asarray(p["box_min"], np.float32)
    inv_d = np.float32(1.0) / np.float32(p["cell_size"])
    t = (xyz.astype(np.float32) - mn) * inv_d          # two float32 roundings
    c = np.floor(t)
    out = np.zeros(c.shape, np.int64)
    for a in range(3):
        ca = c[:, a]
        ok = ca >= 0
        ca = np.where(ok, ca, 0)
        ca = np.minimum(ca, dims[a] - 1)
        out[:, a] = ca.astype(np.int64)
    return out, dims


def stencil_features(p: dict, fluid_pos, fluid_vel, boid_pos, boid_vel) -> np.ndarray:
    fp = np.asarray(fluid_pos, np.float32)[:, :3]
    fv = np.asarray(fluid_vel, np.float32)[:, :3].astype(np.float64)
    bp = np.asarray(boid_pos, np.float32)[:, :3]
    bv = np.asarray(boid_vel, np.float32)[:, :3].astype(np.float64)
    cells, dims = _cells(p, fp)
    ncell = dims[0] * dims[1] * dims[2]
    key = cells[:, 0] + dims[0] * (cells[:, 1] + dims[1] * cells[:, 2])
    count = np.bincount(key, minlength=ncell).astype(np.float64)
    vsum = np.stack([np.bincount(key, weights=fv[:, a], minlength=ncell) for a in range(3)], 1)
    d = float(np.float32(p["cell_size"]))
    dens_scale = float(p["mass"]) / (d ** 3 * float(p["rho0"]))
    mn = np.asarray(p["box_min"], np.float32)
    inv_d = np.float32(1.0) / np.float32(p["cell_size"])
    t = (bp - mn) * inv_d
    c0 = np.floor(t - np.float32(1.5)).astype(np.int64)
    x = np.zeros((len(bp), D_IN))
    for q in range(64):
        off = np.array([q & 3, (q >> 2) & 3, q >> 4])
        c = c0 + off
        inside = np.all((c >= 0) & (c <= np.asarray(dims) - 1), axis=1)
        k = np.where(inside, c[:, 0] + dims[0] * (c[:, 1] + dims[1] * c[:, 2]), 0)
        n = np.where(inside, count[k], 0.0)
        x[:, 4 * q] = n * dens_scale
        safe = np.maximum(n, 1.0)
        for a in range(3):
            x[:, 4 * q + 1 + a] = np.where(n > 0, vsum[k, a] / safe, 0.0)
    x[:, 256:259] = bv
    return x
