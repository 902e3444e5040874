"""Seeded synthetic scene generators (inputs only).

This module produces the initial states and parameter sets of the workloads
the step is run and checked on.  It holds none of the method's arithmetic: no
kernel, no force, no binning.  The random numbers come from the integer hash
the paper uses in its ``initialize_particle`` kernel (section "Boid Motion and
Agent Fluid Interaction"): the state of particle ``id`` starts at
``seed + id`` and every draw scrambles it with the three xor-shift-multiply
rounds and returns ``s / 4294967295``.

Particle ids follow the paper's convention: ids ``0 .. n_boid-1`` are the
particles attached to boids, ids ``n_boid ..`` are the fluid particles.  A
boid's own draws therefore come from the stream of its attached particle id.

All arrays are float32, shaped ``(n, 4)`` (x, y, z, 0) so that they can be
handed to the step library and to the CPU oracle alike.
"""
from __future__ import annotations

import math

import numpy as np

BASE_SEED = 20231115  # base seed; a workload adds its own index to it

_M1 = np.uint32(2747636419)
_M2 = np.uint32(2654435769)
_S16 = np.uint32(16)


class PaperHashRNG:
    """Vectorised copy of the paper's per-thread integer hash generator.

    One independent stream per id: ``s = seed + id`` (mod 2**32).  Each call
    to :meth:`next_u32` advances every stream by one draw.
    """

    def __init__(self, seed: int, ids: np.ndarray):
        ids = np.asarray(ids, dtype=np.int64)
        self.s = ((np.int64(seed) + ids) & 0xFFFFFFFF).astype(np.uint32)

    def next_u32(self) -> np.ndarray:
        s = self.s
        s = s ^ _M1
        s = s * _M2
        s = s ^ (s >> _S16)
        s = s * _M2
        s = s ^ (s >> _S16)
        s = s * _M2
        self.s = s
        return s.copy()

    def next_unit(self) -> np.ndarray:
        """Draw in [0, 1]: the integer over 4294967295 in double, then float32."""
        return (self.next_u32().astype(np.float64) / 4294967295.0).astype(np.float32)

    def uniform(self, a, b) -> np.ndarray:
        """``a + u * (b - a)`` in float32, like the paper's ``r(a, b)``."""
        a = np.float32(a)
        b = np.float32(b)
        u = self.next_unit()
        return (a + u * (b - a)).astype(np.float32)


def f32(x) -> float:
    """Round a Python number to the nearest float32 and return it as float."""
    return float(np.float32(x))


def default_params(**overrides) -> dict:
    """The constant set of the dam-break workloads (every float float32-exact).

    h = 0.0457, rest density 1000, gas constant 3, viscosity 3.5, dt = 1e-3,
    gravity -9.8 along y (y is up), cell size h/2 (the grid cell is a free
    parameter of the method; h/2 lets the walk clip each particle's search
    to its h-sphere; cell_size_x = 0: the same along x), wall restitution
    0.75, boid radii 2h / 4h / 4h and the boid weights below.
    ``mass`` must be supplied by the caller (it depends on the layout).
    """
    h = f32(0.0457)
    p = dict(
        h=h, rho0=1000.0, k=3.0, mu=3.5, dt=f32(1e-3),
        gx=0.0, gy=f32(-9.8), gz=0.0, mass=None,
        box_min=(0.0, 0.0, 0.0), box_max=(1.0, 1.0, 1.0),
        cell_size=f32(np.float32(h) / np.float32(2)), const_set=0, wall_restitution=0.75,
        r_sep=f32(np.float32(2) * np.float32(h)),
        r_vis=f32(np.float32(4) * np.float32(h)),
        w_sep=f32(0.05), w_align=f32(0.05), w_coh=f32(0.005),
        sph_factor=1.0, v_min=f32(0.05), v_max=1.0, edge_turn=f32(0.05),
        boid_cell_size=f32(np.float32(4) * np.float32(h)),
        coupling_mode=0, cell_size_x=0.0,
    )
    p.update(overrides)
    for key, val in list(p.items()):
        if isinstance(val, float):
            p[key] = f32(val)
        elif isinstance(val, tuple):
            p[key] = tuple(f32(v) for v in val)
    return p


def _pack4(xyz: np.ndarray) -> np.ndarray:
    out = np.zeros((xyz.shape[0], 4), dtype=np.float32)
    out[:, :3] = xyz
    return out


def lattice_block(counts, spacing, origin, jitter_frac, rng: PaperHashRNG) -> np.ndarray:
    """Jittered cubic lattice: point (i,j,k) at origin + (idx + 1/2) * spacing
    plus a uniform jitter in +-jitter_frac * spacing per component.
    Points are ordered x fastest, then y, then z; ``rng`` must hold one stream
    per point in that order."""
    nx, ny, nz = counts
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    idx = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1).astype(np.float64)
    base = np.asarray(origin, np.float64) + (idx + 0.5) * float(spacing)
    jit = float(jitter_frac) * float(spacing)
    jx = rng.uniform(-jit, jit)
    jy = rng.uniform(-jit, jit)
    jz = rng.uniform(-jit, jit)
    pos = (base.astype(np.float32) + np.stack([jx, jy, jz], axis=1)).astype(np.float32)
    return _pack4(pos)


def uniform_block(lo, hi, rng: PaperHashRNG, eps=1e-4) -> np.ndarray:
    """Uniform points in [lo + eps, hi - eps] per axis, one stream per point."""
    cols = [rng.uniform(lo[a] + eps, hi[a] - eps) for a in range(3)]
    return _pack4(np.stack(cols, axis=1))


def unit_headings(rng: PaperHashRNG) -> np.ndarray:
    """Uniformly distributed unit vectors (z = 2u - 1, phi = 2 pi u')."""
    z = rng.next_unit().astype(np.float64) * 2.0 - 1.0
    phi = rng.next_unit().astype(np.float64) * (2.0 * math.pi)
    rxy = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([rxy * np.cos(phi), rxy * np.sin(phi), z], axis=1)


def boids_uniform(n_boid, lo, hi, seed, speed=1.0):
    """Boids uniform in the box with random unit headings times ``speed``."""
    rng = PaperHashRNG(seed, np.arange(n_boid))
    pos = uniform_block(lo, hi, rng, eps=1e-3)
    vel = _pack4((unit_headings(rng) * speed).astype(np.float32))
    return pos, vel


def boids_schools(n_boid, n_schools, lo, hi, seed, radius=0.1, speed=0.5, noise=0.1):
    """Schools: centres uniform in [lo, hi]; members uniform in a ball of
    ``radius`` around their centre; heading = school heading + ``noise`` *
    random unit vector, normalised, times ``speed``.  Boid b joins school
    b mod n_schools."""
    crng = PaperHashRNG(seed + 7919, np.arange(n_schools))
    centres = np.stack([crng.uniform(lo[a] + radius, hi[a] - radius) for a in range(3)], axis=1)
    heads = unit_headings(crng)
    rng = PaperHashRNG(seed, np.arange(n_boid))
    school = np.arange(n_boid) % n_schools
    d = unit_headings(rng)
    r = radius * np.cbrt(rng.next_unit().astype(np.float64))
    pos = centres[school].astype(np.float64) + d * r[:, None]
    h = heads[school] + noise * unit_headings(rng)
    h /= np.linalg.norm(h, axis=1, keepdims=True)
    return _pack4(pos.astype(np.float32)), _pack4((h * speed).astype(np.float32))


def _zeros4(n):
    return np.zeros((n, 4), dtype=np.float32)


def dam_break_small(seed_offset=0, n_side=16, n_boid=16):
    """4,096 particles on a 16x16x16 lattice at spacing h/2 (jitter +-0.1
    spacing) in the (0,0,0) corner of the unit box, 16 boids uniform in the
    box with unit-speed random headings.  Mass: the caller calibrates it so
    that the lattice density equals the rest density (``lattice_spacing``)."""
    p = default_params()
    seed = BASE_SEED + 0 + seed_offset
    s = f32(np.float32(p["h"]) / np.float32(2))
    n = n_side ** 3
    rng = PaperHashRNG(seed, n_boid + np.arange(n))
    pos = lattice_block((n_side,) * 3, s, (0.0, 0.0, 0.0), 0.1, rng)
    bpos, bvel = boids_uniform(n_boid, p["box_min"], p["box_max"], seed)
    return dict(name=f"dam-break {n} particles, {n_boid} boids, unit box",
                params=p, fluid_pos=pos, fluid_vel=_zeros4(n),
                boid_pos=bpos, boid_vel=bvel, lattice_spacing=s)


def dam_break_column(seed_offset=0, n_side=64, n_boid=1024):
    """262,144 particles: a 64^3 lattice at spacing 1/64 (jitter +-0.1
    spacing) filling [0,1]^3 of a 2x1x1 tank, 1,024 boids uniform in the
    tank with unit-speed headings."""
    p = default_params(box_max=(2.0, 1.0, 1.0))
    seed = BASE_SEED + 1 + seed_offset
    s = f32(1.0 / n_side)
    n = n_side ** 3
    rng = PaperHashRNG(seed, n_boid + np.arange(n))
    pos = lattice_block((n_side,) * 3, s, (0.0, 0.0, 0.0), 0.1, rng)
    bpos, bvel = boids_uniform(n_boid, p["box_min"], p["box_max"], seed)
    return dict(name=f"dam-break column {n} particles, {n_boid} boids, 2x1x1 tank",
                params=p, fluid_pos=pos, fluid_vel=_zeros4(n),
                boid_pos=bpos, boid_vel=bvel, lattice_spacing=s)


def large_tank(seed_offset=0, n=2_097_152, n_boid=16_384, n_schools=8):
    """2,097,152 particles uniform in the lower 40% ([0,4]x[0,0.8]x[0,2]) of
    a 4x2x2 tank, mass = rest density * fluid volume / n.  The boids (8
    schools) are returned separately; the workload settles the fluid first
    and releases them afterwards.  The grid's cells are h/2 along y and z
    and h/8 along x (a row of cells is one run of sorted slots, so narrow x
    cells clip each row of a particle's walk closer to its h-sphere)."""
    lo, hi = (0.0, 0.0, 0.0), (4.0, 0.8, 2.0)
    vol = (hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2])
    h = np.float32(default_params()["h"])
    p = default_params(box_max=(4.0, 2.0, 2.0), mass=f32(1000.0 * vol / n), cell_size_x=f32(h / np.float32(8)))
    seed = BASE_SEED + 2 + seed_offset
    rng = PaperHashRNG(seed, n_boid + np.arange(n))
    pos = uniform_block(lo, hi, rng)
    bpos, bvel = boids_schools(n_boid, n_schools, lo, hi, seed)
    return dict(name=f"large tank {n} particles, {n_boid} boids in {n_schools} schools, 4x2x2",
                params=p, fluid_pos=pos, fluid_vel=_zeros4(n),
                boid_pos=bpos, boid_vel=bvel, lattice_spacing=None)


def scaled_block(n, n_boid, box_max, region_hi, seed, mass_density=1000.0):
    """A small uniform-random scene of n particles in [0, region_hi] of a
    [0, box_max] tank with mass = rest density * region volume / n and
    n_boid uniform boids; used for parity cases of chosen sizes."""
    vol = region_hi[0] * region_hi[1] * region_hi[2]
    p = default_params(box_max=tuple(box_max), mass=f32(mass_density * vol / max(n, 1)))
    rng = PaperHashRNG(seed, n_boid + np.arange(n))
    pos = uniform_block((0.0, 0.0, 0.0), region_hi, rng) if n else _zeros4(0)
    if n_boid:
        bpos, bvel = boids_uniform(n_boid, p["box_min"], p["box_max"], seed)
    else:
        bpos, bvel = _zeros4(0), _zeros4(0)
    return dict(name=f"uniform block {n} particles, {n_boid} boids",
                params=p, fluid_pos=pos, fluid_vel=_zeros4(n),
                boid_pos=bpos, boid_vel=bvel, lattice_spacing=None)


def batched_tanks(n_scenes=256, seed_offset=0, n_min=2048, n_max=65536, b_min=8, b_max=256):
    """Independent unit-box dam-breaks for the batched workload: particle
    counts log-uniform in [n_min, n_max], boid counts uniform in
    [b_min, b_max].  Scene k: a column of lattice layers at spacing h/2 (width
    min(ceil(N^(1/3)), floor(0.92/s)) points, the first N points of the
    lattice, jitter +-0.1 spacing) in the (0,0,0) corner, boids uniform in
    the box with unit-speed headings.  Mass as in the 4,096-particle
    dam-break (lattice density = rest density; ``lattice_spacing``).
    Returns a list of scene dicts."""
    seed = BASE_SEED + 3 + seed_offset
    size_rng = PaperHashRNG(seed, np.arange(n_scenes))
    u = size_rng.next_unit().astype(np.float64)
    v = size_rng.next_unit().astype(np.float64)
    counts = np.floor(np.exp(math.log(n_min) + u * (math.log(n_max) - math.log(n_min)))).astype(np.int64)
    counts = np.clip(counts, n_min, n_max)
    boids = (b_min + np.floor(v * (b_max - b_min + 1))).astype(np.int64)
    boids = np.clip(boids, b_min, b_max)
    out = []
    for k in range(n_scenes):
        p = default_params()
        s = f32(np.float32(p["h"]) / np.float32(2))
        n, nb = int(counts[k]), int(boids[k])
        w = min(int(math.ceil(n ** (1.0 / 3.0) - 1e-9)), int(math.floor(0.92 / s)))
        layers = int(math.ceil(n / (w * w)))
        rng = PaperHashRNG(seed + 1000 * (k + 1), nb + np.arange(w * w * layers))
        pos = lattice_block((w, layers, w), s, (0.0, 0.0, 0.0), 0.1, rng)[:n]
        bpos, bvel = boids_uniform(nb, p["box_min"], p["box_max"], seed + 1000 * (k + 1))
        out.append(dict(name=f"batched tank {k}: {n} particles, {nb} boids", params=p, fluid_pos=pos,
                        fluid_vel=_zeros4(n), boid_pos=bpos, boid_vel=bvel, lattice_spacing=s))
    return out
