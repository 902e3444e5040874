"""CPU oracle of one SPH-with-boids step -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does; it
shares no code with this package (the two meet only through the seeded
inputs of ``paper_2311_15088_gb300.scenes``, which hold no method arithmetic).

The arithmetic lives in ``sph_oracle.c`` (plain C, double precision, built
with ``-ffp-contract=off``); this module only marshals numpy arrays.  See the
header of ``sph_oracle.c`` for the passages of the paper each pass follows
and the readings it takes where the paper is open.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sph_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` with gcc (OpenMP when the compiler has it)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", _SRC, "-o", _LIB + ".tmp"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:] + ["-lm"], check=True,
                       capture_output=True, text=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + ["-lm"], check=True, capture_output=True, text=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class OrParams(ctypes.Structure):
    _fields_ = [
        ("h", ctypes.c_double), ("rho0", ctypes.c_double), ("k", ctypes.c_double),
        ("mu", ctypes.c_double), ("dt", ctypes.c_double), ("g", ctypes.c_double * 3),
        ("mass", ctypes.c_double), ("box_min", ctypes.c_double * 3),
        ("box_max", ctypes.c_double * 3), ("cell_size", ctypes.c_double),
        ("const_set", ctypes.c_int), ("wall_restitution", ctypes.c_double),
        ("r_sep", ctypes.c_double), ("r_vis", ctypes.c_double), ("w_sep", ctypes.c_double),
        ("w_align", ctypes.c_double), ("w_coh", ctypes.c_double),
        ("sph_factor", ctypes.c_double), ("v_min", ctypes.c_double),
        ("v_max", ctypes.c_double), ("edge_turn", ctypes.c_double),
        ("boid_cell_size", ctypes.c_double), ("coupling_mode", ctypes.c_int),
        ("obstacles", ctypes.c_void_p), ("att_vel", ctypes.c_void_p), ("cell_size_x", ctypes.c_double),
    ]


class OrObstacles(ctypes.Structure):
    _fields_ = [
        ("n_sphere", ctypes.c_int), ("n_box", ctypes.c_int),
        ("sphere", ctypes.c_void_p), ("box", ctypes.c_void_p),
        ("w_obst", ctypes.c_double), ("near_factor", ctypes.c_double),
    ]


def make_obstacles(spheres=None, boxes=None, w_obst=0.05, near_factor=2.0):
    """The oracle's obstacle struct; returns (struct, arrays it points to)."""
    sph = np.ascontiguousarray(np.asarray(spheres if spheres is not None else np.zeros((0, 4)), np.float32)
                               .reshape(-1, 4))
    box = np.ascontiguousarray(np.asarray(boxes if boxes is not None else np.zeros((0, 6)), np.float32)
                               .reshape(-1, 6))
    o = OrObstacles()
    o.n_sphere, o.n_box = len(sph), len(box)
    o.sphere = sph.ctypes.data_as(ctypes.c_void_p) if len(sph) else None
    o.box = box.ctypes.data_as(ctypes.c_void_p) if len(box) else None
    o.w_obst = float(np.float32(w_obst))
    o.near_factor = float(np.float32(near_factor))
    return o, (sph, box)


_P = ctypes.POINTER
_D = _P(ctypes.c_double)
_I = _P(ctypes.c_int)
_U = _P(ctypes.c_uint)


class OrOutputs(ctypes.Structure):
    _fields_ = [
        ("rho", _D), ("pressure", _D), ("acc", _D), ("acc_scale", _D), ("influence", _D),
        ("touched", _I), ("nbr_count", _I),
        ("keys", _U), ("perm", _I), ("cell_start", _I),
        ("new_fluid_pos", _D), ("new_fluid_vel", _D),
        ("pre_wall_pos", _D), ("pre_wall_vel", _D), ("wall_margin", _D),
        ("fb", _D), ("new_boid_pos", _D), ("new_boid_vel", _D), ("boid_vscale", _D),
        ("boid_nsep", _I), ("boid_nvis", _I),
        ("boid_keys", _U), ("boid_perm", _I), ("boid_cell_start", _I),
        ("new_att_vel", _D),
    ]


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        vp = ctypes.c_void_p
        L.or_step.argtypes = [_P(OrParams), ctypes.c_int, ctypes.c_int, vp, vp, vp, vp, _P(OrOutputs)]
        L.or_bin.argtypes = [_P(OrParams), ctypes.c_int, ctypes.c_int, vp, vp, vp, vp]
        L.or_neighbors.argtypes = [_P(OrParams), ctypes.c_int, ctypes.c_int, vp, vp, vp, vp]
        L.or_brute_neighbors.argtypes = L.or_neighbors.argtypes
        L.or_grid_dims.argtypes = [_P(OrParams), ctypes.c_int, vp]
        for fn in ("or_w_poly6", "or_grad_spiky_factor", "or_lap_visc", "or_lattice_mass"):
            getattr(L, fn).argtypes = [_P(OrParams), ctypes.c_double]
            getattr(L, fn).restype = ctypes.c_double
        L.or_rng_stream.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int, vp]
        L.or_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def make_params(p: dict) -> OrParams:
    """Fill the oracle's own parameter struct from a parameter dict."""
    if p.get("mass") is None:
        raise ValueError("params['mass'] must be set")
    o = OrParams()
    for name in ("h", "rho0", "k", "mu", "dt", "mass", "cell_size", "wall_restitution",
                 "r_sep", "r_vis", "w_sep", "w_align", "w_coh", "sph_factor", "v_min",
                 "v_max", "edge_turn", "boid_cell_size"):
        setattr(o, name, float(np.float32(p[name])))
    o.g[:] = [float(np.float32(p["gx"])), float(np.float32(p["gy"])), float(np.float32(p["gz"]))]
    o.box_min[:] = [float(np.float32(v)) for v in p["box_min"]]
    o.box_max[:] = [float(np.float32(v)) for v in p["box_max"]]
    o.const_set = int(p["const_set"])
    o.coupling_mode = int(p["coupling_mode"])
    o.cell_size_x = float(np.float32(p.get("cell_size_x") or 0.0))
    return o


def _xyz(a) -> np.ndarray:
    a = np.asarray(a, dtype=np.float32)
    return np.ascontiguousarray(a[:, :3]) if a.size else np.zeros((0, 3), np.float32)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def grid_dims(p: dict, which: int = 0):
    d = np.zeros(3, np.int32)
    lib().or_grid_dims(ctypes.byref(make_params(p)), which, _ptr(d))
    return tuple(int(v) for v in d)


def num_threads() -> int:
    return int(lib().or_num_threads())


def w_poly6(p, r):
    return lib().or_w_poly6(ctypes.byref(make_params(p)), float(r))


def grad_spiky_factor(p, r):
    return lib().or_grad_spiky_factor(ctypes.byref(make_params(p)), float(r))


def lap_visc(p, r):
    return lib().or_lap_visc(ctypes.byref(make_params(p)), float(r))


def lattice_mass(p, spacing):
    q = dict(p)
    q.setdefault("mass", 1.0)
    if q["mass"] is None:
        q["mass"] = 1.0
    return lib().or_lattice_mass(ctypes.byref(make_params(q)), float(spacing))


def rng_stream(seed: int, pid: int, ncalls: int) -> np.ndarray:
    out = np.zeros(ncalls, np.uint32)
    lib().or_rng_stream(seed & 0xFFFFFFFF, pid & 0xFFFFFFFF, ncalls, _ptr(out))
    return out


def bin_particles(p: dict, pos, which: int = 0):
    """Keys, sorted permutation and cell_start (ncells + 1) of ``pos``."""
    x = _xyz(pos)
    n = x.shape[0]
    dims = grid_dims(p, which)
    keys = np.zeros(n, np.uint32)
    perm = np.zeros(n, np.int32)
    cs = np.zeros(dims[0] * dims[1] * dims[2] + 1, np.int32)
    lib().or_bin(ctypes.byref(make_params(p)), which, n, _ptr(x), _ptr(keys), _ptr(perm), _ptr(cs))
    return keys, perm, cs


def neighbors(p: dict, pos, n_att: int = 0, brute: bool = False, lists: bool = True):
    """Neighbour counts and (optionally) CSR lists.  Grid lists are in walk
    order, brute-force lists in ascending id order."""
    x = _xyz(pos)
    n = x.shape[0]
    counts = np.zeros(n, np.int32)
    fn = lib().or_brute_neighbors if brute else lib().or_neighbors
    pp = ctypes.byref(make_params(p))
    fn(pp, n, n_att, _ptr(x), _ptr(counts), None, None)
    if not lists:
        return counts, None, None
    offsets = np.zeros(n + 1, np.int64)
    np.cumsum(counts, out=offsets[1:])
    lst = np.zeros(int(offsets[-1]), np.int32)
    fn(pp, n, n_att, _ptr(x), _ptr(counts), _ptr(offsets), _ptr(lst))
    return counts, offsets, lst


def obstacle_grid(p: dict, spheres=None, boxes=None) -> np.ndarray:
    """The obstacle grid over the boid grid's cells: (ncells, 4) = mean
    outward normal, count."""
    bd = grid_dims(p, 1)
    out = np.zeros((bd[0] * bd[1] * bd[2], 4))
    o, keep = make_obstacles(spheres, boxes)
    lib().or_obstacle_grid(ctypes.byref(make_params(p)), ctypes.byref(o), _ptr(out))
    return out


def step(p: dict, fluid_pos, fluid_vel, boid_pos, boid_vel, obstacles=None, att_vel=None) -> dict:
    """One oracle step; returns every output as numpy arrays.

    Per-particle arrays are indexed by particle id (ids < n_boid are the
    boid-attached particles), per-fluid arrays by fluid index, per-boid
    arrays by boid index.  obstacles: None or a dict(spheres=(k, 4),
    boxes=(k, 6), w_obst, near_factor) of analytic obstacles the boids
    avoid.  att_vel: with the literal coupling (coupling_mode 1), the
    attached particles' velocities going into the step (None: the boids')."""
    fp, fv, bp, bv = (_xyz(a) for a in (fluid_pos, fluid_vel, boid_pos, boid_vel))
    nf, nb = fp.shape[0], bp.shape[0]
    n = nf + nb
    dims = grid_dims(p, 0)
    bdims = grid_dims(p, 1)
    o = dict(
        rho=np.zeros(n), pressure=np.zeros(n), acc=np.zeros((n, 3)), acc_scale=np.zeros(n),
        influence=np.zeros((n, 3)), touched=np.zeros(n, np.int32), nbr_count=np.zeros(n, np.int32),
        keys=np.zeros(n, np.uint32), perm=np.zeros(n, np.int32),
        cell_start=np.zeros(dims[0] * dims[1] * dims[2] + 1, np.int32),
        new_fluid_pos=np.zeros((nf, 3)), new_fluid_vel=np.zeros((nf, 3)),
        pre_wall_pos=np.zeros((nf, 3)), pre_wall_vel=np.zeros((nf, 3)), wall_margin=np.zeros(nf),
        fb=np.zeros((nb, 3)), new_boid_pos=np.zeros((nb, 3)), new_boid_vel=np.zeros((nb, 3)),
        boid_vscale=np.zeros(nb), boid_nsep=np.zeros(nb, np.int32), boid_nvis=np.zeros(nb, np.int32),
        boid_keys=np.zeros(nb, np.uint32), boid_perm=np.zeros(nb, np.int32),
        boid_cell_start=np.zeros(bdims[0] * bdims[1] * bdims[2] + 1, np.int32),
        new_att_vel=np.zeros((nb, 3)),
    )
    outs = OrOutputs()
    for name, arr in o.items():
        ctype = dict(OrOutputs._fields_)[name]
        setattr(outs, name, arr.ctypes.data_as(ctype))
    par = make_params(p)
    keep = None
    if obstacles is not None:
        ob, keep = make_obstacles(**obstacles)
        par.obstacles = ctypes.cast(ctypes.pointer(ob), ctypes.c_void_p)
    av = None
    if att_vel is not None:
        av = _xyz(att_vel)
        par.att_vel = av.ctypes.data_as(ctypes.c_void_p)
    rc = lib().or_step(ctypes.byref(par), nf, nb, _ptr(fp), _ptr(fv), _ptr(bp), _ptr(bv),
                       ctypes.byref(outs))
    del keep
    if rc != 0:
        raise ValueError(f"oracle step rejected the parameters (rc={rc})")
    return o


STATS = ("fluid", "nbr_mean", "nbr_max", "cell_max", "mom_x", "mom_y", "mom_z", "ke", "rho_min", "rho_max",
         "rho_mean", "speed_max")


def step_stats(p: dict, o: dict, n_boid: int) -> np.ndarray:
    """The step's diagnostics, each written out from its definition over the
    outputs ``o`` of one oracle step (``step``) of a scene with ``n_boid``
    boids, in the order of ``STATS``: the fluid particle count; the mean and
    largest neighbour count of the fluid particles (self excluded, section
    "Neighborhood Search"); the most particles in one cell of the step's
    binning; the momentum sum m v and the kinetic energy sum m |v|^2 / 2 of
    the fluid after the step; the smallest, largest and mean fluid density
    of the step; the largest fluid speed after the step.  Means and density
    bounds are 0 without fluid."""
    m = float(np.float32(p["mass"]))
    v = np.asarray(o["new_fluid_vel"], np.float64)
    nf = v.shape[0]
    nbr = np.asarray(o["nbr_count"][n_boid:], np.float64)
    rho = np.asarray(o["rho"][n_boid:], np.float64)
    occ = np.diff(np.asarray(o["cell_start"], np.int64))
    speed2 = (v * v).sum(axis=1)
    out = np.zeros(len(STATS))
    out[0] = nf
    out[3] = occ.max() if occ.size else 0
    if nf:
        out[1] = nbr.sum() / nf
        out[2] = nbr.max()
        out[4:7] = m * v.sum(axis=0)
        out[7] = 0.5 * m * speed2.sum()
        out[8], out[9], out[10] = rho.min(), rho.max(), rho.sum() / nf
        out[11] = np.sqrt(speed2.max())
    return out
