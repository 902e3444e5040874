"""ctypes binding of the step library (include/sph.h), same names as the C ABI.

Argument marshalling only: every step of the method runs in the CUDA
kernels of ``libsph_gb300.so``.  Importing this module fails loudly if the
library has not been built (``python -m paper_2311_15088_gb300.build``);
there is no CPU fallback.

:class:`Scene` is a thin convenience wrapper that keeps the workspace in a
torch tensor and passes torch's current stream.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

# SPH_GB300_LIB may name the bounds-checked build of the same library
_LIB_PATH = os.environ.get("SPH_GB300_LIB") or os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                                             "libsph_gb300.so")
if not os.path.exists(_LIB_PATH):
    raise ImportError(f"{_LIB_PATH} is missing: build it with `python -m paper_2311_15088_gb300.build`")
_lib = ctypes.CDLL(_LIB_PATH)

SPH_OK, SPH_ERR_ARG, SPH_ERR_CUDA, SPH_ERR_OVERFLOW, SPH_ERR_TIMEOUT, SPH_ERR_STATE = range(6)
SPH_MULLER3D, SPH_PAPER_LITERAL = 0, 1
SPH_COUPLE_FORCE, SPH_COUPLE_LITERAL = 0, 1
SPH_DEV_NONFINITE, SPH_DEV_CLAMPED, SPH_DEV_TIMEOUT, SPH_DEV_LIST_OVERFLOW, SPH_DEV_BOUNDS = 1, 2, 4, 8, 16
SPH_BOID_EXACT, SPH_BOID_SURROGATE, SPH_BOID_SURROGATE_FALLBACK, SPH_BOID_EXACT_LOCAL = 0, 1, 2, 3
SPH_MAX_OBSTACLES = 256
SPH_STATS_N = 12
STATS = ("fluid", "nbr_mean", "nbr_max", "cell_max", "mom_x", "mom_y", "mom_z", "ke", "rho_min", "rho_max",
         "rho_mean", "speed_max")

FIELDS = {
    "rho": (0, np.float32, 1), "pressure": (1, np.float32, 1), "acc": (2, np.float32, 4),
    "touched": (3, np.int32, 1), "influence": (4, np.float32, 4), "nbr_count": (5, np.int32, 1),
    "keys": (6, np.uint32, 1), "perm": (7, np.int32, 1), "cell_start": (8, np.uint32, 1),
    "fb": (9, np.float32, 4), "boid_keys": (10, np.uint32, 1), "boid_perm": (11, np.int32, 1),
    "boid_cell_start": (12, np.uint32, 1), "ncand": (13, np.int32, 1), "fallback": (14, np.int32, 1),
    "obstacle_grid": (15, np.float32, 4), "att_vel": (16, np.float32, 4), "nseg": (17, np.int32, 1),
}


class SphParams(ctypes.Structure):
    _fields_ = [
        ("h", ctypes.c_float), ("rho0", ctypes.c_float), ("k", ctypes.c_float), ("mu", ctypes.c_float),
        ("dt", ctypes.c_float), ("gx", ctypes.c_float), ("gy", ctypes.c_float), ("gz", ctypes.c_float),
        ("mass", ctypes.c_float), ("box_min", ctypes.c_float * 3), ("box_max", ctypes.c_float * 3),
        ("cell_size", ctypes.c_float), ("const_set", ctypes.c_int), ("wall_restitution", ctypes.c_float),
        ("r_sep", ctypes.c_float), ("r_vis", ctypes.c_float), ("w_sep", ctypes.c_float),
        ("w_align", ctypes.c_float), ("w_coh", ctypes.c_float), ("sph_factor", ctypes.c_float),
        ("v_min", ctypes.c_float), ("v_max", ctypes.c_float), ("edge_turn", ctypes.c_float),
        ("boid_cell_size", ctypes.c_float), ("coupling_mode", ctypes.c_int), ("cell_size_x", ctypes.c_float),
    ]


_vp, _i, _sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
_P = ctypes.POINTER(SphParams)
_sig = {
    "sph_workspace_size": (_i, [_P, _i, _i, ctypes.POINTER(_sz)]),
    "sph_grid_dims": (_i, [_P, _i, _vp]),
    "sph_lattice_mass": (_i, [_P, ctypes.c_float, ctypes.POINTER(ctypes.c_float)]),
    "sph_create": (_i, [_P, _i, _i, _vp, _sz, ctypes.POINTER(_vp)]),
    "sph_set_state": (_i, [_vp, _vp, _vp, _vp, _vp, _i, _vp]),
    "sph_get_state": (_i, [_vp, _vp, _vp, _vp, _vp, _i, _vp]),
    "sph_step": (_i, [_vp, _i, _vp]),
    "sph_boid_forces": (_i, [_vp, _i, _vp, _vp]),
    "sph_graph_boid_forces": (_i, [_vp, _i, _vp, _vp]),
    "sph_get_fields": (_i, [_vp, _i, _vp, _i, _vp]),
    "sph_debug_neighbors": (_i, [_vp, _vp, _vp, _vp, _vp]),
    "sph_status": (_i, [_vp, ctypes.POINTER(ctypes.c_uint)]),
    "sph_stats": (_i, [_vp, _vp, _i, _vp]),
    "sph_clear_status": (_i, [_vp, _vp]),
    "sph_last_error": (ctypes.c_char_p, [_vp]),
    "sph_launch_count": (ctypes.c_longlong, [_vp]),
    "sph_destroy": (None, [_vp]),
    "sph_profile_enable": (_i, [_vp, _i]),
    "sph_profile_read": (_i, [_vp, _vp, _vp, _i]),
    "sph_bin_static": (_i, [_P, _i, _vp, _vp, _vp, _vp, _vp, _vp]),
    "sph_batch_workspace_size": (_i, [_P, _vp, _vp, _i, ctypes.POINTER(_sz)]),
    "sph_batch_create": (_i, [_P, _vp, _vp, _i, _vp, _sz, ctypes.POINTER(_vp)]),
    "sph_set_tuning": (_i, [_vp, _i, _i]),
    "sph_set_diagnostics": (_i, [_vp, _i]),
    "sph_set_pipeline": (_i, [_vp, _i, _i]),
    "sph_set_particles_per_thread": (_i, [_vp, _i]),
    "sph_debug_barrier_skip": (_i, [_vp, _i]),
    "sph_set_neighbor_lists": (_i, [_vp, _vp, ctypes.c_size_t]),
    "sph_debug_bucket_neighbors": (_i, [_vp, _vp, ctypes.c_size_t, _i, _vp, _vp, _vp]),
    "sph_graph_step": (_i, [_vp, _i, _vp]),
    "sph_mlp_workspace_size": (_i, [_i, ctypes.POINTER(_sz)]),
    "sph_mlp_create": (_i, [_i, _vp, _sz, ctypes.POINTER(_vp)]),
    "sph_mlp_destroy": (None, [_vp]),
    "sph_mlp_set_params": (_i, [_vp, _vp, _vp]),
    "sph_mlp_get_params": (_i, [_vp, _vp, _vp]),
    "sph_mlp_get_optimizer_state": (_i, [_vp, _vp, _vp, _vp, ctypes.POINTER(ctypes.c_longlong), _vp]),
    "sph_mlp_set_optimizer_state": (_i, [_vp, _vp, _vp, ctypes.c_longlong, _vp]),
    "sph_mlp_forward": (_i, [_vp, _vp, _i, _vp, _vp]),
    "sph_mlp_gradients": (_i, [_vp, _vp, _vp, _i, _vp, _vp]),
    "sph_mlp_train_step": (_i, [_vp, _vp, _vp, _i, _i, ctypes.c_float, _vp, _vp]),
    "sph_mlp_status": (_i, [_vp, ctypes.POINTER(ctypes.c_uint), _vp]),
    "sph_mlp_launch_count": (ctypes.c_longlong, [_vp]),
    "sph_debug_gemm": (_i, [_vp, _i, _vp, _i, _i, _i, _i, _i, _vp, _vp, _vp]),
    "sph_debug_gelu": (_i, [_vp, _i, _i, _vp, _vp]),
    "sph_features": (_i, [_vp, _vp, _vp]),
    "sph_voxel_grid": (_i, [_P, ctypes.c_float, ctypes.c_float, _vp, _vp]),
    "sph_voxel_density": (_i, [_vp, _vp, _vp, ctypes.c_float, ctypes.c_float, ctypes.c_float, _vp, _vp, _vp]),
    "sph_mc_workspace_size": (_i, [_vp, ctypes.POINTER(_sz)]),
    "sph_marching_cubes": (_i, [_vp, _vp, _vp, ctypes.c_float, ctypes.c_float, _vp, _sz, _vp, ctypes.c_longlong,
                                _vp, _vp]),
    "sph_mc_tables": (_i, [_vp, _vp]),
    "sph_set_obstacles": (_i, [_vp, _vp, _i, _vp, _i, ctypes.c_float, ctypes.c_float, _vp]),
    "sph_set_surrogate": (_i, [_vp, _vp, ctypes.c_float, ctypes.c_float]),
    "sph_set_surrogate_bounds": (_i, [_vp, _vp, _vp]),
}
for _name, (_res, _args) in _sig.items():
    _fn = getattr(_lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args

EXPORTED = tuple(_sig)


class SphError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"sph error {code}: {msg}")
        self.code = code


def _check(rc, handle=None):
    if rc != SPH_OK:
        raise SphError(rc, (_lib.sph_last_error(handle) or b"").decode())


def make_params(p: dict) -> SphParams:
    """Fill the library's parameter struct from a parameter dict."""
    if p.get("mass") is None:
        raise ValueError("params['mass'] must be set")
    s = SphParams()
    for name, ctype in SphParams._fields_:
        if name in ("box_min", "box_max"):
            getattr(s, name)[:] = [float(v) for v in p[name]]
        elif ctype is ctypes.c_int:
            setattr(s, name, int(p[name]))
        elif name == "cell_size_x":
            setattr(s, name, float(p.get(name, 0.0)))
        else:
            setattr(s, name, float(p[name]))
    return s


# ----------------------------------------------------------- C-ABI names

def sph_workspace_size(params: dict, n_fluid: int, n_boid: int) -> int:
    out = _sz()
    _check(_lib.sph_workspace_size(ctypes.byref(make_params(params)), n_fluid, n_boid, ctypes.byref(out)))
    return int(out.value)


def sph_grid_dims(params: dict, which: int = 0):
    d = (ctypes.c_int * 3)()
    _check(_lib.sph_grid_dims(ctypes.byref(make_params(params)), which, ctypes.cast(d, _vp)))
    return tuple(d)


def sph_lattice_mass(params: dict, spacing: float) -> float:
    q = dict(params)
    if q.get("mass") is None:
        q["mass"] = 1.0
    m = ctypes.c_float()
    _check(_lib.sph_lattice_mass(ctypes.byref(make_params(q)), float(spacing), ctypes.byref(m)))
    return float(m.value)


def sph_create(params: dict, n_fluid: int, n_boid: int, workspace_ptr: int, ws_bytes: int):
    h = _vp()
    _check(_lib.sph_create(ctypes.byref(make_params(params)), n_fluid, n_boid, workspace_ptr, ws_bytes,
                           ctypes.byref(h)))
    return h


def _param_array(params_list):
    arr = (SphParams * len(params_list))()
    for k, p in enumerate(params_list):
        arr[k] = make_params(p)
    return arr


def sph_batch_workspace_size(params_list, n_fluid, n_boid) -> int:
    S = len(params_list)
    nf = (ctypes.c_int * S)(*n_fluid)
    nb = (ctypes.c_int * S)(*n_boid)
    out = _sz()
    _check(_lib.sph_batch_workspace_size(_param_array(params_list), ctypes.cast(nf, _vp), ctypes.cast(nb, _vp), S,
                                         ctypes.byref(out)))
    return int(out.value)


def sph_batch_create(params_list, n_fluid, n_boid, workspace_ptr: int, ws_bytes: int):
    S = len(params_list)
    nf = (ctypes.c_int * S)(*n_fluid)
    nb = (ctypes.c_int * S)(*n_boid)
    h = _vp()
    _check(_lib.sph_batch_create(_param_array(params_list), ctypes.cast(nf, _vp), ctypes.cast(nb, _vp), S,
                                 workspace_ptr, ws_bytes, ctypes.byref(h)))
    return h


def sph_set_tuning(h, block: int, use_segments: int):
    _check(_lib.sph_set_tuning(h, block, use_segments), h)


def sph_set_diagnostics(h, record: int):
    _check(_lib.sph_set_diagnostics(h, record), h)


def sph_set_particles_per_thread(h, ppt: int):
    _check(_lib.sph_set_particles_per_thread(h, ppt), h)


def sph_set_pipeline(h, tile_slots: int, block: int = 256):
    _check(_lib.sph_set_pipeline(h, tile_slots, block), h)


def sph_debug_barrier_skip(h, cta: int):
    _check(_lib.sph_debug_barrier_skip(h, cta), h)


def sph_set_neighbor_lists(h, pair_buffer_ptr, nbytes: int):
    _check(_lib.sph_set_neighbor_lists(h, pair_buffer_ptr, nbytes), h)


def sph_debug_bucket_neighbors(h, scratch_ptr, nbytes: int, capacity: int, counts_ptr, dropped_ptr, stream: int):
    _check(_lib.sph_debug_bucket_neighbors(h, scratch_ptr, nbytes, capacity, counts_ptr, dropped_ptr, stream), h)


def sph_graph_step(h, nsteps: int, stream: int):
    _check(_lib.sph_graph_step(h, nsteps, stream), h)


def sph_set_state(h, fluid_pos, fluid_vel, boid_pos, boid_vel, on_host: int, stream: int):
    _check(_lib.sph_set_state(h, fluid_pos, fluid_vel, boid_pos, boid_vel, on_host, stream), h)


def sph_get_state(h, fluid_pos, fluid_vel, boid_pos, boid_vel, on_host: int, stream: int):
    _check(_lib.sph_get_state(h, fluid_pos, fluid_vel, boid_pos, boid_vel, on_host, stream), h)


def sph_step(h, nsteps: int, stream: int):
    _check(_lib.sph_step(h, nsteps, stream), h)


def sph_boid_forces(h, mode: int, out_ptr: int, stream: int):
    _check(_lib.sph_boid_forces(h, mode, out_ptr, stream), h)


def sph_graph_boid_forces(h, mode: int, out_ptr: int, stream: int):
    _check(_lib.sph_graph_boid_forces(h, mode, out_ptr, stream), h)


def sph_features(h, x_ptr, stream: int):
    _check(_lib.sph_features(h, x_ptr, stream), h)


def sph_set_surrogate(h, mlp_handle, f_scale: float, log_err_max: float):
    _check(_lib.sph_set_surrogate(h, mlp_handle, float(f_scale), float(log_err_max)), h)


def sph_set_surrogate_bounds(h, lo, hi):
    _check(_lib.sph_set_surrogate_bounds(h, lo, hi), h)


def sph_get_fields(h, field: int, out_ptr: int, on_host: int, stream: int):
    _check(_lib.sph_get_fields(h, field, out_ptr, on_host, stream), h)


def sph_debug_neighbors(h, counts_ptr: int, offsets_ptr, list_ptr, stream: int):
    _check(_lib.sph_debug_neighbors(h, counts_ptr, offsets_ptr, list_ptr, stream), h)


def sph_stats(h, out_ptr: int, on_host: int, stream: int):
    _check(_lib.sph_stats(h, out_ptr, on_host, stream), h)


def sph_status(h) -> int:
    bits = ctypes.c_uint()
    _check(_lib.sph_status(h, ctypes.byref(bits)), h)
    return int(bits.value)


def sph_clear_status(h, stream: int):
    _check(_lib.sph_clear_status(h, stream), h)


def sph_last_error(h) -> str:
    return (_lib.sph_last_error(h) or b"").decode()


def sph_launch_count(h) -> int:
    return int(_lib.sph_launch_count(h))


def sph_destroy(h):
    _lib.sph_destroy(h)


KINDS = ("keys", "scan", "scatter", "sort", "density", "forces", "boid_bin", "boid_rules", "lists", "features",
         "pipeline")


def sph_profile_enable(h, max_passes: int):
    _check(_lib.sph_profile_enable(h, max_passes), h)


def sph_profile_read(h) -> dict:
    """Summed milliseconds and pass counts per kind since the last read."""
    ms = (ctypes.c_double * len(KINDS))()
    n = (ctypes.c_longlong * len(KINDS))()
    _check(_lib.sph_profile_read(h, ctypes.cast(ms, _vp), ctypes.cast(n, _vp), len(KINDS)), h)
    return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(KINDS)}


SPH_STATIC_MAX_PARTICLES = 1 << 22
SPH_STATIC_MAX_CELLS = 1 << 20


def sph_bin_static(params: dict, n: int, pos_ptr, keys_ptr, perm_ptr, cell_start_ptr, stream: int, flags_ptr=None):
    """Allocation-free binning (no device allocation; fixed static scratch).
    flags_ptr: optional device word receiving the call's flags."""
    q = dict(params)
    if q.get("mass") is None:
        q["mass"] = 1.0
    _check(_lib.sph_bin_static(ctypes.byref(make_params(q)), n, pos_ptr, keys_ptr, perm_ptr, cell_start_ptr,
                               flags_ptr, stream))


SPH_MLP_IN, SPH_MLP_HIDDEN, SPH_MLP_OUT, SPH_MLP_PARAMS = 272, 256, 16, 205584


def sph_mlp_workspace_size(max_batch: int) -> int:
    out = _sz()
    _check(_lib.sph_mlp_workspace_size(max_batch, ctypes.byref(out)))
    return int(out.value)


def sph_mlp_create(max_batch: int, workspace_ptr: int, ws_bytes: int):
    h = _vp()
    _check(_lib.sph_mlp_create(max_batch, workspace_ptr, ws_bytes, ctypes.byref(h)))
    return h


def sph_mlp_destroy(m):
    _lib.sph_mlp_destroy(m)


def sph_mlp_set_params(m, params_ptr: int, stream: int):
    _check(_lib.sph_mlp_set_params(m, params_ptr, stream))


def sph_mlp_get_params(m, params_ptr: int, stream: int):
    _check(_lib.sph_mlp_get_params(m, params_ptr, stream))


def sph_mlp_set_optimizer_state(m, m1_ptr: int, m2_ptr: int, step: int, stream: int):
    _check(_lib.sph_mlp_set_optimizer_state(m, m1_ptr, m2_ptr, int(step), stream))


def sph_mlp_get_optimizer_state(m, grads_ptr: int, m1_ptr: int, m2_ptr: int, stream: int) -> int:
    step = ctypes.c_longlong()
    _check(_lib.sph_mlp_get_optimizer_state(m, grads_ptr, m1_ptr, m2_ptr, ctypes.byref(step), stream))
    return int(step.value)


def sph_mlp_forward(m, x_ptr: int, B: int, y_ptr: int, stream: int):
    _check(_lib.sph_mlp_forward(m, x_ptr, B, y_ptr, stream))


def sph_mlp_gradients(m, x_ptr: int, dy_ptr: int, B: int, grads_ptr: int, stream: int):
    _check(_lib.sph_mlp_gradients(m, x_ptr, dy_ptr, B, grads_ptr, stream))


def sph_mlp_train_step(m, x_ptr: int, t_ptr: int, B: int, phase: int, lr: float, loss_ptr, stream: int):
    _check(_lib.sph_mlp_train_step(m, x_ptr, t_ptr, B, phase, lr, loss_ptr, stream))


def sph_mlp_status(m, stream: int) -> int:
    bits = ctypes.c_uint()
    _check(_lib.sph_mlp_status(m, ctypes.byref(bits), stream))
    return int(bits.value)


def sph_mlp_launch_count(m) -> int:
    return int(_lib.sph_mlp_launch_count(m))


def sph_set_obstacles(h, spheres, boxes, w_obst: float, near_factor: float, stream):
    """spheres (k, 4) and boxes (k, 6) as host float32 arrays (or None)."""
    sp = np.ascontiguousarray(np.asarray(spheres if spheres is not None else np.zeros((0, 4)), np.float32)
                              .reshape(-1, 4))
    bx = np.ascontiguousarray(np.asarray(boxes if boxes is not None else np.zeros((0, 6)), np.float32)
                              .reshape(-1, 6))
    _check(_lib.sph_set_obstacles(h, sp.ctypes.data_as(_vp) if len(sp) else None, len(sp),
                                  bx.ctypes.data_as(_vp) if len(bx) else None, len(bx), float(w_obst),
                                  float(near_factor), stream), h)


def sph_voxel_grid(params: dict, spacing: float, radius: float):
    """(origin (3 floats), dims (3 ints)) of the corner grid over the box."""
    o = (ctypes.c_float * 3)()
    d = (ctypes.c_int * 3)()
    _check(_lib.sph_voxel_grid(ctypes.byref(make_params(params)), float(spacing), float(radius),
                               ctypes.cast(o, _vp), ctypes.cast(d, _vp)))
    return tuple(float(x) for x in o), tuple(int(x) for x in d)


def sph_voxel_density(h, origin, dims, spacing: float, radius: float, particle_radius: float, phi_ptr,
                      counts_ptr, stream):
    o = (ctypes.c_float * 3)(*[float(x) for x in origin])
    d = (ctypes.c_int * 3)(*[int(x) for x in dims])
    _check(_lib.sph_voxel_density(h, ctypes.cast(o, _vp), ctypes.cast(d, _vp), float(spacing), float(radius),
                                  float(particle_radius), phi_ptr, counts_ptr, stream), h)


def sph_mc_workspace_size(dims) -> int:
    d = (ctypes.c_int * 3)(*[int(x) for x in dims])
    out = _sz()
    _check(_lib.sph_mc_workspace_size(ctypes.cast(d, _vp), ctypes.byref(out)))
    return int(out.value)


def sph_marching_cubes(phi_ptr, dims, origin, spacing: float, iso: float, ws_ptr, ws_bytes: int, tris_ptr,
                       max_tris: int, ntri_ptr, stream):
    d = (ctypes.c_int * 3)(*[int(x) for x in dims])
    o = (ctypes.c_float * 3)(*[float(x) for x in origin])
    _check(_lib.sph_marching_cubes(phi_ptr, ctypes.cast(d, _vp), ctypes.cast(o, _vp), float(spacing), float(iso),
                                   ws_ptr, ws_bytes, tris_ptr, int(max_tris), ntri_ptr, stream))


def sph_mc_tables():
    """(edge_table uint16 [256], tri_table int8 [256, 16]) as numpy arrays."""
    e = np.zeros(256, np.uint16)
    t = np.zeros((256, 16), np.int8)
    _check(_lib.sph_mc_tables(e.ctypes.data_as(_vp), t.ctypes.data_as(_vp)))
    return e, t


def marching_cubes(phi, dims, origin, spacing: float, iso: float = 0.0, max_tris: int | None = None):
    """Triangles of the iso-surface of a device float32 corner grid:
    returns (tris, total), tris a (min(total, max_tris), 3, 3) float32
    tensor on phi's device (default capacity: 5 per cube)."""
    import torch

    ncubes = max(0, (dims[0] - 1) * (dims[1] - 1) * (dims[2] - 1))
    cap = 5 * ncubes if max_tris is None else int(max_tris)
    ws_bytes = sph_mc_workspace_size(dims)
    ws = torch.empty(ws_bytes + 256, dtype=torch.uint8, device=phi.device)
    ws_ptr = (ws.data_ptr() + 255) & ~255
    tris = torch.empty((max(cap, 1), 3, 3), dtype=torch.float32, device=phi.device)
    ntri = torch.zeros(1, dtype=torch.int32, device=phi.device)
    stream = torch.cuda.current_stream(phi.device).cuda_stream
    sph_marching_cubes(phi.data_ptr(), dims, origin, spacing, iso, ws_ptr, ws_bytes, tris.data_ptr(), cap,
                       ntri.data_ptr(), stream)
    total = int(ntri.item()) & 0xFFFFFFFF
    return tris[:min(total, cap)], total


def sph_debug_gelu(z_ptr, n: int, grad: int, out_ptr, stream):
    _check(_lib.sph_debug_gelu(z_ptr, n, grad, out_ptr, stream))


def sph_debug_gemm(a_ptr, lda, b_ptr, ldb, M, N, K, splits, c_ptr, err_ptr, stream):
    _check(_lib.sph_debug_gemm(a_ptr, lda, b_ptr, ldb, M, N, K, splits, c_ptr, err_ptr, stream))


class Mlp:
    """The surrogate MLP with its workspace in a torch tensor.  Inputs are
    torch tensors on the device: x bfloat16 [B][272], targets float32 [B][4];
    B is padded up to a multiple of 128 inside (padded rows are zero and
    their outputs dropped; padded targets are zero with zero input, so they
    add nothing but a constant to the loss)."""

    def __init__(self, max_batch: int, device="cuda"):
        import torch

        self.torch = torch
        self.device = torch.device(device)
        self.max_batch = (int(max_batch) + 127) // 128 * 128
        nbytes = sph_mlp_workspace_size(self.max_batch)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        self._ws = (self.workspace.data_ptr() + 255) & ~255
        self.handle = sph_mlp_create(self.max_batch, self._ws, nbytes)
        self.loss = torch.zeros(1, dtype=torch.float32, device=self.device)

    @property
    def launches(self) -> int:
        return sph_mlp_launch_count(self.handle)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None:
            sph_mlp_destroy(h)
            self.handle = None

    @property
    def stream(self) -> int:
        return self.torch.cuda.current_stream(self.device).cuda_stream

    def _pad(self, x, width, dtype):
        t = self.torch
        B = x.shape[0]
        Bp = (B + 127) // 128 * 128
        if Bp == B and x.dtype == dtype and x.is_contiguous():
            return x, B
        out = t.zeros((Bp, width), dtype=dtype, device=self.device)
        out[:B] = x
        return out, B

    def set_params(self, params):
        p = self.torch.as_tensor(params, dtype=self.torch.float32, device=self.device).contiguous()
        assert p.numel() == SPH_MLP_PARAMS
        self._params = p
        sph_mlp_set_params(self.handle, p.data_ptr(), self.stream)

    def get_params(self):
        p = self.torch.empty(SPH_MLP_PARAMS, dtype=self.torch.float32, device=self.device)
        sph_mlp_get_params(self.handle, p.data_ptr(), self.stream)
        return p

    def optimizer_state(self):
        """(last gradient, first moment, second moment, step count)."""
        t = self.torch
        g, m1, m2 = (t.empty(SPH_MLP_PARAMS, dtype=t.float32, device=self.device) for _ in range(3))
        step = sph_mlp_get_optimizer_state(self.handle, g.data_ptr(), m1.data_ptr(), m2.data_ptr(), self.stream)
        return g, m1, m2, step

    def state_dict(self):
        """A training checkpoint of plain tensors (device copies): the FP32
        parameters, both Adam moments and the step count."""
        _g, m1, m2, step = self.optimizer_state()
        return {"params": self.get_params(), "adam_m1": m1, "adam_m2": m2,
                "adam_step": self.torch.tensor(step, dtype=self.torch.int64)}

    def load_state_dict(self, sd):
        """Restore a checkpoint of state_dict: later train steps are bit for
        bit those the saved network would have taken."""
        t = self.torch
        self.set_params(sd["params"])
        m1 = t.as_tensor(sd["adam_m1"], dtype=t.float32, device=self.device).contiguous()
        m2 = t.as_tensor(sd["adam_m2"], dtype=t.float32, device=self.device).contiguous()
        assert m1.numel() == SPH_MLP_PARAMS and m2.numel() == SPH_MLP_PARAMS
        self._moments = (m1, m2)  # alive until the copies on the stream have run
        sph_mlp_set_optimizer_state(self.handle, m1.data_ptr(), m2.data_ptr(), int(sd["adam_step"]), self.stream)

    def forward(self, x):
        xp, B = self._pad(x, SPH_MLP_IN, self.torch.bfloat16)
        y = self.torch.empty((xp.shape[0], SPH_MLP_OUT), dtype=self.torch.float32, device=self.device)
        sph_mlp_forward(self.handle, xp.data_ptr(), xp.shape[0], y.data_ptr(), self.stream)
        return y[:B]

    def gradients(self, x, dy):
        xp, B = self._pad(x, SPH_MLP_IN, self.torch.bfloat16)
        dyp, _ = self._pad(dy, SPH_MLP_OUT, self.torch.float32)
        g = self.torch.empty(SPH_MLP_PARAMS, dtype=self.torch.float32, device=self.device)
        sph_mlp_gradients(self.handle, xp.data_ptr(), dyp.data_ptr(), xp.shape[0], g.data_ptr(), self.stream)
        return g

    def train_step(self, x, t, lr, phase=0):
        """One Adam step; returns the loss tensor (device, not synchronised)."""
        assert x.shape[0] % 128 == 0, "training batches are multiples of 128"
        sph_mlp_train_step(self.handle, x.data_ptr(), t.data_ptr(), x.shape[0], phase, float(lr),
                           self.loss.data_ptr(), self.stream)
        return self.loss

    def status(self) -> int:
        return sph_mlp_status(self.handle, self.stream)


# ------------------------------------------------------ torch convenience

class Scene:
    """A scene whose workspace and state live in torch tensors on ``device``.

    Inputs are float32 ``(n, 4)`` arrays (numpy or torch); outputs are torch
    tensors on the device.  All calls use torch's current stream."""

    def __init__(self, params, n_fluid, n_boid, device="cuda", diagnostics=False):
        """One scene (params a dict, counts ints) or a batch (params a list
        of dicts, counts lists); a batch concatenates the scenes' arrays.
        diagnostics: the steps record acc, touched and influence."""
        import torch

        self.torch = torch
        batch = isinstance(params, (list, tuple))
        self.params_list = [dict(p) for p in params] if batch else [dict(params)]
        self.params = self.params_list[0]
        nf = list(n_fluid) if batch else [int(n_fluid)]
        nbl = list(n_boid) if batch else [int(n_boid)]
        self.scene_n_fluid, self.scene_n_boid = nf, nbl
        self.n_fluid, self.n_boid = int(sum(nf)), int(sum(nbl))
        self.n = self.n_fluid + self.n_boid
        self.device = torch.device(device)
        nbytes = sph_batch_workspace_size(self.params_list, nf, nbl)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        self._ws_ptr = (base + 255) & ~255
        self.handle = sph_batch_create(self.params_list, nf, nbl, self._ws_ptr, nbytes)
        dims = [sph_grid_dims(p, 0) for p in self.params_list]
        bdims = [sph_grid_dims(p, 1) for p in self.params_list]
        self.dims, self.bdims = dims[0], bdims[0]
        self.ncells = int(sum(d[0] * d[1] * d[2] for d in dims))
        self.nbcells = int(sum(d[0] * d[1] * d[2] for d in bdims))
        self.tuning = (256, 1)  # the library's default (block, use_segments)
        self.ppt = 1
        self.pipeline = (0, 256)  # separate neighbour-pass launches
        self.diagnostics = False
        if diagnostics:
            self.set_diagnostics(True)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None:
            sph_destroy(h)
            self.handle = None

    @property
    def stream(self) -> int:
        return self.torch.cuda.current_stream(self.device).cuda_stream

    def _dev4(self, a, n):
        t = self.torch.as_tensor(np.asarray(a, np.float32) if not self.torch.is_tensor(a) else a)
        t = t.to(device=self.device, dtype=self.torch.float32).reshape(n, 4).contiguous()
        return t

    def set_state(self, fluid_pos, fluid_vel, boid_pos, boid_vel):
        ts = [self._dev4(fluid_pos, self.n_fluid), self._dev4(fluid_vel, self.n_fluid),
              self._dev4(boid_pos, self.n_boid), self._dev4(boid_vel, self.n_boid)]
        self._keep = ts
        sph_set_state(self.handle, *[t.data_ptr() if t.numel() else None for t in ts], 0, self.stream)

    def set_state_host(self, fluid_pos, fluid_vel, boid_pos, boid_vel):
        """Upload from (preferably pinned) host tensors; synchronises the stream."""
        ts = [fluid_pos, fluid_vel, boid_pos, boid_vel]
        sph_set_state(self.handle, *[t.data_ptr() if t.numel() else None for t in ts], 1, self.stream)

    def get_state(self):
        t = self.torch
        out = [t.empty((self.n_fluid, 4), dtype=t.float32, device=self.device),
               t.empty((self.n_fluid, 4), dtype=t.float32, device=self.device),
               t.empty((self.n_boid, 4), dtype=t.float32, device=self.device),
               t.empty((self.n_boid, 4), dtype=t.float32, device=self.device)]
        sph_get_state(self.handle, *[o.data_ptr() if o.numel() else None for o in out], 0, self.stream)
        return out

    def get_state_host(self, outs):
        """Download into host tensors (pinned for speed); synchronises the stream."""
        sph_get_state(self.handle, *[o.data_ptr() if o.numel() else None for o in outs], 1, self.stream)

    def step(self, nsteps: int = 1):
        sph_step(self.handle, nsteps, self.stream)

    def graph_step(self, nsteps: int = 1):
        """sph_step replayed from a captured CUDA graph (non-default stream)."""
        sph_graph_step(self.handle, nsteps, self.stream)

    def set_neighbor_lists(self, max_pairs: int):
        """Keep a device pair buffer of max_pairs entries and build neighbour
        lists every step (0 turns them off)."""
        if max_pairs > 0:
            self.pair_buffer = self.torch.empty(int(max_pairs), dtype=self.torch.int32, device=self.device)
            sph_set_neighbor_lists(self.handle, self.pair_buffer.data_ptr(), 4 * int(max_pairs))
        else:
            sph_set_neighbor_lists(self.handle, None, 0)
            self.pair_buffer = None

    def bucket_neighbors(self, capacity: int):
        """Neighbour counts by particle id through the lossy fixed-capacity
        hash grid, and the number of particles its buckets dropped."""
        t = self.torch
        scratch = t.empty(self.ncells * (1 + capacity), dtype=t.int32, device=self.device)
        counts = t.empty(self.n, dtype=t.int32, device=self.device)
        dropped = t.zeros(1, dtype=t.int64, device=self.device)
        sph_debug_bucket_neighbors(self.handle, scratch.data_ptr(), 4 * scratch.numel(), capacity,
                                   counts.data_ptr(), dropped.data_ptr(), self.stream)
        return counts, dropped

    def set_tuning(self, block: int, use_segments: int):
        sph_set_tuning(self.handle, block, use_segments)
        self.tuning = (int(block), int(use_segments))

    def set_particles_per_thread(self, ppt: int):
        """Particles per thread of the separate neighbour-pass launches."""
        sph_set_particles_per_thread(self.handle, ppt)
        self.ppt = int(ppt)

    def set_pipeline(self, tile_slots: int, block: int = 256):
        """Both neighbour passes in one persistent launch over tiles of
        tile_slots sorted slots (0: separate launches)."""
        sph_set_pipeline(self.handle, tile_slots, block)
        self.pipeline = (int(tile_slots), int(block))

    def set_diagnostics(self, record: bool):
        """Record acc, touched and influence in later steps (off by default)."""
        sph_set_diagnostics(self.handle, int(bool(record)))
        self.diagnostics = bool(record)

    def field(self, name: str):
        t = self.torch
        code, dtype, width = FIELDS[name]
        if name == "cell_start":
            n = self.ncells + 1
        elif name == "boid_cell_start":
            n = self.nbcells + 1
        elif name == "obstacle_grid":
            n = self.nbcells
        elif name in ("fb", "boid_keys", "boid_perm", "fallback", "att_vel"):
            n = self.n_boid
        else:
            n = self.n
        tdtype = {np.float32: t.float32, np.int32: t.int32, np.uint32: t.int32}[dtype]
        out = t.empty((n, width) if width > 1 else (n,), dtype=tdtype, device=self.device)
        if out.numel():
            sph_get_fields(self.handle, code, out.data_ptr(), 0, self.stream)
        return out

    def stats(self):
        """Per-scene statistics of the most recent step (sph_stats): a float64
        (scenes, SPH_STATS_N) tensor on the device, columns named by STATS."""
        t = self.torch
        out = t.empty((len(self.params_list), SPH_STATS_N), dtype=t.float64, device=self.device)
        sph_stats(self.handle, out.data_ptr(), 0, self.stream)
        return out

    def boid_forces(self, mode: int = 0):
        """F_b of every boid for the current state (SPH_BOID_* mode)."""
        t = self.torch
        out = t.empty((self.n_boid, 4), dtype=t.float32, device=self.device)
        sph_boid_forces(self.handle, mode, out.data_ptr() if out.numel() else None, self.stream)
        return out

    def graph_boid_forces(self, mode: int = 0):
        """boid_forces replayed from a captured CUDA graph (non-default
        stream).  Returns this mode's output buffer, which the next call of
        the same mode overwrites."""
        t = self.torch
        bufs = self.__dict__.setdefault("_graph_out", {})
        if mode not in bufs:
            bufs[mode] = t.empty((self.n_boid, 4), dtype=t.float32, device=self.device)
        out = bufs[mode]
        sph_graph_boid_forces(self.handle, mode, out.data_ptr() if out.numel() else None, self.stream)
        return out

    def set_obstacles(self, spheres=None, boxes=None, w_obst: float = 0.05, near_factor: float = 2.0):
        """Analytic obstacles the boids avoid (spheres (k, 4), boxes (k, 6));
        none turns obstacle avoidance off."""
        sph_set_obstacles(self.handle, spheres, boxes, w_obst, near_factor, self.stream)

    def voxel_density(self, spacing: float, radius: float, particle_radius: float, counts: bool = True):
        """phi and neighbour counts on the corner grid over the box (sph_voxel_grid):
        returns (phi (nz, ny, nx) float32, counts or None, origin, dims)."""
        t = self.torch
        origin, dims = sph_voxel_grid(self.params, spacing, radius)
        n = dims[0] * dims[1] * dims[2]
        phi = t.empty(n, dtype=t.float32, device=self.device)
        cnt = t.empty(n, dtype=t.int32, device=self.device) if counts else None
        sph_voxel_density(self.handle, origin, dims, spacing, radius, particle_radius, phi.data_ptr(),
                          cnt.data_ptr() if counts else None, self.stream)
        return phi, cnt, origin, dims

    def features(self):
        """Stencil features of every boid (BF16 [n_boid][272])."""
        t = self.torch
        x = t.empty((self.n_boid, SPH_MLP_IN), dtype=t.bfloat16, device=self.device)
        sph_features(self.handle, x.data_ptr() if x.numel() else None, self.stream)
        return x

    def set_surrogate(self, mlp, f_scale: float, log_err_max: float, bounds=None):
        """Attach the surrogate network; bounds = (lo, hi), SPH_MLP_IN floats
        each, turns on the gate's input-range check (None: off)."""
        self._mlp = mlp
        sph_set_surrogate(self.handle, mlp.handle if mlp is not None else None, f_scale, log_err_max)
        self.set_surrogate_bounds(bounds)

    def set_surrogate_bounds(self, bounds):
        t = self.torch
        if bounds is None:
            self._bounds = None
            sph_set_surrogate_bounds(self.handle, None, None)
            return
        lo, hi = (t.as_tensor(v, dtype=t.float32).to(self.device).contiguous() for v in bounds)
        if lo.numel() != SPH_MLP_IN or hi.numel() != SPH_MLP_IN:
            raise ValueError(f"bounds need {SPH_MLP_IN} floats each")
        self._bounds = (lo, hi)  # the library keeps the pointers
        sph_set_surrogate_bounds(self.handle, lo.data_ptr(), hi.data_ptr())

    def neighbors(self, lists: bool = True):
        t = self.torch
        counts = t.zeros(self.n, dtype=t.int32, device=self.device)
        sph_debug_neighbors(self.handle, counts.data_ptr(), None, None, self.stream)
        if not lists:
            return counts, None, None
        offsets = t.zeros(self.n + 1, dtype=t.int64, device=self.device)
        offsets[1:] = t.cumsum(counts.to(t.int64), 0)
        total = int(offsets[-1].item())
        lst = t.zeros(max(total, 1), dtype=t.int32, device=self.device)
        sph_debug_neighbors(self.handle, counts.data_ptr(), offsets.data_ptr(), lst.data_ptr(), self.stream)
        return counts, offsets, lst[:total]

    def status(self) -> int:
        return sph_status(self.handle)

    def clear_status(self):
        sph_clear_status(self.handle, self.stream)

    @property
    def launches(self) -> int:
        return sph_launch_count(self.handle)
