"""Helpers of the GPU-vs-oracle parity tests (test infrastructure).

Tolerances (one step, same float32 input state; the oracle in double):
  keys, perm, cell_start, neighbour counts/lists, touched    bit-exact
  rho        |d| <= 1e-5 rho
  pressure   |d| <= 1e-5 k rho          (p cancels near rho0)
  acc, F_b, boid_influence
             |d| <= 1e-5 S_i per particle, S_i = (1/rho_i) sum_j m/rho_j
             [C_p (|p_i| + |p_j|)/2 h (1-q) + C_v mu |v_ij| (1 - q/2)] + |g|:
             per term its magnitude plus r^2 |d term / d r^2| (the float32
             squared distance is rounded and 1 - q cancels at the kernel
             edge), summed in magnitude (interior forces cancel, and so does
             p_i + p_j where rho_i < rho0 < rho_j); and
             ||d||_2 / ||a||_2 <= 1e-5 over the field
  v after    |d| <= 1e-5 (|v| + dt S_i)
  x after    |d| <= 2.4e-7 |x| + dt 1e-5 (|v| + dt S_i): the velocity error
             times dt plus two float32 roundings of x
  boids      |d v| <= 1e-5 V_b, V_b the sum of the magnitudes of the rule
             terms; x as above with V_b
Wall decisions: where the oracle's pre-wall position lies within the
position tolerance of a wall, either side of the decision is accepted.
"""
import numpy as np

import oracle
from paper_2311_15088_gb300.sph import Scene

REL = 1e-5


def _ratio(a, b):
    """a / b with 0 / 0 = 0 (both sides exactly zero)."""
    return np.divide(a, b, out=np.where(a > 0, np.inf, 0.0), where=b > 0)


def run_gpu(p, sc, steps=1, device="cuda"):
    s = Scene(p, len(sc["fluid_pos"]), len(sc["boid_pos"]), device=device, diagnostics=True)
    s.set_state(sc["fluid_pos"], sc["fluid_vel"], sc["boid_pos"], sc["boid_vel"])
    s.step(steps)
    return s


def gpu_outputs(s):
    out = {}
    for name in ("rho", "pressure", "acc", "touched", "influence", "nbr_count", "keys", "perm",
                 "cell_start", "fb", "boid_keys", "boid_perm", "boid_cell_start"):
        out[name] = s.field(name).cpu().numpy()
    fp, fv, bp, bv = (t.cpu().numpy() for t in s.get_state())
    out.update(new_fluid_pos=fp[:, :3], new_fluid_vel=fv[:, :3], new_boid_pos=bp[:, :3], new_boid_vel=bv[:, :3])
    out["keys"] = out["keys"].view(np.uint32)
    out["cell_start"] = out["cell_start"].view(np.uint32)
    out["boid_keys"] = out["boid_keys"].view(np.uint32)
    out["boid_cell_start"] = out["boid_cell_start"].view(np.uint32)
    return out


def compare_step(p, g, o, nb, check_boids=True):
    """Assert every field of one GPU step against the oracle's step."""
    n = len(o["rho"])
    # binning and counters: bit-exact
    assert np.array_equal(g["keys"], o["keys"]), "keys differ"
    assert np.array_equal(g["perm"], o["perm"]), "sorted order differs"
    assert np.array_equal(g["cell_start"], o["cell_start"].astype(np.uint32)), "cell_start differs"
    assert np.array_equal(g["nbr_count"], o["nbr_count"]), "neighbour counts differ"
    assert np.array_equal(g["touched"], o["touched"]), "touched_by_boid differs"
    # density and pressure
    drho = np.abs(g["rho"] - o["rho"])
    assert np.all(drho <= REL * o["rho"]), f"rho: max rel {np.max(drho / o['rho']):.3e}"
    dp = np.abs(g["pressure"] - o["pressure"])
    assert np.all(dp <= REL * p["k"] * o["rho"] + 1e-30), f"pressure: max {np.max(dp / (p['k'] * o['rho'])):.3e}"
    # accelerations (fluid) and F_b (attached)
    S = o["acc_scale"]
    da = np.abs(g["acc"][:, :3] - o["acc"])
    ok = da.max(axis=1) <= REL * S if n else np.ones(0, bool)
    assert np.all(ok), f"acc differs at ids {np.flatnonzero(~ok)[:5]}: |d|/S = {_ratio(da.max(1), S)[~ok][:5]}"
    if n:
        l2 = np.linalg.norm(da) / max(np.linalg.norm(o["acc"]), 1e-300)
        assert l2 <= REL, f"acc: field L2 rel {l2:.3e}"
    dinf = np.abs(g["influence"][:, :3] - o["influence"]).max(axis=1) if n else np.zeros(0)
    assert np.all(dinf <= REL * S), "boid_influence differs"
    if nb:
        dfb = np.abs(g["fb"][:, :3] - o["fb"]).max(axis=1)
        assert np.all(dfb <= REL * S[:nb]), f"F_b: max {np.max(_ratio(dfb, S[:nb])):.3e}"
    # integrated fluid state
    nf = len(o["new_fluid_pos"])
    if nf:
        dt = p["dt"]
        Sf = S[nb:]
        vref = o["new_fluid_vel"]
        tol_v = REL * (np.abs(vref) + dt * Sf[:, None])
        tol_x = 2.4e-7 * np.abs(o["new_fluid_pos"]) + dt * tol_v
        amb = o["wall_margin"] < tol_x.max(axis=1) * 4
        dv = np.abs(g["new_fluid_vel"] - vref)
        dx = np.abs(g["new_fluid_pos"] - o["new_fluid_pos"])
        ok_v = np.all(dv <= tol_v, axis=1)
        ok_x = np.all(dx <= tol_x, axis=1)
        if amb.any():
            gv, pre, cr = g["new_fluid_vel"], o["pre_wall_vel"], p["wall_restitution"]
            comp_ok = (dv <= tol_v) | (np.abs(gv - pre) <= tol_v) | (np.abs(gv + cr * pre) <= tol_v)
            ok_v = ok_v | (amb & np.all(comp_ok, axis=1))
            ok_x = ok_x | (amb & np.all(dx <= tol_x + 2 * o["wall_margin"][:, None], axis=1))
        assert np.all(ok_v), f"fluid velocity differs at {np.flatnonzero(~ok_v)[:5]}"
        assert np.all(ok_x), f"fluid position differs at {np.flatnonzero(~ok_x)[:5]}"
    if nb and check_boids:
        assert np.array_equal(g["boid_keys"], o["boid_keys"]), "boid keys differ"
        assert np.array_equal(g["boid_perm"], o["boid_perm"]), "boid order differs"
        assert np.array_equal(g["boid_cell_start"], o["boid_cell_start"].astype(np.uint32))
        V = o["boid_vscale"]
        dvb = np.abs(g["new_boid_vel"] - o["new_boid_vel"]).max(axis=1)
        assert np.all(dvb <= REL * V), f"boid velocity: max {np.max(_ratio(dvb, V)):.3e}"
        dxb = np.abs(g["new_boid_pos"] - o["new_boid_pos"]).max(axis=1)
        assert np.all(dxb <= 2.4e-7 * np.abs(o["new_boid_pos"]).max(axis=1) + p["dt"] * REL * V), "boid position"


def oracle_step(p, sc):
    return oracle.step(p, sc["fluid_pos"], sc["fluid_vel"], sc["boid_pos"], sc["boid_vel"])


def lattice_params(sc):
    p = dict(sc["params"])
    if p.get("mass") is None:
        p["mass"] = float(np.float32(oracle.lattice_mass(p, sc["lattice_spacing"])))
    return p
