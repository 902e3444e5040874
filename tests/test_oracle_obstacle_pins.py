"""The oracle's obstacle grid and obstacle avoidance pinned to geometry and
to hand-computed cases (CPU)."""
import math

import numpy as np
import pytest

import oracle
from paper_2311_15088_gb300 import scenes


def _params():
    p = scenes.default_params(mass=scenes.f32(0.01))
    return p


def _centres(p):
    dims = oracle.grid_dims(p, 1)
    d = np.float32(p["boid_cell_size"])
    mn = np.asarray(p["box_min"], np.float32)
    idx = np.arange(dims[0] * dims[1] * dims[2])
    ijk = np.stack([idx % dims[0], (idx // dims[0]) % dims[1], idx // (dims[0] * dims[1])], 1)
    return (((ijk.astype(np.float32) + np.float32(0.5)) * d).astype(np.float32) + mn).astype(np.float32), dims


def test_sphere_cells_hold_the_radial_normal():
    p = _params()
    c, r = np.array([0.5, 0.45, 0.55], np.float32), np.float32(0.3)
    g = oracle.obstacle_grid(p, spheres=[[*c, r]])
    X, _ = _centres(p)
    d = X.astype(np.float64) - c
    dist = np.linalg.norm(d, axis=1) - float(r)
    half = float(np.float32(0.866025403784) * np.float32(p["boid_cell_size"]))
    on = g[:, 3] > 0
    # cells whose centre is clearly within / beyond half a diagonal of the surface
    assert np.all(on[np.abs(dist) < half - 1e-6]) and not np.any(on[np.abs(dist) > half + 1e-6])
    n = d[on] / np.linalg.norm(d[on], axis=1)[:, None]
    assert np.allclose(g[on, :3], n, atol=1e-12)
    assert np.all(g[on, 3] == 1)


def test_box_cells_hold_face_and_corner_normals():
    p = _params()
    lo, hi = np.array([0.3, 0.2, 0.3], np.float32), np.array([0.7, 0.5, 0.6], np.float32)
    g = oracle.obstacle_grid(p, boxes=[[*lo, *hi]])
    X, _ = _centres(p)
    on = g[:, 3] > 0
    assert on.sum() > 10
    for x, v in zip(X[on].astype(np.float64), g[on]):
        nrm = v[:3]
        assert abs(np.linalg.norm(nrm) - 1.0) < 1e-12
        inside = np.all((x >= lo) & (x <= hi))
        if inside:  # the nearest face's outward normal: one axis, +-1
            ax = int(np.argmax(np.abs(nrm)))
            assert abs(nrm[ax]) == 1.0 and np.count_nonzero(nrm) == 1
            near = min(x[ax] - lo[ax], hi[ax] - x[ax])
            assert near <= min(min(x[a] - lo[a], hi[a] - x[a]) for a in range(3)) + 1e-7
            assert (nrm[ax] > 0) == (hi[ax] - x[ax] <= x[ax] - lo[ax])
        else:  # points from the nearest surface point to the centre
            q = np.clip(x, lo, hi)
            assert np.allclose(nrm, (x - q) / np.linalg.norm(x - q), atol=1e-7)


def test_two_obstacles_in_a_cell_average_their_normals():
    p = _params()
    X, _ = _centres(p)
    k = 2 + 6 * (3 + 6 * 2)  # cell (2, 3, 2) of the 6^3 boid grid
    x = X[k].astype(np.float64)
    # two spheres whose surfaces pass through that centre, from +x and from -x
    s1 = [x[0] + 0.1, x[1], x[2], 0.1]
    s2 = [x[0] - 0.1, x[1], x[2], 0.1]
    g = oracle.obstacle_grid(p, spheres=[s1, s2])
    assert g[k, 3] == 2
    assert np.allclose(g[k, :3], 0.0, atol=1e-6)  # the two normals cancel


def _one_boid_step(p, bpos, bvel, obstacles):
    z = np.zeros((0, 4), np.float32)
    return oracle.step(p, z, z, np.asarray([bpos], np.float32), np.asarray([bvel], np.float32), obstacles=obstacles)


def test_single_cell_in_range_gives_w_times_its_normal():
    """A boid with one obstacle cell in its visual range, outside its
    protection range: v gains w_obst * n (before the speed limit, which the
    chosen speed stays inside)."""
    p = _params()
    p.update(v_min=scenes.f32(0.0), v_max=scenes.f32(10.0))
    X, dims = _centres(p)
    k = 2 + dims[0] * (2 + dims[1] * 2)
    cell = X[k].astype(np.float64)
    sph = [cell[0] + 0.04, cell[1], cell[2], 0.04]  # surface through the cell's centre, normal -x
    g = oracle.obstacle_grid(p, spheres=[sph])
    assert g[k, 3] == 1
    rv, rs = float(p["r_vis"]), float(p["r_sep"])
    # a boid at distance between r_sep and r_vis from that centre and no other obstacle cell in range
    for dist in np.linspace(rs * 1.05, rv * 0.95, 40):
        b = cell + np.array([-dist, 0.0, 0.0])
        X64 = X.astype(np.float64)
        inr = (g[:, 3] > 0) & (np.linalg.norm(X64 - b, axis=1) < rv)
        if inr.sum() == 1:
            break
    else:
        pytest.skip("no position with a single obstacle cell in range")
    w = 0.05
    v0 = np.array([0.3, 0.0, 0.0, 0.0], np.float32)
    o_on = _one_boid_step(p, [*b, 0], v0, dict(spheres=[sph], w_obst=w, near_factor=2.0))
    o_off = _one_boid_step(p, [*b, 0], v0, None)
    dv = o_on["new_boid_vel"][0] - o_off["new_boid_vel"][0]
    n = g[inr][0, :3]
    assert np.allclose(dv, float(np.float32(w)) * n, atol=1e-12)


def test_protection_range_weighs_near_factor():
    p = _params()
    p.update(v_min=scenes.f32(0.0), v_max=scenes.f32(10.0))
    X, dims = _centres(p)
    k = 2 + dims[0] * (2 + dims[1] * 2)
    cell = X[k].astype(np.float64)
    sph = [cell[0] + 0.04, cell[1], cell[2], 0.04]
    g = oracle.obstacle_grid(p, spheres=[sph])
    X64 = X.astype(np.float64)
    rs = float(p["r_sep"])
    b = cell + np.array([-0.5 * rs, 0.0, 0.0])
    inr = (g[:, 3] > 0) & (np.linalg.norm(X64 - b, axis=1) < float(p["r_vis"]))
    near = inr & (np.linalg.norm(X64 - b, axis=1) < rs)
    assert near.sum() >= 1
    w, nf = 0.05, 3.0
    v0 = np.array([0.3, 0.0, 0.0, 0.0], np.float32)
    dv = (_one_boid_step(p, [*b, 0], v0, dict(spheres=[sph], w_obst=w, near_factor=nf))["new_boid_vel"][0]
          - _one_boid_step(p, [*b, 0], v0, None)["new_boid_vel"][0])
    wts = np.where(near[inr], nf, 1.0)
    want = float(np.float32(w)) * (wts[:, None] * g[inr, :3]).sum(0) / inr.sum()
    assert np.allclose(dv, want, atol=1e-12)


def test_boids_far_from_obstacles_are_unaffected_and_steer_away_when_near():
    p = _params()
    rng = np.random.default_rng(2)
    sph = [0.5, 0.5, 0.5, 0.15]
    far = rng.uniform(0.0, 1.0, (200, 3)).astype(np.float32)
    far = far[np.linalg.norm(far - 0.5, axis=1) > 0.15 + 0.0457 * 8 + 0.06][:20]
    bv = np.zeros((len(far), 4), np.float32)
    bv[:, 0] = 0.2
    z = np.zeros((0, 4), np.float32)
    bp = np.concatenate([far, np.zeros((len(far), 1), np.float32)], 1)
    a = oracle.step(p, z, z, bp, bv, obstacles=dict(spheres=[sph]))
    b = oracle.step(p, z, z, bp, bv)
    assert np.array_equal(a["new_boid_vel"], b["new_boid_vel"])
    # a boid heading into the sphere is turned outwards: its radial velocity grows
    x = np.array([[0.5 - 0.15 - 0.03, 0.5, 0.5, 0]], np.float32)
    v = np.array([[0.2, 0.0, 0.0, 0]], np.float32)
    on = oracle.step(p, z, z, x, v, obstacles=dict(spheres=[sph], w_obst=0.05))["new_boid_vel"][0]
    off = oracle.step(p, z, z, x, v)["new_boid_vel"][0]
    assert on[0] < off[0]  # pushed back along -x, away from the sphere
