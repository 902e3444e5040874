"""Pins of the CPU oracle against things other than itself (CPU only).

Each test checks the oracle against something the paper or the mathematics
fixes: closed forms, normalisation integrals, derivatives of independently
stated kernels, brute force, invariants and hand-solved cases.  A plausible
mistake in the oracle (a dropped term, a wrong sign, a swapped index, a
wrong constant) fails at least one of them.
"""
import math

import numpy as np
import pytest
from scipy import integrate

from paper_2311_15088_gb300 import scenes


def _params(**kw):
    p = scenes.default_params(**kw)
    if p["mass"] is None:
        p["mass"] = scenes.f32(0.01)
    return p


def _z4(n):
    return np.zeros((n, 4), np.float32)


def _p4(xyz):
    a = np.zeros((len(xyz), 4), np.float32)
    a[:, :3] = np.asarray(xyz, np.float32)
    return a


# ---------------------------------------------------------------- P7 RNG

def test_rng_generator_matches_c_stream(orc):
    """The numpy generator and the C copy of the paper's hash agree on every
    integer of 64 draws for 4096 streams."""
    seed = scenes.BASE_SEED
    ids = np.arange(4096) * 977 + 3
    rng = scenes.PaperHashRNG(seed, ids)
    draws = np.stack([rng.next_u32() for _ in range(64)], axis=1)
    for k in range(0, 4096, 97):
        assert np.array_equal(draws[k], orc.rng_stream(seed, int(ids[k]), 64))


def test_rng_first_draw_by_integer_arithmetic(orc):
    """First draw of stream s = 0 computed with Python integers."""
    M = (1 << 32) - 1
    s = 0 ^ 2747636419
    s = (s * 2654435769) & M
    s ^= s >> 16
    s = (s * 2654435769) & M
    s ^= s >> 16
    s = (s * 2654435769) & M
    assert orc.rng_stream(0, 0, 1)[0] == s


# ------------------------------------------------------------ P1 binning

def test_cell_of_positions_on_faces_and_outside(orc):
    """get_cell = floor((p - m)/d) clamped to the grid; d = 0.25 is exact in
    binary, so a point on a face belongs to the upper cell."""
    p = _params(cell_size=0.25, boid_cell_size=0.5)
    assert orc.grid_dims(p, 0) == (4, 4, 4)
    xs = [0.0, 0.25, 0.5, 0.9999, 1.0, -0.1, 1.3]
    expect = [0, 1, 2, 3, 3, 0, 3]
    pos = _p4([[x, 0.3, 0.8] for x in xs])
    keys, _, _ = orc.bin_particles(p, pos)
    # hash = cx + dim_x (cy + dim_y cz) with cy = 1, cz = 3
    assert list(keys) == [c + 4 * (1 + 4 * 3) for c in expect]


def test_hash_is_row_major_x_fastest(orc):
    p = _params(box_max=(0.75, 1.0, 1.25), cell_size=0.25, boid_cell_size=0.5)
    assert orc.grid_dims(p, 0) == (3, 4, 5)
    pts, expect = [], []
    for cz in range(5):
        for cy in range(4):
            for cx in range(3):
                pts.append([(cx + 0.5) * 0.25, (cy + 0.5) * 0.25, (cz + 0.5) * 0.25])
                expect.append(cx + 3 * (cy + 4 * cz))
    keys, perm, cs = orc.bin_particles(p, _p4(pts))
    assert list(keys) == expect
    assert list(perm) == list(range(len(pts)))
    assert list(cs) == list(range(len(pts) + 1))


def test_counting_sort_orders_by_key_then_id(orc):
    sc = scenes.scaled_block(3000, 0, (1.0, 1.0, 1.0), (0.3, 0.5, 0.4), seed=11)
    p = sc["params"]
    keys, perm, cs = orc.bin_particles(p, sc["fluid_pos"])
    ids = np.arange(len(keys))
    assert np.array_equal(perm, np.lexsort((ids, keys)))
    counts = np.bincount(keys, minlength=len(cs) - 1)
    assert cs[0] == 0 and np.array_equal(np.diff(cs), counts)


def _sets(counts, offsets, lst):
    return [set(lst[offsets[i]:offsets[i + 1]].tolist()) for i in range(len(counts))]


@pytest.mark.parametrize("n,n_att,cell", [(2500, 0, 1.0), (2000, 40, 1.0), (2500, 30, 0.5), (1500, 10, 0.34)])
def test_grid_neighbors_equal_brute_force(orc, n, n_att, cell):
    """The grid walk finds exactly the pairs an all-pairs scan finds, for
    cells of h, h/2 and about h/3, including particles pushed into the corner
    and edge cells."""
    sc = scenes.scaled_block(n, 0, (1.0, 1.0, 1.0), (1.0, 1.0, 1.0), seed=5)
    pos = sc["fluid_pos"].copy()
    # squeeze a third of them against the corners of the box
    k = n // 3
    pos[:k, :3] = np.where(pos[:k, :3] < 0.5, pos[:k, :3] * 0.08, 1.0 - (1.0 - pos[:k, :3]) * 0.08)
    p = dict(sc["params"], cell_size=scenes.f32(sc["params"]["h"] * cell))
    c1, o1, l1 = orc.neighbors(p, pos, n_att)
    c2, o2, l2 = orc.neighbors(p, pos, n_att, brute=True)
    assert np.array_equal(c1, c2)
    assert _sets(c1, o1, l1) == _sets(c2, o2, l2)
    assert c1.sum() > 10 * n  # the case is not trivially sparse
    if n_att:  # no pair of two attached particles
        for i in range(n_att):
            assert not any(j < n_att for j in l1[o1[i]:o1[i + 1]])


@pytest.mark.parametrize("cell,cell_x", [(0.5, 0.25), (1.0, 0.2), (0.34, 0.125)])
def test_grid_neighbors_equal_brute_force_narrow_x_cells(orc, cell, cell_x):
    """Cells narrower along x than along y and z (the walk then reaches
    ceil(h / dx) + 1 cells along x): still exactly the all-pairs set, with
    particles squeezed into the corners."""
    sc = scenes.scaled_block(2000, 20, (1.0, 1.0, 1.0), (1.0, 1.0, 1.0), seed=9)
    pos = sc["fluid_pos"].copy()
    k = 600
    pos[:k, :3] = np.where(pos[:k, :3] < 0.5, pos[:k, :3] * 0.08, 1.0 - (1.0 - pos[:k, :3]) * 0.08)
    h = sc["params"]["h"]
    p = dict(sc["params"], cell_size=scenes.f32(h * cell), cell_size_x=scenes.f32(h * cell_x))
    c1, o1, l1 = orc.neighbors(p, pos, 20)
    c2, o2, l2 = orc.neighbors(p, pos, 20, brute=True)
    assert np.array_equal(c1, c2)
    assert _sets(c1, o1, l1) == _sets(c2, o2, l2)
    assert c1.sum() > 10 * len(pos)


def test_narrow_x_cells_sort_by_the_x_cell(orc):
    """With cells h/4 wide along x and h/2 along y and z, a particle's key
    is floor((x - m) / dx) + dim_x (floor((y - m) / d) + dim_y floor((z - m)
    / d)) in float32, and dim_x = ceil(extent / dx)."""
    p = _params()
    h = np.float32(p["h"])
    p = dict(p, cell_size=scenes.f32(h / 2), cell_size_x=scenes.f32(h / 4), box_max=(1.0, 0.5, 0.5))
    dims = orc.grid_dims(p, 0)
    assert dims[0] == int(np.ceil(1.0 / np.float64(np.float32(h / 4))))
    assert dims[1] == int(np.ceil(0.5 / np.float64(np.float32(h / 2))))
    rng = np.random.default_rng(3)
    pos = _p4(rng.uniform(0.0, [1.0, 0.5, 0.5], size=(500, 3)).astype(np.float32))
    keys, perm, cs = orc.bin_particles(p, pos)
    inv_dx, inv_d = np.float32(1) / np.float32(h / 4), np.float32(1) / np.float32(h / 2)
    cx = np.minimum(np.floor(pos[:, 0] * inv_dx), dims[0] - 1).astype(np.int64)
    cy = np.minimum(np.floor(pos[:, 1] * inv_d), dims[1] - 1).astype(np.int64)
    cz = np.minimum(np.floor(pos[:, 2] * inv_d), dims[2] - 1).astype(np.int64)
    assert np.array_equal(keys, cx + dims[0] * (cy + dims[1] * cz))


def test_lattice_ties_at_exactly_h(orc):
    """Unjittered lattice of spacing h/2: pairs at exactly r = h in real
    arithmetic are decided by the float predicate; grid and brute force agree."""
    p = _params()
    s = np.float32(p["h"]) / np.float32(2)
    n = 10
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    pos = _p4(np.stack([i.ravel(), j.ravel(), k.ravel()], 1) * s + np.float32(0.3))
    c1, o1, l1 = orc.neighbors(p, pos)
    c2, o2, l2 = orc.neighbors(p, pos, brute=True)
    assert _sets(c1, o1, l1) == _sets(c2, o2, l2)


# ------------------------------------------------------------ P2 kernels

def _radial_integral(f, h, dim):
    if dim == 3:
        val, _ = integrate.quad(lambda r: 4 * math.pi * r * r * f(r), 0, h, limit=200)
    else:
        val, _ = integrate.quad(lambda r: 2 * math.pi * r * f(r), 0, h, limit=200)
    return val


def test_poly6_normalised_and_shape(orc):
    """poly6: integral over R^3 is 1; W is a cubic in r^2 with a triple root
    at r^2 = h^2 (the only such even degree-6 polynomial)."""
    p = _params()
    h = p["h"]
    assert abs(_radial_integral(lambda r: orc.w_poly6(p, r), h, 3) - 1.0) < 1e-9
    u = np.linspace(0.0, h * h, 9)
    w = np.array([orc.w_poly6(p, math.sqrt(x)) for x in u])
    coef = np.polyfit(u / (h * h), w / w[0], 3)
    assert np.allclose(np.polyval(coef, u / (h * h)), w / w[0], atol=1e-12)
    roots = np.roots(coef)
    assert np.allclose(roots, 1.0, atol=1e-4)
    assert orc.w_poly6(p, h * 1.0001) == 0.0


def _spiky(h, dim):
    c = 15.0 / (math.pi * h ** 6) if dim == 3 else 10.0 / (math.pi * h ** 5)
    return lambda r: c * (h - r) ** 3 if r < h else 0.0


def _visc3(h):
    c = 15.0 / (2 * math.pi * h ** 3)
    return lambda r: c * (-r ** 3 / (2 * h ** 3) + r * r / (h * h) + h / (2 * r) - 1.0) if r < h else 0.0


@pytest.mark.parametrize("const_set,dim", [(0, 3), (1, 2)])
def test_spiky_gradient_is_derivative_of_normalised_kernel(orc, const_set, dim):
    """The pressure kernel gradient -C_p (1-q)^2/q r equals the derivative of
    the spiky kernel normalised in 3-D (default) or in 2-D (the printed
    30/(pi h^4) constant)."""
    p = _params(const_set=const_set)
    h = p["h"]
    W = _spiky(h, dim)
    assert abs(_radial_integral(W, h, dim) - 1.0) < 1e-9
    for q in (0.1, 0.35, 0.6, 0.9):
        r = q * h
        e = 1e-7 * h
        dW = (W(r + e) - W(r - e)) / (2 * e)           # dW/dr; grad W = dW/dr * r_vec / r
        assert orc.grad_spiky_factor(p, r) == pytest.approx(dW / r, rel=1e-6)


def test_viscosity_laplacian_is_laplacian_of_normalised_kernel(orc):
    p = _params(const_set=0)
    h = p["h"]
    W = _visc3(h)
    assert abs(_radial_integral(W, h, 3) - 1.0) < 1e-7
    for q in (0.2, 0.5, 0.8):
        r = q * h
        e = 1e-4 * h
        d1 = (W(r + e) - W(r - e)) / (2 * e)
        d2 = (W(r + e) - 2 * W(r) + W(r - e)) / (e * e)
        assert orc.lap_visc(p, r) == pytest.approx(d2 + 2 * d1 / r, rel=1e-5)


def test_printed_constants_of_const_set_1(orc):
    """const_set 1 keeps the printed prefactors 30/(pi h^4) (spiky gradient)
    and 40/(pi h^4) (viscosity Laplacian), section "Pressure and Viscosity"."""
    p1, p0 = _params(const_set=1), _params(const_set=0)
    h = p0["h"]
    r = 0.4 * h
    q = 0.4
    assert orc.grad_spiky_factor(p1, r) == pytest.approx(-30 / (math.pi * h ** 4) * (1 - q) ** 2 / q, rel=1e-12)
    assert orc.lap_visc(p1, r) == pytest.approx(40 / (math.pi * h ** 4) * (1 - q), rel=1e-12)
    assert orc.lap_visc(p1, r) / orc.lap_visc(p0, r) == pytest.approx(40 * h / 45, rel=1e-12)


# ------------------------------------------------- P3 two-particle forces

def _two_particles(orc, p, r_vec, vi=(0, 0, 0), vj=(0, 0, 0)):
    xi = np.array([0.5, 0.5, 0.5], np.float32)
    xj = (xi + np.asarray(r_vec, np.float32)).astype(np.float32)
    pos = _p4([xj, xi])  # fluid index 1 is particle i
    vel = _p4([vj, vi])
    o = orc.step(p, pos, vel, _z4(0), _z4(0))
    xi64, xj64 = pos[1, :3].astype(np.float64), pos[0, :3].astype(np.float64)
    return o, xi64, xj64


@pytest.mark.parametrize("const_set,dim", [(0, 3), (1, 2)])
def test_two_particle_pressure_acceleration(orc, const_set, dim):
    """a_i = -(1/rho_i) m (p_i + p_j)/(2 rho_j) grad_i W_spiky(x_i - x_j),
    the gradient by central differences of the normalised spiky kernel."""
    p = _params(const_set=const_set, mu=0.0, gy=0.0, k=3.0, mass=0.02, rho0=500.0)
    h = p["h"]
    o, xi, xj = _two_particles(orc, p, np.array([0.3, -0.2, 0.15]) * h)
    rho_i, rho_j = o["rho"][1], o["rho"][0]
    assert rho_i == pytest.approx(rho_j, rel=1e-12)
    # density of the pair: m (W(0) + W(r)), W the normalised poly6
    r = np.linalg.norm(xi - xj)
    assert rho_i == pytest.approx(p["mass"] * (orc.w_poly6(p, 0) + orc.w_poly6(p, r)), rel=1e-12)
    pi_, pj_ = o["pressure"][1], o["pressure"][0]
    assert pi_ == pytest.approx(p["k"] * (rho_i - p["rho0"]), rel=1e-12)
    W = _spiky(h, dim)
    grad = np.zeros(3)
    e = 1e-6 * h
    for a in range(3):
        dxp, dxm = xi - xj, xi - xj
        dxp = dxp.copy(); dxp[a] += e
        dxm = dxm.copy(); dxm[a] -= e
        grad[a] = (W(np.linalg.norm(dxp)) - W(np.linalg.norm(dxm))) / (2 * e)
    expect = -(1 / rho_i) * p["mass"] * (pi_ + pj_) / (2 * rho_j) * grad
    assert np.allclose(o["acc"][1], expect, rtol=1e-6, atol=1e-9 * np.abs(expect).max())
    assert np.allclose(o["acc"][0], -o["acc"][1], rtol=1e-12)
    # repulsive when compressed (p > 0): a_i points from j to i
    assert (pi_ + pj_ > 0) == (np.dot(o["acc"][1], xi - xj) > 0)


def test_two_particle_viscous_acceleration(orc):
    """a_i = (1/rho_i) mu m (v_j - v_i)/rho_j lap W_visc(r), the Laplacian by
    finite differences of the normalised 3-D viscosity kernel."""
    p = _params(const_set=0, k=0.0, gy=0.0, mu=3.5, mass=0.02)
    h = p["h"]
    vi = (0.3, -0.2, 0.1)
    o, xi, xj = _two_particles(orc, p, np.array([0.1, 0.4, -0.2]) * h, vi=vi)
    r = np.linalg.norm(xi - xj)
    W = _visc3(h)
    e = 1e-4 * h
    lap = (W(r + e) - 2 * W(r) + W(r - e)) / (e * e) + 2 * (W(r + e) - W(r - e)) / (2 * e) / r
    rho_i, rho_j = o["rho"][1], o["rho"][0]
    vi32 = np.asarray(vi, np.float32).astype(np.float64)
    expect = (1 / rho_i) * p["mu"] * p["mass"] * (0 - vi32) / rho_j * lap
    assert np.allclose(o["acc"][1], expect, rtol=1e-5)


def test_coincident_pair_density_but_no_force(orc):
    p = _params(gy=0.0)
    pos = _p4([[0.5, 0.5, 0.5], [0.5, 0.5, 0.5]])
    o = orc.step(p, pos, _z4(2), _z4(0), _z4(0))
    assert o["rho"][0] == pytest.approx(2 * p["mass"] * orc.w_poly6(p, 0), rel=1e-12)
    assert np.all(o["acc"] == 0)


# ------------------------------------------------------- P4 momentum

@pytest.mark.parametrize("const_set", [0, 1])
def test_internal_forces_conserve_momentum(orc, const_set):
    """Sum_i m a_i = 0 without gravity: every pair term is antisymmetric,
    fluid-fluid and fluid-attached alike."""
    sc = scenes.scaled_block(3000, 24, (0.4, 0.4, 0.4), (0.4, 0.4, 0.4), seed=21)
    p = dict(sc["params"], gy=0.0, const_set=const_set)
    vel = sc["fluid_vel"].copy()
    vel[:, :3] = np.random.default_rng(0).normal(size=(len(vel), 3)).astype(np.float32)
    o = orc.step(p, sc["fluid_pos"], vel, sc["boid_pos"] * np.float32(0.4), sc["boid_vel"])
    mom = (p["mass"] * o["acc"]).sum(axis=0)
    scale = (p["mass"] * np.linalg.norm(o["acc"], axis=1)).sum()
    assert np.all(np.abs(mom) <= 1e-12 * scale)
    assert o["touched"].sum() > 0


# ---------------------------------------------------- P5 rest density

def test_lattice_interior_at_rest_density(orc):
    """With the calibrated mass the interior of the unjittered lattice has
    the rest density; the mass matches the closed-form lattice sum at h/2."""
    p = _params(gy=0.0)
    s = scenes.f32(np.float32(p["h"]) / np.float32(2))
    m = orc.lattice_mass(p, s)
    h = p["h"]
    # spacing h/2: sum_o (h^2 - |o|^2 h^2/4)^3 over |o|^2 in {0,1,2,3} (1, 6, 12, 8
    # offsets) = (1 + 6 (3/4)^3 + 12 (1/2)^3 + 8 (1/4)^3) h^6 = 5.15625 h^6
    expect_m = p["rho0"] / (315.0 / (64 * math.pi * h ** 9) * 5.15625 * h ** 6)
    assert m == pytest.approx(expect_m, rel=2e-6)
    p["mass"] = scenes.f32(m)
    n = 14
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    pos = _p4(np.stack([i.ravel(), j.ravel(), k.ravel()], 1) * np.float32(s) + np.float32(0.25))
    o = orc.step(p, pos, _z4(len(pos)), _z4(0), _z4(0))
    inner = np.all((np.stack([i.ravel(), j.ravel(), k.ravel()], 1) >= 3) &
                   (np.stack([i.ravel(), j.ravel(), k.ravel()], 1) <= n - 4), axis=1)
    assert np.all(np.abs(o["rho"][inner] / p["rho0"] - 1) < 1e-5)
    # and the interior feels no net pressure force (symmetric neighbourhood):
    # what is left comes from the float32 lattice and is far below gravity
    assert np.all(np.abs(o["acc"][inner]) < 1e-4 * 9.8)


# ------------------------------------------------------------- P6 boids

def test_two_boids_by_hand(orc):
    p = _params()
    rs, wsep, wal, wco, dt = p["r_sep"], p["w_sep"], p["w_align"], p["w_coh"], p["dt"]
    bp = _p4([[0.5, 0.5, 0.5], [0.5625, 0.5, 0.5]])
    bv = _p4([[0.2, 0.0, 0.0], [0.0, 0.3, 0.0]])
    o = orc.step(p, _z4(0), _z4(0), bp, bv)
    # boid A: d = (-0.0625, 0, 0), |d| = 0.0625 < r_sep
    w = 1 - 0.0625 / rs
    v = np.array([0.2, 0.0, 0.0]) + wsep * np.array([-0.0625 * w, 0, 0])   # separation
    v = v + wal * (np.array([0.0, np.float32(0.3), 0.0]) - v)              # alignment (mean of B)
    v = v + wco * np.array([0.0625, 0.0, 0.0])                              # cohesion (towards B)
    v0 = np.array([np.float32(0.2), 0, 0]) + wsep * np.array([-0.0625 * w, 0, 0])
    v0 = v0 + wal * (np.array([0.0, np.float32(0.3), 0.0]) - v0) + wco * np.array([0.0625, 0, 0])
    assert np.allclose(o["new_boid_vel"][0], v0, rtol=1e-12)
    assert np.allclose(o["new_boid_pos"][0], np.array([0.5, 0.5, 0.5]) + v0 * dt, rtol=1e-12)
    assert o["boid_nsep"][0] == 1 and o["boid_nvis"][0] == 1
    assert np.all(o["fb"] == 0)


def test_symmetric_school_has_no_net_steer_at_centre(orc):
    p = _params()
    c = 0.5
    e = 0.0625
    pts = [[c, c, c]] + [[c + s * e * (a == 0), c + s * e * (a == 1), c + s * e * (a == 2)]
                         for a in range(3) for s in (-1, 1)]
    o = orc.step(p, _z4(0), _z4(0), _p4(pts), _z4(len(pts)))
    assert np.all(o["new_boid_vel"][0] == 0)
    # the outer boids are pushed outward along their axis
    for b in range(1, 7):
        d = np.asarray(pts[b]) - c
        assert np.dot(o["new_boid_vel"][b], d) > 0


def test_school_rules_conserve_boid_momentum(orc):
    """Separation is antisymmetric and, in a fully connected group,
    alignment and cohesion move every boid towards means that sum to the
    totals: the summed velocity is unchanged (no fluid, no walls, speeds
    inside [v_min, v_max])."""
    p = _params(v_min=0.0, v_max=100.0)
    rng = np.random.default_rng(3)
    pts = 0.5 + rng.uniform(-0.04, 0.04, size=(12, 3))
    vel = rng.normal(size=(12, 3)) * 0.3
    o = orc.step(p, _z4(0), _z4(0), _p4(pts), _p4(vel))
    assert np.all(o["boid_nvis"] == 11)
    assert np.all(o["boid_nsep"] > 0)
    v32 = _p4(vel)[:, :3].astype(np.float64)
    assert np.allclose(o["new_boid_vel"].sum(0), v32.sum(0), atol=1e-12)


def test_speed_limit_and_edge_turn(orc):
    p = _params()
    bp = _p4([[0.2, 0.2, 0.2], [0.8, 0.8, 0.8], [-0.1, 0.5, 1.2]])
    bv = _p4([[3.0, 0.0, 0.0], [0.0, 0.0, 0.01], [0.0, 0.0, 0.0]])
    o = orc.step(p, _z4(0), _z4(0), bp, bv)
    assert np.linalg.norm(o["new_boid_vel"][0]) == pytest.approx(p["v_max"], rel=1e-12)
    assert np.linalg.norm(o["new_boid_vel"][1]) == pytest.approx(p["v_min"], rel=1e-12)
    # outside on x (below min) and on z (above max): steered by +-edge_turn, then clamped up to v_min
    v = o["new_boid_vel"][2]
    assert v[0] > 0 and v[2] < 0 and v[1] == 0


# --------------------------------------------------------- integrator

def test_free_fall_is_euler_cromer(orc):
    """A lone particle: after n steps x_n = x_0 + v_0 n dt + g dt^2 n(n+1)/2
    (the semi-implicit Euler sum), v_n = v_0 + g n dt."""
    p = _params(box_max=(1.0, 10.0, 1.0))
    g, dt = p["gy"], p["dt"]
    pos = _p4([[0.5, 5.0, 0.5]])
    vel = _p4([[0.0, 0.25, 0.0]])
    x, v = pos[0, 1].astype(np.float64), vel[0, 1].astype(np.float64)
    n = 20
    for _ in range(n):
        o = orc.step(p, pos, vel, _z4(0), _z4(0))
        pos = _p4(o["new_fluid_pos"])
        vel = _p4(o["new_fluid_vel"])
    assert pos[0, 1] == pytest.approx(x + v * n * dt + g * dt * dt * n * (n + 1) / 2, rel=1e-6)
    assert vel[0, 1] == pytest.approx(v + g * n * dt, rel=1e-5)


def test_wall_reflection_by_hand(orc):
    p = _params()
    pos = _p4([[0.5, 0.0005, 0.5]])
    vel = _p4([[0.0, -1.0, 0.0]])
    o = orc.step(p, pos, vel, _z4(0), _z4(0))
    vy = -1.0 + p["gy"] * p["dt"]
    y = np.float64(np.float32(0.0005)) + vy * p["dt"]
    assert y < 0
    assert o["new_fluid_pos"][0, 1] == pytest.approx(-y, rel=1e-12)
    assert o["new_fluid_vel"][0, 1] == pytest.approx(-0.75 * vy, rel=1e-12)
