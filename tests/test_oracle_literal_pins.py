"""Pins of the oracle's literal coupling (coupling_mode 1, section "Boid
Motion and Agent Fluid Interaction": the attached particle keeps its own
velocity, is integrated like every particle, and the boid adds sph_factor
times that velocity).  The dynamics of this reading have no published
values; these tests pin what follows from its definition."""
import math

import numpy as np

import oracle
from paper_2311_15088_gb300 import scenes

LIT = 1


def _params(**kw):
    p = scenes.default_params(mass=scenes.f32(0.01))
    p.update(kw)
    return p


def test_zero_factor_equals_force_coupling():
    """With sph_factor = 0 and the attached velocities equal to the boids'
    (a freshly loaded state), the literal and the force coupling give the
    same step bit for bit; only the attached velocity carried into the next
    step differs (integrated v_b + dt (F_b + g) against the boid's)."""
    sc = scenes.scaled_block(3000, 40, (0.5, 0.5, 0.5), (0.5, 0.3, 0.5), seed=7)
    sc["boid_pos"][:, 1] *= np.float32(0.5)
    a = oracle.step(dict(sc["params"], sph_factor=0.0), sc["fluid_pos"], sc["fluid_vel"], sc["boid_pos"],
                    sc["boid_vel"])
    b = oracle.step(dict(sc["params"], sph_factor=0.0, coupling_mode=LIT), sc["fluid_pos"], sc["fluid_vel"],
                    sc["boid_pos"], sc["boid_vel"])
    for k in a:
        if k not in ("new_att_vel", "boid_vscale"):
            assert np.array_equal(a[k], b[k]), k
    assert np.array_equal(a["new_att_vel"], a["new_boid_vel"])
    p = sc["params"]
    g = np.array([p["gx"], p["gy"], p["gz"]], np.float64)
    nb = len(sc["boid_pos"])
    want = sc["boid_vel"][:, :3].astype(np.float64) + np.float32(p["dt"]) * (b["fb"] + g.astype(np.float32))
    assert np.allclose(b["new_att_vel"], want, rtol=0, atol=1e-12)
    assert b["fb"].shape == (nb, 3) and np.abs(b["fb"]).max() > 0


def test_lone_boid_by_hand():
    """A boid with no fluid and no other boid around: F_b = 0, so its
    attached particle falls freely, v_att' = v_att + dt g, and the boid gets
    v_b' = v_b + sph_factor v_att' (inside the speed limits), x_b' = x_b +
    dt v_b'."""
    p = _params(coupling_mode=LIT, sph_factor=scenes.f32(0.5))
    z = np.zeros((0, 4), np.float32)
    bp = np.array([[0.5, 0.5, 0.5, 0.0]], np.float32)
    bv = np.array([[0.3, 0.0, 0.0, 0.0]], np.float32)
    va = np.array([[0.0, 0.1, 0.0, 0.0]], np.float32)
    o = oracle.step(p, z, z, bp, bv, att_vel=va)
    dt, sf = float(np.float32(p["dt"])), float(np.float32(p["sph_factor"]))
    g = np.array([p["gx"], p["gy"], p["gz"]], np.float32).astype(np.float64)
    vatt = va[0, :3].astype(np.float64) + dt * g
    vb = bv[0, :3].astype(np.float64) + sf * vatt
    assert 0.05 < np.linalg.norm(vb) < 1.0
    assert np.allclose(o["fb"][0], 0.0, atol=0)
    assert np.allclose(o["new_att_vel"][0], vatt, rtol=1e-15, atol=0)
    assert np.allclose(o["new_boid_vel"][0], vb, rtol=1e-15, atol=0)
    assert np.allclose(o["new_boid_pos"][0], bp[0, :3].astype(np.float64) + dt * vb, rtol=1e-15, atol=0)


def test_attached_velocity_enters_the_fluid_force():
    """One fluid particle and one boid at distance r < h.  The attached
    particle's velocity enters the fluid particle's viscous term: giving it
    velocity u instead of the boid's v_b changes the fluid acceleration by
    (1/rho_f) m/rho_b C_v mu (1 - q) (u - v_b), q = r / h, C_v = 45 / (pi
    h^5) (the force is linear in the neighbour's velocity; the densities do
    not depend on velocities)."""
    p = _params(coupling_mode=LIT, gx=0.0, gy=0.0, gz=0.0)
    fp = np.array([[0.5, 0.5, 0.5, 0.0]], np.float32)
    fv = np.array([[0.1, -0.2, 0.05, 0.0]], np.float32)
    bp = np.array([[0.52, 0.49, 0.505, 0.0]], np.float32)
    bv = np.array([[0.2, 0.0, 0.0, 0.0]], np.float32)
    u = np.array([[-0.4, 0.3, 0.6, 0.0]], np.float32)
    a = oracle.step(p, fp, fv, bp, bv, att_vel=bv)
    b = oracle.step(p, fp, fv, bp, bv, att_vel=u)
    h = float(np.float32(p["h"]))
    mu, m = float(np.float32(p["mu"])), float(np.float32(p["mass"]))
    r = float(np.linalg.norm(bp[0, :3].astype(np.float64) - fp[0, :3].astype(np.float64)))
    assert r < h
    q = r / h
    cv = 45.0 / (math.pi * h ** 5)
    rho_f, rho_b = a["rho"][1], a["rho"][0]  # ids: the attached particle is 0
    want = (1.0 / rho_f) * (m / rho_b) * cv * mu * (1.0 - q) * (u[0, :3].astype(np.float64) - bv[0, :3])
    got = b["acc"][1] - a["acc"][1]
    assert np.allclose(got, want, rtol=1e-9, atol=1e-12), (got, want)
    assert np.array_equal(a["rho"], b["rho"])
