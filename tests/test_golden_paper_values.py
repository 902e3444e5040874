"""The oracle against the values the paper prints (tests/golden/
paper_printed_values.txt, each with where it is printed) (CPU)."""
import math
import os

import numpy as np
import pytest

from paper_2311_15088_gb300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_printed_values.txt")


def _golden():
    out = {}
    for line in open(GOLDEN):
        line = line.split("#", 1)[0].strip()
        if "=" in line:
            k, v = (t.strip() for t in line.split("=", 1))
            out[k] = v
    return out


@pytest.fixture(scope="module")
def g():
    return _golden()


def _p(**kw):
    p = scenes.default_params(mass=scenes.f32(0.02), **kw)
    return p


def test_poly6_prefactor(orc, g):
    p = _p()
    h = float(p["h"])
    r = 0.3 * h
    c = int(g["poly6_prefactor_numerator"]) / (int(g["poly6_prefactor_denominator_over_pi"]) * math.pi)
    want = c / h ** int(g["poly6_h_power"]) * (h * h - r * r) ** 3
    assert orc.w_poly6(p, r) == pytest.approx(want, rel=1e-12)


def test_printed_spiky_and_viscosity_prefactors(orc, g):
    p = _p(const_set=1)  # the printed constant set
    h = float(p["h"])
    r, q = 0.55 * h, 0.55
    spiky = -int(g["spiky_gradient_numerator"]) / (math.pi * h ** int(g["spiky_gradient_h_power"]))
    assert orc.grad_spiky_factor(p, r) == pytest.approx(spiky * (1 - q) ** 2 / q, rel=1e-12)
    lap = int(g["viscosity_laplacian_numerator"]) / (math.pi * h ** int(g["viscosity_laplacian_h_power"]))
    assert orc.lap_visc(p, r) == pytest.approx(lap * (1 - q), rel=1e-12)


def test_expanded_pressure_form(orc, g):
    """Two fluid particles at rest, printed constant set: the pressure part of
    the acceleration equals the expanded printed form 15 k/(pi h^4) m
    (rho_i + rho_j - 2 rho0)/rho_j (1 - q)^2/q r_ij, divided by rho_i
    (the acceleration reading)."""
    p = _p(const_set=1, gy=scenes.f32(0.0))
    h = float(p["h"])
    xi = np.array([0.5, 0.5, 0.5], np.float32)
    xj = (xi + np.array([0.4 * h, 0.1 * h, -0.2 * h], np.float32)).astype(np.float32)
    pos = np.zeros((2, 4), np.float32)
    pos[0, :3], pos[1, :3] = xj, xi
    z = np.zeros((0, 4), np.float32)
    o = orc.step(p, pos, np.zeros_like(pos), z, z)
    rho_i, rho_j = o["rho"][1], o["rho"][0]
    rij = xi.astype(np.float64) - xj.astype(np.float64)
    q = np.linalg.norm(rij) / h
    k, rho0, m = float(p["k"]), float(p["rho0"]), float(p["mass"])
    pref = int(g["pressure_sum_numerator"]) * k / (math.pi * h ** 4)
    want = pref * m * (rho_i + rho_j - 2 * rho0) / rho_j * (1 - q) ** 2 / q * rij / rho_i
    assert np.allclose(o["acc"][1], want, rtol=1e-10, atol=0)


def test_rng_listing(orc, g):
    """First draws of the printed generator, by Python integers, for a few
    streams: the oracle's integers and its float s / divisor."""
    A, B, S = int(g["rng_xor"]), int(g["rng_multiplier"]), int(g["rng_shift"])
    D = float(g["rng_divisor"])
    M = (1 << 32) - 1
    for seed, pid in ((0, 0), (scenes.BASE_SEED, 7), (123, 4095)):
        s = (seed + pid) & M
        draws = []
        for _ in range(3):
            s ^= A
            s = (s * B) & M
            s ^= s >> S
            s = (s * B) & M
            s ^= s >> S
            s = (s * B) & M
            draws.append(s)
        assert list(orc.rng_stream(seed, pid, 3)) == draws
        assert float(np.float32(draws[0] / D)) == float(np.float32(draws[0] / 4294967295.0))


def test_hash_form(orc, g):
    assert g["hash_form"].replace(" ", "") == "x+dim_x*(y+dim_y*z)"
    p = _p(cell_size=scenes.f32(0.1), box_max=(1.0, 0.7, 0.5))
    dx, dy, dz = orc.grid_dims(p, 0)
    pts = np.array([[0.05 + 0.1 * x, 0.05 + 0.1 * y, 0.05 + 0.1 * z, 0]
                    for x, y, z in ((3, 2, 1), (9, 6, 4), (0, 0, 0), (5, 0, 3))], np.float32)
    keys = orc.bin_particles(p, pts)[0]
    for (x, y, z), k in zip(((3, 2, 1), (9, 6, 4), (0, 0, 0), (5, 0, 3)), keys):
        assert k == x + dx * (y + dy * z)
