"""The oracle's step statistics pinned to a hand-computed example, to brute
force and to the momentum invariant (CPU only)."""
import numpy as np
import pytest

import oracle
from paper_2311_15088_gb300 import scenes


def test_hand_example():
    """Two attached particles (ids 0, 1) and three fluid particles (ids 2-4)
    with chosen outputs; every statistic worked out by hand."""
    o = dict(
        nbr_count=np.array([9, 9, 2, 4, 0], np.int32),
        rho=np.array([5.0, 5.0, 1000.0, 1010.0, 990.0]),
        new_fluid_vel=np.array([[1.0, 0.0, 0.0], [0.0, 2.0, 0.0], [0.0, 0.0, -2.0]]),
        cell_start=np.array([0, 2, 2, 5], np.int32),  # cells of 2, 0 and 3 particles
    )
    got = oracle.step_stats({"mass": np.float32(2.0)}, o, n_boid=2)
    want = dict(fluid=3, nbr_mean=2.0, nbr_max=4, cell_max=3, mom_x=2.0, mom_y=4.0, mom_z=-4.0,
                ke=9.0, rho_min=990.0, rho_max=1010.0, rho_mean=1000.0, speed_max=2.0)
    assert list(oracle.STATS) == list(want)
    assert np.array_equal(got, np.array(list(want.values()), np.float64))


def test_no_fluid_gives_zero_means():
    o = dict(nbr_count=np.array([3], np.int32), rho=np.array([7.0]), new_fluid_vel=np.zeros((0, 3)),
             cell_start=np.array([0, 1], np.int32))
    got = oracle.step_stats({"mass": np.float32(1.0)}, o, n_boid=1)
    assert np.array_equal(got, [0, 0, 0, 1, 0, 0, 0, 0, 0, 0, 0, 0])


def test_neighbour_statistics_equal_brute_force():
    """Mean and largest neighbour count of the fluid particles against the
    brute-force O(N^2) neighbour search (attached particles count as
    neighbours of the fluid, not as fluid); the fullest cell against a
    direct count of the cell keys."""
    sc = scenes.scaled_block(2500, 40, (0.5, 0.4, 0.5), (0.5, 0.4, 0.5), seed=4)
    p = dict(sc["params"])
    o = oracle.step(p, sc["fluid_pos"], sc["fluid_vel"], sc["boid_pos"], sc["boid_vel"])
    nb = len(sc["boid_pos"])
    allpos = np.concatenate([sc["boid_pos"], sc["fluid_pos"]])
    counts, _, _ = oracle.neighbors(p, allpos, n_att=nb, brute=True, lists=False)
    st = oracle.step_stats(p, o, nb)
    assert st[0] == len(sc["fluid_pos"])
    assert st[1] == counts[nb:].sum() / len(sc["fluid_pos"])
    assert st[2] == counts[nb:].max()
    keys, _, _ = oracle.bin_particles(p, allpos)
    assert st[3] == np.bincount(keys).max()


@pytest.mark.parametrize("const_set", [0, 1])
def test_momentum_of_a_released_block_is_zero(const_set):
    """From rest, without gravity and away from the walls, one step gives
    every fluid particle dt a_i: the internal pair forces cancel, so the
    momentum statistic is zero to round-off against sum m |v|, and the
    kinetic energy equals (1/2) m dt^2 sum |a_i|^2."""
    sc = scenes.scaled_block(3000, 0, (0.4, 0.4, 0.4), (0.4, 0.4, 0.4), seed=9)
    p = dict(sc["params"], gy=0.0, const_set=const_set)
    z = np.zeros((0, 4), np.float32)
    o = oracle.step(p, sc["fluid_pos"], np.zeros_like(sc["fluid_pos"]), z, z)
    st = oracle.step_stats(p, o, 0)
    m, dt = float(np.float32(p["mass"])), float(np.float32(p["dt"]))
    v = np.asarray(o["new_fluid_vel"])
    scale = m * np.abs(v).sum()
    assert scale > 0
    assert np.all(np.abs(st[4:7]) <= 1e-12 * scale)
    a = np.asarray(o["acc"])
    assert st[7] == pytest.approx(0.5 * m * dt * dt * (a * a).sum(), rel=1e-12)
    assert st[11] == pytest.approx(dt * np.sqrt((a * a).sum(axis=1)).max(), rel=1e-12)
