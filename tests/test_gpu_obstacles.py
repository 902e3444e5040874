"""Obstacle grid and obstacle avoidance on the GPU against the oracle
(needs a GB300): the grid's counts bit-exact (float32 signed distances in
the same order on both sides) and its normals within float32 rounding; one
step with obstacles within the step's tolerances (tests/parity.py)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2311_15088_gb300 import scenes, sph
from paper_2311_15088_gb300.sph import Scene

from parity import compare_step, gpu_outputs

pytestmark = pytest.mark.gpu

SPHERES = np.array([[0.30, 0.25, 0.30, 0.12], [0.62, 0.30, 0.55, 0.08], [0.45, 0.15, 0.70, 0.2]], np.float32)
BOXES = np.array([[0.05, 0.02, 0.55, 0.25, 0.30, 0.80], [0.50, 0.35, 0.10, 0.58, 0.50, 0.40]], np.float32)


def _scene(seed=11):
    sc = scenes.scaled_block(12000, 400, (0.8, 0.55, 0.8), (0.8, 0.55, 0.8), seed=seed)
    p = dict(sc["params"])
    return sc, p


def _obstacles(w=0.08, near=2.5):
    return dict(spheres=SPHERES, boxes=BOXES, w_obst=w, near_factor=near)


def test_obstacle_grid_matches_oracle():
    sc, p = _scene()
    s = Scene(p, len(sc["fluid_pos"]), len(sc["boid_pos"]))
    s.set_state(sc["fluid_pos"], sc["fluid_vel"], sc["boid_pos"], sc["boid_vel"])
    s.set_obstacles(SPHERES, BOXES, 0.08, 2.5)
    g = s.field("obstacle_grid").cpu().numpy().astype(np.float64)
    o = oracle.obstacle_grid(p, spheres=SPHERES, boxes=BOXES)
    assert np.array_equal(g[:, 3], o[:, 3])
    assert (o[:, 3] > 0).sum() > 20 and (o[:, 3] > 1).sum() > 0
    assert np.all(np.abs(g[:, :3] - o[:, :3]) <= 1e-6)


@pytest.mark.parametrize("cell", [1.0, 0.5])
def test_step_with_obstacles_matches_oracle(cell):
    sc, p = _scene()
    p["cell_size"] = scenes.f32(p["h"] * cell)
    s = Scene(p, len(sc["fluid_pos"]), len(sc["boid_pos"]), diagnostics=True)
    s.set_state(sc["fluid_pos"], sc["fluid_vel"], sc["boid_pos"], sc["boid_vel"])
    s.set_obstacles(SPHERES, BOXES, 0.08, 2.5)
    s.step(1)
    g = gpu_outputs(s)
    o = oracle.step(p, sc["fluid_pos"], sc["fluid_vel"], sc["boid_pos"], sc["boid_vel"], obstacles=_obstacles())
    compare_step(p, g, o, len(sc["boid_pos"]))
    assert s.status() & 1 == 0
    # the obstacles changed some boids' velocities
    plain = oracle.step(p, sc["fluid_pos"], sc["fluid_vel"], sc["boid_pos"], sc["boid_vel"])
    moved = np.abs(o["new_boid_vel"] - plain["new_boid_vel"]).max(axis=1) > 1e-3
    assert moved.sum() > 20


def test_obstacles_off_and_graph_replay():
    sc, p = _scene(5)
    a = Scene(p, len(sc["fluid_pos"]), len(sc["boid_pos"]))
    b = Scene(p, len(sc["fluid_pos"]), len(sc["boid_pos"]))
    for s in (a, b):
        s.set_state(sc["fluid_pos"], sc["fluid_vel"], sc["boid_pos"], sc["boid_vel"])
    b.set_obstacles(SPHERES, BOXES, 0.08, 2.5)
    b.set_obstacles(None, None, 0.08, 2.5)  # off again
    a.step(3)
    b.step(3)
    for x, y in zip(a.get_state(), b.get_state()):
        assert torch.equal(x, y)
    # the captured step reads the obstacle settings when it runs
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        c = Scene(p, len(sc["fluid_pos"]), len(sc["boid_pos"]))
        d = Scene(p, len(sc["fluid_pos"]), len(sc["boid_pos"]))
        for s in (c, d):
            s.set_state(sc["fluid_pos"], sc["fluid_vel"], sc["boid_pos"], sc["boid_vel"])
            s.set_obstacles(SPHERES, BOXES, 0.08, 2.5)
        c.step(4)
        d.graph_step(4)
        states = [(x.clone(), y.clone()) for x, y in zip(c.get_state(), d.get_state())]
    torch.cuda.synchronize()
    for x, y in states:
        assert torch.equal(x, y)


def test_bad_obstacles_are_rejected():
    sc, p = _scene()
    s = Scene(p, len(sc["fluid_pos"]), len(sc["boid_pos"]))
    with pytest.raises(sph.SphError):
        s.set_obstacles(np.array([[0.5, 0.5, 0.5, 0.0]], np.float32), None)
    with pytest.raises(sph.SphError):
        s.set_obstacles(None, np.array([[0.5, 0.5, 0.5, 0.4, 0.6, 0.6]], np.float32))
    with pytest.raises(sph.SphError):
        s.set_obstacles(np.tile(SPHERES[:1], (sph.SPH_MAX_OBSTACLES + 1, 1)), None)
    with pytest.raises(sph.SphError):
        s.set_obstacles(SPHERES, None, float("nan"), 2.0)
