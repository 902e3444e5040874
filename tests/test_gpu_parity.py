"""GPU step vs the CPU oracle, element by element (needs a GB300).

Every case runs the CUDA path through the C ABI (via the ctypes binding)
and the oracle on the same seeded float32 state, then compares every field
of one step with the tolerances listed in tests/parity.py.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2311_15088_gb300 import scenes, sph
from paper_2311_15088_gb300.sph import Scene

from parity import compare_step, gpu_outputs, lattice_params, oracle_step, run_gpu

pytestmark = pytest.mark.gpu


def _state_of(s, p):
    fp, fv, bp, bv = (t.cpu().numpy() for t in s.get_state())
    return dict(params=p, fluid_pos=fp, fluid_vel=fv, boid_pos=bp, boid_vel=bv)


def _check(p, sc):
    nb = len(sc["boid_pos"])
    s = run_gpu(p, sc, steps=1)
    g = gpu_outputs(s)
    o = oracle_step(p, sc)
    compare_step(p, g, o, nb)
    assert s.status() & (sph.SPH_DEV_NONFINITE | sph.SPH_DEV_BOUNDS) == 0
    return s, g, o


CELLS = [1.0, 0.5, 0.34]  # cell size in units of h


@pytest.mark.parametrize("cell", CELLS)
def test_dam_break_4096_first_step(cell):
    sc = scenes.dam_break_small()
    p = lattice_params(sc)
    p["cell_size"] = scenes.f32(p["h"] * cell)
    _check(p, sc)


@pytest.mark.parametrize("cell,cell_x", [(0.5, 0.25), (1.0, 0.5), (0.5, 0.125)])
def test_narrow_x_cells_first_step(cell, cell_x):
    """Cells narrower along x than along y and z: keys, order, neighbour
    sets and every field of the step as with cubic cells."""
    sc = scenes.scaled_block(12000, 300, (0.6, 0.6, 0.6), (0.6, 0.4, 0.6), seed=78)
    sc["boid_pos"][:, 1] *= np.float32(0.4 / 0.6)
    p = dict(sc["params"])
    p["cell_size"] = scenes.f32(p["h"] * cell)
    p["cell_size_x"] = scenes.f32(p["h"] * cell_x)
    _s, _g, o = _check(p, sc)
    assert o["touched"].sum() > 1000


def test_dam_break_4096_after_80_gpu_steps():
    """Run the GPU 80 steps (the column collapses and compresses), then one
    more step on the GPU and in the oracle from the GPU's state."""
    sc = scenes.dam_break_small()
    p = lattice_params(sc)
    s = run_gpu(p, sc, steps=80)
    st = _state_of(s, p)
    _check(p, st)


@pytest.mark.parametrize("const_set,cell", [(0, 0.5), (1, 0.5), (0, 1.0), (1, 0.34)])
def test_fluid_with_boids_inside(const_set, cell):
    """12k particles with 300 boids moving through the fluid: coupling,
    touched_by_boid and boid_influence are all exercised."""
    sc = scenes.scaled_block(12000, 300, (0.6, 0.6, 0.6), (0.6, 0.4, 0.6), seed=77)
    sc["boid_pos"][:, 1] *= np.float32(0.4 / 0.6)
    p = dict(sc["params"], const_set=const_set)
    p["cell_size"] = scenes.f32(p["h"] * cell)
    _s, _g, o = _check(p, sc)
    assert o["touched"].sum() > 1000


@pytest.mark.parametrize("cell", [1.0, 0.5])
def test_column_262144_first_step(cell):
    sc = scenes.dam_break_column()
    p = lattice_params(sc)
    p["cell_size"] = scenes.f32(p["h"] * cell)
    _check(p, sc)


@pytest.mark.parametrize("cell", CELLS + [0.25])
def test_neighbor_lists_bit_exact(cell):
    """Neighbour lists, in walk order, equal the oracle's; particles are
    squeezed into the corners and some lie outside the box."""
    sc = scenes.scaled_block(6000, 40, (0.5, 0.5, 0.5), (0.5, 0.5, 0.5), seed=3)
    p = dict(sc["params"], cell_size=scenes.f32(sc["params"]["h"] * cell))
    fp = sc["fluid_pos"]
    k = len(fp) // 4
    fp[:k, :3] = np.where(fp[:k, :3] < 0.25, fp[:k, :3] * 0.1, 0.5 - (0.5 - fp[:k, :3]) * 0.1)
    fp[k:k + 50, 0] = np.float32(-0.02)
    fp[k + 50:k + 100, 1] = np.float32(0.53)
    s = Scene(p, len(sc["fluid_pos"]), len(sc["boid_pos"]))
    s.set_state(sc["fluid_pos"], sc["fluid_vel"], sc["boid_pos"], sc["boid_vel"])
    counts, offsets, lst = s.neighbors()
    pos = np.concatenate([sc["boid_pos"], sc["fluid_pos"]])
    c2, o2, l2 = oracle.neighbors(p, pos, n_att=len(sc["boid_pos"]))
    assert np.array_equal(counts.cpu().numpy(), c2)
    assert np.array_equal(offsets.cpu().numpy(), o2)
    assert np.array_equal(lst.cpu().numpy(), l2)


@pytest.mark.parametrize("cell", [1.0, 0.5])
def test_crowded_cells_sort_paths(cell):
    """Crowded cells take the block-sort path of the per-cell sort, and the
    5,000-particle clump gives its particles more hit segments than the
    density pass can store (128 of 32 slots), so the force pass tests their
    candidates again; order and sums must still match."""
    rng = np.random.default_rng(5)
    p = scenes.default_params(mass=scenes.f32(0.001))
    h = p["h"]
    p["cell_size"] = scenes.f32(h * cell)
    a = 0.5 + rng.uniform(0, 0.9 * h, size=(5000, 3))       # > 4,096 candidates each
    b = 0.2 + rng.uniform(0, 0.4 * h, size=(100, 3))        # one crowded cell
    c = rng.uniform(0.05, 0.95, size=(3000, 3))             # sparse background
    pos = np.zeros((8100, 4), np.float32)
    pos[:, :3] = np.concatenate([a, b, c])
    sc = dict(fluid_pos=pos, fluid_vel=np.zeros_like(pos), boid_pos=np.zeros((0, 4), np.float32),
              boid_vel=np.zeros((0, 4), np.float32))
    s, _, _ = _check(p, sc)
    nseg = s.field("nseg").cpu().numpy()
    assert (nseg > 128).sum() > 1000 and (nseg <= 128).sum() > 1000


def test_edge_cases_small_scenes():
    p = scenes.default_params(mass=scenes.f32(0.01))
    z = np.zeros((0, 4), np.float32)
    one = np.array([[0.5, 0.5, 0.5, 0]], np.float32)
    # a single fluid particle
    _check(p, dict(fluid_pos=one, fluid_vel=np.zeros_like(one), boid_pos=z, boid_vel=z))
    # boids only (their attached particles have no fluid neighbours)
    bp, bv = scenes.boids_uniform(50, (0, 0, 0), (1, 1, 1), seed=9)
    _check(p, dict(fluid_pos=z, fluid_vel=z, boid_pos=bp, boid_vel=bv))
    # coincident particles and particles outside the box (clamped cells)
    pts = np.array([[0.3, 0.3, 0.3, 0], [0.3, 0.3, 0.3, 0], [0.31, 0.3, 0.3, 0], [-0.05, 0.5, 0.5, 0],
                    [1.02, 0.99, 0.5, 0], [0.99, 1.03, 0.5, 0]], np.float32)
    _check(p, dict(fluid_pos=pts, fluid_vel=np.zeros_like(pts), boid_pos=z, boid_vel=z))


def test_unjittered_lattice_ties():
    p = scenes.default_params()
    s = np.float32(p["h"]) / np.float32(2)
    p["mass"] = scenes.f32(oracle.lattice_mass(p, s))
    n = 12
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    pos = np.zeros((n ** 3, 4), np.float32)
    pos[:, :3] = np.stack([i.ravel(), j.ravel(), k.ravel()], 1) * s + np.float32(0.2)
    z = np.zeros((0, 4), np.float32)
    _check(p, dict(fluid_pos=pos, fluid_vel=np.zeros_like(pos), boid_pos=z, boid_vel=z))


def test_deterministic_and_resumable():
    """Two runs agree bit for bit; stopping, reading the state back and
    loading it again continues bit-identically."""
    sc = scenes.dam_break_small()
    p = lattice_params(sc)
    a = run_gpu(p, sc, steps=30)
    b = run_gpu(p, sc, steps=15)
    fp, fv, bp, bv = b.get_state()
    c = Scene(p, len(sc["fluid_pos"]), len(sc["boid_pos"]))
    c.set_state(fp, fv, bp, bv)
    c.step(15)
    sa = [t.cpu().numpy() for t in a.get_state()]
    sc_ = [t.cpu().numpy() for t in c.get_state()]
    for x, y in zip(sa, sc_):
        assert np.array_equal(x, y)
    d = run_gpu(p, sc, steps=30)
    for x, y in zip(sa, [t.cpu().numpy() for t in d.get_state()]):
        assert np.array_equal(x, y)


def test_boid_forces_entry_point_matches_step():
    sc = scenes.scaled_block(8000, 200, (0.5, 0.5, 0.5), (0.5, 0.3, 0.5), seed=12)
    sc["boid_pos"][:, 1] *= np.float32(0.3 / 0.5)
    p = sc["params"]
    s = Scene(p, len(sc["fluid_pos"]), len(sc["boid_pos"]))
    s.set_state(sc["fluid_pos"], sc["fluid_vel"], sc["boid_pos"], sc["boid_vel"])
    f_now = s.boid_forces().cpu().numpy()
    s.step(1)
    f_step = s.field("fb").cpu().numpy()
    assert np.array_equal(f_now, f_step)
    o = oracle_step(p, sc)
    assert np.all(np.abs(f_now[:, :3] - o["fb"]).max(1) <= 1e-5 * o["acc_scale"][:len(f_now)])


def test_host_buffers_round_trip():
    sc = scenes.dam_break_small(n_side=10, n_boid=8)
    p = lattice_params(sc)
    s = Scene(p, len(sc["fluid_pos"]), len(sc["boid_pos"]))
    host = [torch.from_numpy(a).pin_memory() for a in (sc["fluid_pos"], sc["fluid_vel"], sc["boid_pos"], sc["boid_vel"])]
    s.set_state_host(*host)
    s.step(3)
    outs = [torch.empty_like(t).pin_memory() for t in host]
    s.get_state_host(outs)
    dev = run_gpu(p, sc, steps=3).get_state()
    for a, b in zip(outs, dev):
        assert np.array_equal(a.numpy(), b.cpu().numpy())


def test_pageable_host_buffers_round_trip():
    """Host buffers that are not page-locked round-trip like page-locked
    ones: both give the device path's state bit for bit."""
    sc = scenes.dam_break_small(n_side=10, n_boid=8)
    p = lattice_params(sc)
    s = Scene(p, len(sc["fluid_pos"]), len(sc["boid_pos"]))
    host = [torch.from_numpy(a.copy()) for a in (sc["fluid_pos"], sc["fluid_vel"], sc["boid_pos"], sc["boid_vel"])]
    assert not any(t.is_pinned() for t in host)
    s.set_state_host(*host)
    s.step(3)
    outs = [torch.empty_like(t) for t in host]
    s.get_state_host(outs)
    pinned = [torch.empty_like(t).pin_memory() for t in host]
    s.get_state_host(pinned)
    dev = run_gpu(p, sc, steps=3).get_state()
    for a, b, c in zip(outs, pinned, dev):
        assert np.array_equal(a.numpy(), c.cpu().numpy())
        assert np.array_equal(b.numpy(), c.cpu().numpy())


def test_nonfinite_input_sets_status_bit():
    sc = scenes.dam_break_small(n_side=8, n_boid=4)
    p = lattice_params(sc)
    fp = sc["fluid_pos"].copy()
    fp[7, 0] = np.nan
    s = Scene(p, len(fp), len(sc["boid_pos"]))
    s.set_state(fp, sc["fluid_vel"], sc["boid_pos"], sc["boid_vel"])
    s.step(1)
    assert s.status() & 1
    s.clear_status()
    assert s.status() == 0


def test_large_tank_settled_step_full_size():
    """The 2,097,152-particle tank of the benchmark: 200 settling steps on
    the GPU, boids released, 20 more steps, then one step compared with the
    oracle on every particle."""
    sc = scenes.large_tank()
    p = dict(sc["params"])
    z = np.zeros((0, 4), np.float32)
    s = Scene(p, len(sc["fluid_pos"]), 0)
    s.set_state(sc["fluid_pos"], sc["fluid_vel"], z, z)
    s.step(200)
    fp, fv, _, _ = s.get_state()
    s2 = Scene(p, len(sc["fluid_pos"]), len(sc["boid_pos"]))
    s2.set_state(fp, fv, sc["boid_pos"], sc["boid_vel"])
    s2.step(20)
    st = _state_of(s2, p)
    _check(p, st)


@pytest.mark.parametrize("cell", [1.0, 0.5, 0.25])
def test_candidate_counts_cover_neighbours(cell):
    """Every neighbour is a candidate the walk visited (the particle itself
    too), so ncand >= nbr_count + 1 for every particle."""
    sc = scenes.dam_break_column(n_side=32, n_boid=64)
    p = lattice_params(sc)
    p["cell_size"] = scenes.f32(p["h"] * cell)
    s = run_gpu(p, sc, steps=3)
    nc = s.field("ncand").cpu().numpy().astype(np.int64)
    nbr = s.field("nbr_count").cpu().numpy().astype(np.int64)
    assert np.all(nc >= nbr + 1)


@pytest.mark.parametrize("cap", ["ample", "tiny"])
def test_neighbor_lists_bitwise_equal_to_walk(cap):
    """With pair lists the force pass reads each particle's neighbours from
    its list (walk order) instead of testing candidates: 20 steps give the
    walk's bits.  A pair buffer too small for the lists makes the particles
    that do not fit walk instead, flagged SPH_DEV_LIST_OVERFLOW (8)."""
    sc = scenes.scaled_block(12000, 300, (0.6, 0.6, 0.6), (0.6, 0.4, 0.6), seed=77)
    sc["boid_pos"][:, 1] *= np.float32(0.4 / 0.6)
    p = sc["params"]
    a = run_gpu(p, sc, steps=20)
    b = Scene(p, len(sc["fluid_pos"]), len(sc["boid_pos"]), diagnostics=True)
    b.set_state(sc["fluid_pos"], sc["fluid_vel"], sc["boid_pos"], sc["boid_vel"])
    b.step(1)
    pairs = int(b.field("nbr_count").cpu().numpy().astype(np.int64).sum())
    b.set_state(sc["fluid_pos"], sc["fluid_vel"], sc["boid_pos"], sc["boid_vel"])
    b.set_neighbor_lists(3 * pairs if cap == "ample" else pairs // 3)
    b.step(20)
    for x, y in zip(a.get_state(), b.get_state()):
        assert torch.equal(x, y)
    assert torch.equal(a.field("acc"), b.field("acc"))
    overflow = b.status() & 8
    assert (overflow == 0) if cap == "ample" else (overflow != 0)


@pytest.mark.parametrize("cell", [1.0, 0.5])
def test_bucket_grid_ablation(cell):
    """The paper's fixed-capacity hash grid: with buckets as large as the
    most crowded cell its neighbour counts are the exact ones; with smaller
    buckets it drops particles and never finds more neighbours than exist."""
    sc = scenes.scaled_block(12000, 300, (0.6, 0.6, 0.6), (0.6, 0.4, 0.6), seed=77)
    sc["boid_pos"][:, 1] *= np.float32(0.4 / 0.6)
    p = dict(sc["params"], cell_size=scenes.f32(sc["params"]["h"] * cell))
    s = Scene(p, len(sc["fluid_pos"]), len(sc["boid_pos"]))
    s.set_state(sc["fluid_pos"], sc["fluid_vel"], sc["boid_pos"], sc["boid_vel"])
    exact, _, _ = s.neighbors()
    exact = exact.cpu().numpy()
    s.step(1)
    occupancy = int(np.diff(s.field("cell_start").cpu().numpy().astype(np.int64)).max())
    s.set_state(sc["fluid_pos"], sc["fluid_vel"], sc["boid_pos"], sc["boid_vel"])
    counts, dropped = s.bucket_neighbors(occupancy)
    assert np.array_equal(counts.cpu().numpy(), exact) and int(dropped.item()) == 0
    small = max(1, occupancy // 3)
    counts, dropped = s.bucket_neighbors(small)
    c = counts.cpu().numpy()
    assert int(dropped.item()) > 0
    assert np.all(c <= exact) and c.sum() < exact.sum()


def test_clamp_flag_marks_fluid_outside_the_tank_only():
    """SPH_DEV_CLAMPED (2) reports a fluid particle binned outside the tank:
    particles resting on the faces (box_min, box_max) and boids flying
    outside the tank do not raise it; a fluid particle loaded outside does."""
    p = scenes.default_params(mass=scenes.f32(0.01))
    lo, hi = np.asarray(p["box_min"], np.float32), np.asarray(p["box_max"], np.float32)
    fp = np.zeros((6, 4), np.float32)
    fp[0, :3], fp[1, :3] = hi, lo
    fp[2, :3] = (hi[0], 0.5, 0.5)
    fp[3, :3] = (0.5, hi[1], 0.5)
    fp[4, :3] = (0.5, 0.5, hi[2])
    fp[5, :3] = (0.3, 0.3, 0.3)
    bp = np.array([[1.4, 0.5, 0.5, 0.0], [0.5, -0.3, 0.5, 0.0]], np.float32)
    bv = np.array([[0.5, 0.0, 0.0, 0.0], [0.0, -0.5, 0.0, 0.0]], np.float32)
    s = Scene(p, len(fp), len(bp))
    s.set_state(fp, np.zeros_like(fp), bp, bv)
    s.step(3)
    assert s.status() & 2 == 0
    fp[5, 0] = np.float32(1.2)
    s.set_state(fp, np.zeros_like(fp), bp, bv)
    s.step(1)
    assert s.status() & 2


@pytest.mark.parametrize("cell", [1.0, 0.5])
def test_literal_coupling_two_steps(cell):
    """SPH_COUPLE_LITERAL: the attached particle keeps and integrates its own
    velocity and the boid adds sph_factor times it.  Step 1 from a loaded
    state (v_att = v_b) and step 2 from the GPU's state after step 1 (its
    attached velocities read back) against the oracle, every field at the
    usual tolerances, and the attached velocity carried into the next step
    within the fluid velocity's tolerance."""
    sc = scenes.scaled_block(8000, 120, (0.6, 0.6, 0.6), (0.6, 0.35, 0.6), seed=21)
    sc["boid_pos"][:, 1] *= np.float32(0.35 / 0.6)
    p = dict(sc["params"], coupling_mode=sph.SPH_COUPLE_LITERAL, sph_factor=scenes.f32(0.05),
             cell_size=scenes.f32(sc["params"]["h"] * cell))
    nb = len(sc["boid_pos"])
    s = Scene(p, len(sc["fluid_pos"]), nb, diagnostics=True)
    s.set_state(sc["fluid_pos"], sc["fluid_vel"], sc["boid_pos"], sc["boid_vel"])
    att = sc["boid_vel"]
    state = sc
    g_ = np.float64(np.linalg.norm([np.float32(p["gx"]), np.float32(p["gy"]), np.float32(p["gz"])]))
    for it in range(2):
        s.step(1)
        g = gpu_outputs(s)
        o = oracle.step(p, state["fluid_pos"], state["fluid_vel"], state["boid_pos"], state["boid_vel"],
                        att_vel=att)
        compare_step(p, g, o, nb)
        ga = s.field("att_vel").cpu().numpy()
        Sb = o["acc_scale"][:nb] + g_
        tol = 1e-5 * (np.abs(o["new_att_vel"]) + p["dt"] * Sb[:, None])
        assert np.all(np.abs(ga[:, :3] - o["new_att_vel"]) <= tol), it
        # the attached particles move on their own: not the boids' velocities
        assert np.abs(ga[:, :3] - g["new_boid_vel"]).max() > 1e-3
        assert s.status() & 1 == 0
        fp, fv, bp, bv = (t.cpu().numpy() for t in s.get_state())
        # get_state staged through the scratch arrays: step again from the
        # state read back (set_state would reset v_att to the boids')
        state = dict(fluid_pos=fp, fluid_vel=fv, boid_pos=bp, boid_vel=bv)
        att = ga
