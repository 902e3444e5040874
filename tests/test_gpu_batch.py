"""Batched scenes, graph replay and launch tuning (needs a GB300).

A batch runs every pass as one launch over all scenes; each scene's result
must be bitwise the result of that scene run alone (per-particle arithmetic
and summation order depend only on the scene), whatever the launch shape.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2311_15088_gb300 import scenes, shard, sph, tune
from paper_2311_15088_gb300.sph import Scene

from parity import compare_step, gpu_outputs, lattice_params, oracle_step

pytestmark = pytest.mark.gpu


def _small_batch(k=6):
    """A few batched tanks of varied size plus an empty-boid scene and a
    scene with a different cell size."""
    out = scenes.batched_tanks(n_scenes=k, n_min=300, n_max=6000, b_min=0, b_max=40)
    for sc in out:
        sc["params"] = lattice_params(sc)
    out[1]["params"]["cell_size"] = scenes.f32(out[1]["params"]["h"])
    z = np.zeros((0, 4), np.float32)
    out[2]["boid_pos"], out[2]["boid_vel"] = z, z
    return out


def _cat(scs, key):
    return np.concatenate([sc[key] for sc in scs]) if scs else np.zeros((0, 4), np.float32)


def _batch(scs):
    b = Scene([sc["params"] for sc in scs], [len(sc["fluid_pos"]) for sc in scs],
              [len(sc["boid_pos"]) for sc in scs], diagnostics=True)
    b.set_state(_cat(scs, "fluid_pos"), _cat(scs, "fluid_vel"), _cat(scs, "boid_pos"), _cat(scs, "boid_vel"))
    return b


def _split(arr, counts):
    return np.split(arr, np.cumsum(counts)[:-1])


def _singles(scs, steps):
    out = []
    for sc in scs:
        s = Scene(sc["params"], len(sc["fluid_pos"]), len(sc["boid_pos"]))
        s.set_state(sc["fluid_pos"], sc["fluid_vel"], sc["boid_pos"], sc["boid_vel"])
        s.step(steps)
        out.append([t.cpu().numpy() for t in s.get_state()])
    return out


def test_batch_is_bitwise_the_scenes_run_alone():
    scs = _small_batch()
    b = _batch(scs)
    b.step(12)
    fp, fv, bp, bv = (t.cpu().numpy() for t in b.get_state())
    nf = [len(sc["fluid_pos"]) for sc in scs]
    nb = [len(sc["boid_pos"]) for sc in scs]
    alone = _singles(scs, 12)
    for k, (a_fp, a_fv, a_bp, a_bv) in enumerate(alone):
        assert np.array_equal(_split(fp, nf)[k], a_fp), f"scene {k} positions"
        assert np.array_equal(_split(fv, nf)[k], a_fv), f"scene {k} velocities"
        assert np.array_equal(_split(bp, nb)[k], a_bp), f"scene {k} boid positions"
        assert np.array_equal(_split(bv, nb)[k], a_bv), f"scene {k} boid velocities"


@pytest.mark.parametrize("k", [3, 1])
def test_batch_first_step_against_oracle(k):
    """Scene k of a batch, one step, every field against the oracle (the
    batch's fields carry global ids; they are mapped back to the scene's);
    scene 3 has cells of h/2, scene 1 cells of h."""
    scs = _small_batch()
    b = _batch(scs)
    b.step(1)
    g = gpu_outputs(b)
    nf = np.array([len(sc["fluid_pos"]) for sc in scs])
    nb = np.array([len(sc["boid_pos"]) for sc in scs])
    sc = scs[k]
    B_all = int(nb.sum())
    ids = np.concatenate([nb[:k].sum() + np.arange(nb[k]), B_all + nf[:k].sum() + np.arange(nf[k])])
    o = oracle_step(sc["params"], sc)
    local = {}
    for name in ("rho", "pressure", "acc", "touched", "influence", "nbr_count"):
        local[name] = g[name][ids]
    local["fb"] = g["fb"][nb[:k].sum():nb[:k + 1].sum()]
    for name, cnt in (("new_fluid_pos", nf), ("new_fluid_vel", nf)):
        local[name] = g[name][cnt[:k].sum():cnt[:k + 1].sum()]
    for name in ("new_boid_pos", "new_boid_vel"):
        local[name] = g[name][nb[:k].sum():nb[:k + 1].sum()]
    # binning: the scene's keys are offset by the cells of the scenes before it
    cells_before = sum(int(np.prod(oracle.grid_dims(s["params"], 0))) for s in scs[:k])
    local["keys"] = (g["keys"][ids] - cells_before).astype(np.uint32)
    ncell = int(np.prod(oracle.grid_dims(sc["params"], 0)))
    cs = g["cell_start"][cells_before:cells_before + ncell + 1].astype(np.int64)
    local["cell_start"] = (cs - cs[0]).astype(np.uint32)
    remap = np.full(B_all + int(nf.sum()), -1, np.int64)
    remap[ids] = np.arange(len(ids))
    local["perm"] = remap[g["perm"][cs[0]:cs[-1]]].astype(np.int32)
    bcells_before = sum(int(np.prod(oracle.grid_dims(s["params"], 1))) for s in scs[:k])
    nbcell = int(np.prod(oracle.grid_dims(sc["params"], 1)))
    local["boid_keys"] = (g["boid_keys"][nb[:k].sum():nb[:k + 1].sum()] - bcells_before).astype(np.uint32)
    bcs = g["boid_cell_start"][bcells_before:bcells_before + nbcell + 1].astype(np.int64)
    local["boid_cell_start"] = (bcs - bcs[0]).astype(np.uint32)
    local["boid_perm"] = (g["boid_perm"][bcs[0]:bcs[-1]] - nb[:k].sum()).astype(np.int32)
    compare_step(sc["params"], local, o, int(nb[k]))


def test_graph_replay_equals_step():
    scs = _small_batch()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        a = _batch(scs)
        a.step(8)
        b = _batch(scs)
        b.graph_step(8)
        sa = [t.cpu().numpy() for t in a.get_state()]
        sb = [t.cpu().numpy() for t in b.get_state()]
    for x, y in zip(sa, sb):
        assert np.array_equal(x, y)
    assert b.launches > a.launches * 0.5


@pytest.mark.parametrize("block,use_segments,ppt,tile,pblock",
                         [(64, 0, 1, 0, 256), (128, 1, 2, 0, 256), (256, 0, 4, 0, 256), (512, 0, 1, 0, 256),
                          (512, 1, 4, 0, 256), (64, 1, 2, 0, 256), (256, 1, 1, 32, 128), (256, 1, 1, 512, 256),
                          (256, 0, 2, 2048, 256), (256, 1, 1, 65536, 128)])
def test_launch_shape_changes_no_bit(block, use_segments, ppt, tile, pblock):
    """Block size, particles per thread, the source of the force pass's
    pairs (hit segments or a second candidate test) and the fused persistent
    pipeline (both passes in one cooperative launch over work tiles of any
    size) change no bit of the state or of the fields."""
    scs = _small_batch()
    ref = _batch(scs)
    ref.step(6)
    t = _batch(scs)
    t.set_tuning(block, use_segments)
    t.set_particles_per_thread(ppt)
    t.set_pipeline(tile, pblock)
    t.step(6)
    for x, y in zip(ref.get_state(), t.get_state()):
        assert torch.equal(x, y)
    for name in ("acc", "touched", "influence", "rho", "fb"):
        assert torch.equal(ref.field(name), t.field(name)), name


def test_diagnostics_switch_changes_no_result():
    """Without diagnostics the step writes no acc, touched or influence (the
    fields are refused) and its state is bit for bit the recorded step's."""
    scs = _small_batch()
    a = _batch(scs)
    b = Scene([sc["params"] for sc in scs], [len(sc["fluid_pos"]) for sc in scs],
              [len(sc["boid_pos"]) for sc in scs])
    b.set_state(_cat(scs, "fluid_pos"), _cat(scs, "fluid_vel"), _cat(scs, "boid_pos"), _cat(scs, "boid_vel"))
    a.step(5)
    b.step(5)
    for x, y in zip(a.get_state(), b.get_state()):
        assert torch.equal(x, y)
    for name in ("rho", "fb", "nbr_count"):
        assert torch.equal(a.field(name), b.field(name)), name
    for name in ("acc", "touched", "influence"):
        with pytest.raises(sph.SphError):
            b.field(name)
    b.set_diagnostics(True)
    b.step(1)
    a.step(1)
    assert torch.equal(a.field("acc"), b.field("acc"))


def test_autotuner_restores_state_and_caches(tmp_path):
    scs = _small_batch()
    b = _batch(scs)
    before = [t.clone() for t in b.get_state()]
    cache = str(tmp_path / "tune.json")
    best = tune.autotune(b, steps=2, cache=cache)
    assert not best["cached"] and len(best["ms_per_step"]) == len(tune.CANDIDATES)
    for x, y in zip(before, b.get_state()):
        assert torch.equal(x, y)
    again = tune.autotune(b, cache=cache)
    assert again["cached"] and again["block"] == best["block"]


def test_rank_shares_step_like_the_scenes_alone():
    """The scene split across two ranks (in one process here: each rank's
    batch built in turn): every scene on one rank, each rank's batched
    handle steps its scenes bit for bit as each scene alone, and the gather
    returns every scene once, in order."""
    scs = _small_batch()
    parts = shard.assign([shard.scene_weight(sc) for sc in scs], 2)
    assert sorted(parts[0] + parts[1]) == list(range(len(scs))) and parts[0] and parts[1]
    local = {}
    for r in range(2):
        rb = shard.RankBatch(scs, parts[r])
        rb.step(6)
        local.update(rb.states())
    out, owner = shard.gather(local, len(scs), 1)
    for k, want in enumerate(_singles(scs, 6)):
        assert owner[k] == 0
        for x, y in zip(out[k], want):
            assert np.array_equal(x[:, :3], y[:, :3])


def test_pipeline_graph_replay_equals_step():
    """The fused pipeline (a cooperative launch) captured in the step's CUDA
    graph and replayed gives the separate launches' bits."""
    scs = _small_batch()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        a = _batch(scs)
        a.step(8)
        b = _batch(scs)
        b.set_pipeline(1024, 256)
        b.graph_step(8)
        sa = [t.cpu().numpy() for t in a.get_state()]
        sb = [t.cpu().numpy() for t in b.get_state()]
    torch.cuda.synchronize()
    for x, y in zip(sa, sb):
        assert np.array_equal(x, y)


def test_pipeline_barrier_wait_gives_up():
    """A bounded wait that runs out: the test hook keeps CTA 0 from arriving
    at the pipeline's grid barrier, so every CTA gives up after its limit
    (about a second), SPH_DEV_TIMEOUT is set and the step returns.  No fault:
    the context stays usable, and after the hook is cleared and a state is
    loaded again the scene steps bit for bit like a fresh one."""
    scs = _small_batch()
    ref = _batch(scs)
    ref.step(3)
    b = _batch(scs)
    b.set_pipeline(256, 256)
    b.step(1)
    assert b.status() & sph.SPH_DEV_TIMEOUT == 0
    sph.sph_debug_barrier_skip(b.handle, 0)
    b.step(1)
    assert b.status() & sph.SPH_DEV_TIMEOUT
    sph.sph_debug_barrier_skip(b.handle, -1)
    b.clear_status()
    b.set_state(_cat(scs, "fluid_pos"), _cat(scs, "fluid_vel"), _cat(scs, "boid_pos"), _cat(scs, "boid_vel"))
    b.step(3)
    assert b.status() == 0
    for x, y in zip(ref.get_state(), b.get_state()):
        assert torch.equal(x, y)
