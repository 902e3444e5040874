"""The surrogate's data path and gating on the GPU (needs a GB300)."""
import numpy as np
import pytest
import torch

from oracle.features import stencil_features
from paper_2311_15088_gb300 import scenes, sph, surrogate
from paper_2311_15088_gb300.sph import (SPH_BOID_EXACT, SPH_BOID_EXACT_LOCAL, SPH_BOID_SURROGATE,
                                        SPH_BOID_SURROGATE_FALLBACK, Mlp, Scene)

from parity import lattice_params

pytestmark = pytest.mark.gpu


def _boids_in_fluid(n_fluid=20000, n_boid=500, seed=31):
    sc = scenes.scaled_block(n_fluid, n_boid, (0.8, 0.8, 0.8), (0.8, 0.4, 0.8), seed=seed)
    sc["boid_pos"][:, 1] *= np.float32(0.5)
    rng = np.random.default_rng(seed)
    sc["fluid_vel"][:, :3] = rng.normal(scale=0.2, size=(n_fluid, 3)).astype(np.float32)
    return sc


def _scene(sc, p=None):
    p = p or sc["params"]
    s = Scene(p, len(sc["fluid_pos"]), len(sc["boid_pos"]))
    s.set_state(sc["fluid_pos"], sc["fluid_vel"], sc["boid_pos"], sc["boid_vel"])
    return s


@pytest.mark.parametrize("cell", [0.5, 1.0])
def test_features_match_oracle(cell):
    sc = _boids_in_fluid()
    p = dict(sc["params"], cell_size=scenes.f32(sc["params"]["h"] * cell))
    s = _scene(sc, p)
    x = s.features().float().cpu().numpy()
    ref, scale = stencil_features(p, sc["fluid_pos"], sc["fluid_vel"], sc["boid_pos"], sc["boid_vel"],
                                  with_scale=True)
    # BF16 rounding (2^-9 relative) of float32 sums: 2^-7 of each feature's scale
    assert np.all(np.abs(x - ref) <= 2.0 ** -7 * scale + 1e-30)
    assert (ref[:, 0:256:4] > 0).mean() > 0.3  # the boids sit in fluid
    assert (ref[:, 263] > 0).mean() > 0.3       # and have fluid neighbours


def test_exact_local_is_bitwise_exact():
    sc = _boids_in_fluid()
    s = _scene(sc)
    a = s.boid_forces(SPH_BOID_EXACT)
    b = s.boid_forces(SPH_BOID_EXACT_LOCAL)
    assert torch.equal(a, b)
    assert (a[:, :3].abs().sum(1) > 0).float().mean() > 0.3


def test_fallback_takes_exact_forces_for_flagged_boids():
    sc = _boids_in_fluid()
    s = _scene(sc)
    m = Mlp(512)
    m.set_params(torch.from_numpy(surrogate.init_params(7)))
    exact = s.boid_forces(SPH_BOID_EXACT)
    s.set_surrogate(m, 3.0, 1e9)                 # never falls back
    sur = s.boid_forces(SPH_BOID_SURROGATE)
    y = m.forward(s.features())
    assert torch.equal(sur[:, :3], y[:, :3] * 3.0)
    thr = float(torch.median(y[:, 3]).item())
    s.set_surrogate(m, 3.0, thr)
    mixed = s.boid_forces(SPH_BOID_SURROGATE_FALLBACK)
    flag = s.field("fallback").bool()
    assert torch.equal(flag, y[:, 3] > thr)
    assert 0 < int(flag.sum()) < len(flag)
    assert torch.equal(mixed[flag, :3], exact[flag, :3]) and torch.all(mixed[flag, 3] == 1)
    assert torch.equal(mixed[~flag, :3], sur[~flag, :3]) and torch.all(mixed[~flag, 3] == 0)


def test_fallback_flags_features_out_of_range():
    sc = _boids_in_fluid()
    s = _scene(sc)
    m = Mlp(512)
    m.set_params(torch.from_numpy(surrogate.init_params(5)))
    exact = s.boid_forces(SPH_BOID_EXACT)
    x = s.features().float()
    lo, hi = x.min(0).values.clone(), x.max(0).values.clone()
    s.set_surrogate(m, 3.0, 1e9, (lo, hi))      # the boids' own range: none out
    s.boid_forces(SPH_BOID_SURROGATE_FALLBACK)
    assert int(s.field("fallback").sum()) == 0
    # the density column capped at its median, a velocity column floored
    hi[262] = torch.median(x[:, 262])
    lo[257] = torch.median(x[:, 257])
    s.set_surrogate_bounds((lo, hi))
    mixed = s.boid_forces(SPH_BOID_SURROGATE_FALLBACK)
    flag = s.field("fallback").bool()
    expect = (x[:, 262] > hi[262]) | (x[:, 257] < lo[257])
    assert torch.equal(flag, expect) and 0 < int(flag.sum()) < len(flag)
    assert torch.equal(mixed[flag, :3], exact[flag, :3])
    assert torch.equal(flag, surrogate.out_of_range(s.features(), (lo, hi)))
    s.set_surrogate_bounds(None)
    s.boid_forces(SPH_BOID_SURROGATE_FALLBACK)
    assert int(s.field("fallback").sum()) == 0
    with pytest.raises(RuntimeError):
        sph.sph_set_surrogate_bounds(s.handle, lo.data_ptr(), None)


def test_trained_surrogate_beats_no_network():
    """Train on pairs logged from a 262,144-particle column run and compare
    with predicting the mean force, on pairs from a run of another seed."""
    torch.manual_seed(0)
    mk = lambda sd: scenes.dam_break_column(seed_offset=sd)
    mlp, info = surrogate.build_and_train(mk, [10, 11, 12], [13], steps=40, epochs=6, batch=4096, head_epochs=4)
    assert info["status"] == 0
    assert info["loss_last_epoch"] < info["loss_first_epoch"]
    Xe, Fe, _ = surrogate.log_pairs(scenes.dam_break_column(seed_offset=14), 30)
    ev = surrogate.evaluate(mlp, Xe, Fe, info["f_scale"], info["threshold"])
    assert ev["aggregate_error_surrogate"] < 0.9 * ev["aggregate_error_mean_predictor"], ev
    assert ev["aggregate_error_with_fallback"] <= ev["aggregate_error_surrogate"]
