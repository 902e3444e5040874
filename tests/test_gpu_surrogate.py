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


def _time_modes(s, modes, n_states):
    """Per mode: summed ms of sph_graph_boid_forces (CUDA events on the
    current stream, after two warm-up calls: the plain one and the capture)
    over n_states states one step apart, and the forces."""
    ms = {k: 0.0 for k in modes}
    got = {k: [] for k in modes}
    for _ in range(2):
        for mode in modes.values():
            s.graph_boid_forces(mode)
        s.step(1)
    for _ in range(n_states):
        for name, mode in modes.items():
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            f = s.graph_boid_forces(mode)
            e1.record()
            torch.cuda.synchronize()
            ms[name] += e0.elapsed_time(e1)
            got[name].append(f.clone())
        s.step(1)
    return ms, {k: torch.cat(v) for k, v in got.items()}


def test_surrogate_gain_within_five_percent_in_distribution():
    """What the trained network gains over the method without it, on queries
    it was not trained or calibrated on: trained on 48 runs of the
    262,144-particle column (64 steps each), error head and fallback
    threshold calibrated on 2 more, then 32 states x 1,024 boids of a held-out
    run.  With the gate (error head + input range, the exact F_b where it
    fires) the aggregate error ||F_used - F||_2 / ||F||_2 stays within 5 %,
    and the queries per second beat the faster of the two exact modes (full
    density pass, or densities only where the boids need them); each mode's
    time includes the state's binning, and every mode is replayed from its
    captured graph (sph_graph_boid_forces)."""
    mk = lambda sd: scenes.dam_break_column(seed_offset=100 + sd)
    train_runs = list(range(16)) + list(range(18, 40)) + list(range(41, 51))
    mlp, info = surrogate.build_and_train(mk, train_runs, [16, 17], steps=64, epochs=40)
    assert info["status"] == 0
    sc = mk(40)
    p = dict(sc["params"])
    p["mass"] = sph.sph_lattice_mass(p, sc["lattice_spacing"])  # as the training runs
    modes = {"exact": SPH_BOID_EXACT, "exact_local": SPH_BOID_EXACT_LOCAL, "gated": SPH_BOID_SURROGATE_FALLBACK}
    n_states = 32
    with torch.cuda.stream(torch.cuda.Stream()):
        s = _scene(sc, p)
        s.set_surrogate(mlp, info["f_scale"], info["threshold"], mlp.bounds)
        ms, got = _time_modes(s, modes, n_states)
    F = got["exact"][:, :3]
    assert torch.equal(F, got["exact_local"][:, :3])
    err = surrogate.aggregate_error(got["gated"][:, :3], F)
    q = n_states * s.n_boid
    qps = {k: q / (v * 1e-3) for k, v in ms.items()}
    fallback = float(got["gated"][:, 3].mean().item())
    speedup = qps["gated"] / max(qps["exact"], qps["exact_local"])
    print(f"\nsurrogate gain: aggregate error {err:.4f} with {fallback:.2%} falling back; queries/s gated "
          f"{qps['gated']:.3e}, exact {qps['exact']:.3e}, exact-local {qps['exact_local']:.3e}; "
          f"speed-up {speedup:.2f}x over the faster exact mode")
    assert err <= 0.05, err
    assert speedup > 1.0, (qps, fallback)


def test_graph_boid_forces_equal_plain_calls():
    """Every mode replayed from its captured graph gives the plain call's
    forces bit for bit, over steps of the state, and a new surrogate
    setting is seen by the next replay."""
    sc = _boids_in_fluid()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        a, b = _scene(sc), _scene(sc)
        m = Mlp(512)
        m.set_params(torch.from_numpy(surrogate.init_params(7)))
        for s in (a, b):
            s.set_surrogate(m, 3.0, 0.0)
        modes = (SPH_BOID_EXACT, SPH_BOID_EXACT_LOCAL, SPH_BOID_SURROGATE, SPH_BOID_SURROGATE_FALLBACK)
        pairs = []
        for it in range(4):
            for mode in modes:
                pairs.append((a.boid_forces(mode), b.graph_boid_forces(mode).clone()))
            if it == 2:  # a new gate threshold: recaptured
                for s in (a, b):
                    s.set_surrogate(m, 3.0, 1e9)
            a.step(1)
            b.step(1)
    torch.cuda.synchronize()
    for x, y in pairs:
        assert torch.equal(x, y)
    assert pairs[-1][0][:, 3].sum() == 0  # threshold 1e9: nothing falls back
