"""The step statistics (sph_stats) on the GPU against the oracle's
definitions (needs a GB300): counts bit-exact, the float sums within the
step's tolerances; per scene in a batch bit for bit what the scene gives
alone."""
import numpy as np
import pytest
import torch

import oracle
from paper_2311_15088_gb300 import scenes, sph
from paper_2311_15088_gb300.sph import Scene

pytestmark = pytest.mark.gpu


def _check(st, ref, p):
    """st: the GPU statistics of one scene, ref: the oracle's."""
    m = float(np.float32(p["mass"]))
    assert st[0] == ref[0] and st[2] == ref[2] and st[3] == ref[3]
    assert st[1] == ref[1]  # the same integer counts summed and divided in float64
    return m


@pytest.mark.parametrize("nf,nb,seed", [(3000, 40, 1), (12000, 400, 2), (40000, 600, 3)])
def test_first_step_statistics_match_oracle(nf, nb, seed):
    sc = scenes.scaled_block(nf, nb, (0.8, 0.55, 0.8), (0.8, 0.55, 0.8), seed=seed)
    p = dict(sc["params"])
    s = Scene(p, nf, nb)
    s.set_state(sc["fluid_pos"], sc["fluid_vel"], sc["boid_pos"], sc["boid_vel"])
    s.step(1)
    st = s.stats().cpu().numpy()[0]
    assert s.status() & 1 == 0
    o = oracle.step(p, sc["fluid_pos"], sc["fluid_vel"], sc["boid_pos"], sc["boid_vel"])
    ref = oracle.step_stats(p, o, nb)
    m = _check(st, ref, p)
    v = np.asarray(o["new_fluid_vel"])
    dt = float(np.float32(p["dt"]))
    # each velocity component agrees within 1e-5 (|v| + dt S_i) (the step's
    # tolerance, S_i the oracle's absolute-sum scale), which bounds the sums
    dv = 1e-5 * (np.abs(v) + dt * np.asarray(o["acc_scale"][nb:])[:, None])
    assert np.all(np.abs(st[4:7] - ref[4:7]) <= m * dv.sum(axis=0) * 1.01)
    assert abs(st[7] - ref[7]) <= m * (np.abs(v) * dv + 0.5 * dv * dv).sum() * 1.01
    assert abs(st[11] - ref[11]) <= np.sqrt((dv * dv).sum(axis=1)).max() * 1.01 + 1e-12
    # densities within 1e-5 relative
    assert np.all(np.abs(st[8:11] - ref[8:11]) <= 1e-5 * ref[8:11])


def test_batch_statistics_equal_scenes_alone_and_host_copy():
    cases = [(3000, 40, 1), (12000, 400, 2), (0, 30, 4), (9000, 0, 5)]
    built = [scenes.scaled_block(nf, nb, (0.8, 0.55, 0.8), (0.8, 0.55, 0.8), seed=sd) if nf else None
             for nf, nb, sd in cases]
    ps, states = [], []
    for (nf, nb, sd), sc in zip(cases, built):
        if sc is None:  # boids only
            base = scenes.scaled_block(3000, nb, (0.8, 0.55, 0.8), (0.8, 0.55, 0.8), seed=sd)
            p = dict(base["params"])
            z = np.zeros((0, 4), np.float32)
            states.append((z, z, base["boid_pos"], base["boid_vel"]))
        else:
            p = dict(sc["params"])
            states.append((sc["fluid_pos"], sc["fluid_vel"], sc["boid_pos"], sc["boid_vel"]))
        ps.append(p)
    alone = []
    for p, (fp, fv, bp, bv) in zip(ps, states):
        s = Scene(p, len(fp), len(bp))
        s.set_state(fp, fv, bp, bv)
        s.step(3)
        alone.append(s.stats().cpu().numpy()[0])
    b = Scene(ps, [len(x[0]) for x in states], [len(x[2]) for x in states])
    b.set_state(*[np.concatenate([x[i] for x in states]) for i in range(4)])
    b.step(3)
    got = b.stats().cpu().numpy()
    assert got.shape == (len(cases), sph.SPH_STATS_N)
    for k in range(len(cases)):
        assert np.array_equal(got[k], alone[k]), k
    # the scene without fluid: zero count, means and density bounds
    assert got[2][0] == 0 and got[2][1] == 0 and np.all(got[2][4:] == 0)
    # the host copy gives the same bits
    host = np.zeros((len(cases), sph.SPH_STATS_N), np.float64)
    sph.sph_stats(b.handle, host.ctypes.data, 1, b.stream)
    assert np.array_equal(host, got)


def test_statistics_need_a_step_and_are_reproducible():
    sc = scenes.scaled_block(5000, 50, (0.8, 0.55, 0.8), (0.8, 0.55, 0.8), seed=7)
    p = dict(sc["params"])
    s = Scene(p, 5000, 50)
    s.set_state(sc["fluid_pos"], sc["fluid_vel"], sc["boid_pos"], sc["boid_vel"])
    out = torch.empty(sph.SPH_STATS_N, dtype=torch.float64, device="cuda")
    with pytest.raises(sph.SphError):
        sph.sph_stats(s.handle, out.data_ptr(), 0, s.stream)
    s.step(2)
    a, b = s.stats(), s.stats()
    assert torch.equal(a, b)
