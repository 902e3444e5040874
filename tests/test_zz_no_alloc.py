"""The allocation-free binning entry point (sph_bin_static) against the
binning of sph_step (needs a GB300).

sph_bin_static serves callers that cannot allocate device memory (code
running inside another framework's hook that owns only its input and
output buffers, or a real-time loop that must not synchronise the device):
its scratch is a fixed static device array.  This file is named so that
pytest collects it last; it must pass alone in a fresh process as well as
after the other tests.
"""
import numpy as np
import pytest
import torch

from paper_2311_15088_gb300 import scenes, sph
from paper_2311_15088_gb300.sph import Scene

pytestmark = pytest.mark.gpu


def _step_binning(p, pos):
    """keys (by index), perm and cell_start of the step's binning."""
    z = np.zeros((0, 4), np.float32)
    s = Scene(p, len(pos), 0)
    s.set_state(pos, np.zeros_like(pos), z, z)
    s.step(1)
    return (s.field("keys").cpu().numpy().view(np.uint32), s.field("perm").cpu().numpy(),
            s.field("cell_start").cpu().numpy().view(np.uint32))


def _static_binning(p, pos, with_flags=False):
    dims = sph.sph_grid_dims(p, 0)
    ncells = dims[0] * dims[1] * dims[2]
    n = len(pos)
    x = torch.from_numpy(pos).cuda()
    keys = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    perm = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    cs = torch.full((ncells + 1,), -1, dtype=torch.int32, device="cuda")
    flags = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    sph.sph_bin_static(p, n, x.data_ptr(), keys.data_ptr(), perm.data_ptr(), cs.data_ptr(),
                       torch.cuda.current_stream().cuda_stream, flags.data_ptr() if with_flags else None)
    torch.cuda.synchronize()
    out = (keys.cpu().numpy().view(np.uint32), perm.cpu().numpy(), cs.cpu().numpy().view(np.uint32))
    return out + (int(flags.item()),) if with_flags else out


def _crowded_column():
    """The 262,144-particle column plus cells of 100 and 9,000 particles, so
    that every path of the per-cell sort runs."""
    sc = scenes.dam_break_column()
    p = dict(sc["params"], mass=0.004)
    rng = np.random.default_rng(1)
    h = p["h"]
    extra = np.concatenate([1.5 + rng.uniform(0, 0.9 * h, size=(9000, 3)),
                            1.2 + rng.uniform(0, 0.9 * h, size=(100, 3))])
    pos = np.zeros((len(sc["fluid_pos"]) + len(extra), 4), np.float32)
    pos[:len(sc["fluid_pos"])] = sc["fluid_pos"]
    pos[len(sc["fluid_pos"]):, :3] = extra
    return p, pos


def test_static_binning_equals_step_binning_on_two_calls_in_a_row():
    p1, pos1 = _crowded_column()
    sc2 = scenes.dam_break_small()
    p2 = dict(sc2["params"], mass=0.01)
    pos2 = sc2["fluid_pos"]
    for p, pos in ((p1, pos1), (p2, pos2)):
        got = _static_binning(p, pos)
        want = _step_binning(p, pos)
        for g, w, name in zip(got, want, ("keys", "perm", "cell_start")):
            assert np.array_equal(g, w), f"{name} differs for {len(pos)} particles"


def test_static_binning_reports_positions_outside_the_box():
    """The call's flag word: 0 for positions inside the box (faces included),
    SPH_DEV_CLAMPED (2) for one outside; the scratch keeps no flag from the
    previous call."""
    sc = scenes.dam_break_small()
    p = dict(sc["params"], mass=0.01)
    pos = sc["fluid_pos"].copy()
    pos[0, :3] = np.asarray(p["box_max"], np.float32)
    pos[1, :3] = np.asarray(p["box_min"], np.float32)
    assert _static_binning(p, pos, with_flags=True)[3] == 0
    pos[2, 0] = np.float32(1.5)
    assert _static_binning(p, pos, with_flags=True)[3] == sph.SPH_DEV_CLAMPED
    pos[2, 0] = np.float32(0.5)
    assert _static_binning(p, pos, with_flags=True)[3] == 0


def test_static_binning_rejects_sizes_beyond_its_limits():
    p = scenes.default_params(mass=0.01)
    with pytest.raises(sph.SphError) as e:
        sph.sph_bin_static(p, sph.SPH_STATIC_MAX_PARTICLES + 1, None, None, None, None, 0)
    assert e.value.code == sph.SPH_ERR_ARG and "SPH_STATIC_MAX_PARTICLES" in str(e.value)
    big = dict(p, box_max=(60.0, 60.0, 60.0))
    with pytest.raises(sph.SphError) as e:
        sph.sph_bin_static(big, 10, None, None, None, None, 0)
    assert e.value.code == sph.SPH_ERR_ARG and "SPH_STATIC_MAX_CELLS" in str(e.value)
