"""CPU-side checks of the step library: it loads, exports every entry point
of include/sph.h, validates its arguments and agrees with the oracle on the
host-side set-up values.  No compute call needs a GPU here."""
import os
import re

import numpy as np
import pytest

from paper_2311_15088_gb300 import scenes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2311_15088_gb300 import build

    build.build()
    from paper_2311_15088_gb300 import sph

    return sph


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "sph.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sph_[a-z_]+)\s*\(", text)))


def test_library_exports_every_declared_entry_point(lib):
    names = _declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib._lib, name), f"{name} is declared in include/sph.h but not exported"
        assert name in lib.EXPORTED, f"{name} has no Python binding"


def test_library_is_independent_of_the_oracle(lib):
    data = open(lib._LIB_PATH, "rb").read()
    assert b"or_step" not in data and b"liboracle" not in data


def _p(**kw):
    p = scenes.default_params(**kw)
    if p["mass"] is None:
        p["mass"] = 0.01
    return p


def test_workspace_size_grows_with_particles(lib):
    a = lib.sph_workspace_size(_p(), 1000, 10)
    b = lib.sph_workspace_size(_p(), 100000, 10)
    assert b - a >= 99000 * 110  # about 120 bytes of per-particle arrays


@pytest.mark.parametrize("bad", [
    dict(h=0.0), dict(cell_size=0.01), dict(mass=-1.0), dict(dt=0.0), dict(box_max=(0.0, 1.0, 1.0)),
    dict(const_set=7), dict(coupling_mode=2), dict(boid_cell_size=0.04), dict(r_sep=0.5),
    dict(v_min=2.0), dict(k=float("nan")), dict(wall_restitution=-1.0), dict(cell_size_x=0.001),
    dict(cell_size_x=float("inf")),
])
def test_invalid_parameters_are_rejected(lib, bad):
    with pytest.raises(lib.SphError) as e:
        lib.sph_workspace_size(_p(**bad), 100, 4)
    assert e.value.code == lib.SPH_ERR_ARG


def test_negative_counts_and_huge_grids(lib):
    with pytest.raises(lib.SphError) as e:
        lib.sph_workspace_size(_p(), -1, 0)
    assert e.value.code == lib.SPH_ERR_ARG
    with pytest.raises(lib.SphError) as e:
        lib.sph_workspace_size(_p(box_max=(2000.0, 2000.0, 2000.0)), 10, 0)
    assert e.value.code == lib.SPH_ERR_OVERFLOW


def test_grid_dims_match_oracle(lib, orc):
    for p in (_p(), _p(box_max=(2.0, 1.0, 1.0)), _p(box_max=(4.0, 2.0, 2.0))):
        assert lib.sph_grid_dims(p, 0) == orc.grid_dims(p, 0)
        assert lib.sph_grid_dims(p, 1) == orc.grid_dims(p, 1)
    h = scenes.default_params()["h"]
    assert lib.sph_grid_dims(_p(box_max=(4.0, 2.0, 2.0), cell_size=h), 0) == (88, 44, 44)
    assert lib.sph_grid_dims(_p(box_max=(4.0, 2.0, 2.0)), 0) == (176, 88, 88)
    assert lib.sph_grid_dims(_p(box_max=(4.0, 2.0, 2.0)), 1) == (22, 11, 11)
    q = _p(box_max=(4.0, 2.0, 2.0), cell_size_x=h / 4)
    dx = np.float64(np.float32(q["cell_size_x"]))
    assert lib.sph_grid_dims(q, 0) == orc.grid_dims(q, 0) == (int(np.ceil(4.0 / dx)), 88, 88)
    assert lib.sph_grid_dims(q, 1) == (22, 11, 11)  # the boid grid keeps cubic cells


@pytest.mark.parametrize("spacing", [0.02285, 1.0 / 64, 0.03])
def test_lattice_mass_matches_oracle(lib, orc, spacing):
    p = _p()
    assert lib.sph_lattice_mass(p, spacing) == pytest.approx(orc.lattice_mass(p, np.float32(spacing)), rel=1e-6)


def test_library_mc_tables_equal_the_oracle_generator(lib):
    """The library and the oracle each generate the marching-cubes tables
    from the cube's numbering (two independent implementations of the same
    rules); they must agree entry for entry, and the library's must hold
    the paper's worked example (cube index 8: edges 2, 3, 11; triangle
    3, 11, 2 up to rotation)."""
    import numpy as np

    from oracle import surface

    e, t = lib.sph_mc_tables()
    oe, ot = surface.tables()
    assert np.array_equal(e.astype(np.int64), oe)
    assert np.array_equal(t.astype(np.int64), ot)
    assert e[8] == 0x80C and list(t[8][:4]) == [2, 3, 11, -1]


def test_surrogate_per_query_error_by_hand():
    """Median and 90th percentile of |dF| / max(|F|, 0.05 RMS F): three
    queries worked by hand (RMS |F| = sqrt(5/3), floor 0.0645...)."""
    import math

    import torch

    from paper_2311_15088_gb300 import surrogate

    F = torch.tensor([[1.0, 0.0, 0.0], [0.0, 2.0, 0.0], [0.0, 0.0, 0.0]], dtype=torch.float64)
    Fu = F + torch.tensor([[0.1, 0.0, 0.0], [0.0, 0.0, 0.0], [0.0, 0.0, 0.01]], dtype=torch.float64)
    med, p90 = surrogate.per_query_error(Fu, F)
    floor = 0.05 * math.sqrt(5.0 / 3.0)
    rel = sorted([0.1, 0.0, 0.01 / floor])
    assert med == pytest.approx(rel[1], rel=1e-12)
    assert p90 == pytest.approx(rel[1] + 0.8 * (rel[2] - rel[1]), rel=1e-12)
