"""Surface reconstruction on the GPU (voxel density, marching cubes) against
the oracle of tests' own oracle/surface.py (needs a GB300).

Voxel density: neighbour counts bit-exact (the float32 predicate is the
same on both sides), phi within 1e-5 R (float32 sums of at most a few
hundred terms, each bounded by R).  Marching cubes: both sides take the same
float32 field, so cube indices are exact; the triangle count and order are
exact and the vertices agree within float32 rounding of the interpolation
(|dp| <= 4 ulp of the coordinates plus 1e-6 of the cube spacing)."""
import numpy as np
import pytest
import torch

from oracle import surface as osurf
from paper_2311_15088_gb300 import scenes, sph
from paper_2311_15088_gb300.sph import Scene

from parity import lattice_params

pytestmark = pytest.mark.gpu


def _scene_state(sc, p):
    s = Scene(p, len(sc["fluid_pos"]), len(sc["boid_pos"]))
    s.set_state(sc["fluid_pos"], sc["fluid_vel"], sc["boid_pos"], sc["boid_vel"])
    return s


def _compare_phi(phi, cnt, ophi, ocnt, R):
    assert np.array_equal(cnt, ocnt)
    assert np.all(np.abs(phi.astype(np.float64) - ophi) <= 1e-5 * R), float(np.max(np.abs(phi - ophi)) / R)


@pytest.mark.parametrize("spacing_over_h,R_over_h", [(0.5, 1.0), (0.25, 0.75), (0.4, 1.6)])
def test_voxel_density_matches_oracle(spacing_over_h, R_over_h):
    """The 4,096-particle dam-break (with its 16 boids, whose attached
    particles must not count) on the padded corner grid of the unit box."""
    sc = scenes.dam_break_small()
    p = lattice_params(sc)
    h = float(p["h"])
    sp, R, r = scenes.f32(h * spacing_over_h), scenes.f32(h * R_over_h), scenes.f32(h * 0.25)
    s = _scene_state(sc, p)
    phi, cnt, origin, dims = s.voxel_density(sp, R, r)
    torch.cuda.synchronize()
    assert s.status() & 1 == 0
    ophi, ocnt = osurf.voxel_density(sc["fluid_pos"], origin, sp, dims, R, r)
    _compare_phi(phi.cpu().numpy(), cnt.cpu().numpy(), ophi, ocnt, float(R))
    assert (ocnt > 0).sum() > 1000 and (ocnt == 0).sum() > 1000


def test_voxel_density_column_sampled():
    """The 262,144-particle column: every corner's count and phi, against the
    oracle on a slab of corners."""
    sc = scenes.dam_break_column()
    p = lattice_params(sc)
    h = float(p["h"])
    sp, R, r = scenes.f32(h * 0.5), scenes.f32(h), scenes.f32(h * 0.25)
    s = _scene_state(sc, p)
    phi, cnt, origin, dims = s.voxel_density(sp, R, r)
    torch.cuda.synchronize()
    nx, ny, nz = dims
    phi = phi.cpu().numpy().reshape(nz, ny, nx)
    cnt = cnt.cpu().numpy().reshape(nz, ny, nx)
    z0 = nz // 2
    # the slab's origin is the full grid's corner z0, fl(origin + fl(z0 sp)),
    # and its own corner 0 is fl(that + 0): the same float32 coordinates
    o2 = np.array(origin, np.float32)
    o2[2] = np.float32(np.float32(z0) * np.float32(sp)) + np.float32(origin[2])
    ophi, ocnt = osurf.voxel_density(sc["fluid_pos"], o2, sp, (nx, ny, 1), R, r)
    _compare_phi(phi[z0].reshape(-1), cnt[z0].reshape(-1), ophi, ocnt, float(R))


def _field(seed, dims, kind):
    rng = np.random.default_rng(seed)
    nx, ny, nz = dims
    z, y, x = np.meshgrid(np.linspace(-1, 1, nz), np.linspace(-1, 1, ny), np.linspace(-1, 1, nx), indexing="ij")
    if kind == "spheres":
        f = np.full(z.shape, 1e9)
        for _ in range(6):
            c = rng.uniform(-0.7, 0.7, 3)
            f = np.minimum(f, np.sqrt((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2) - rng.uniform(0.1, 0.35))
    else:
        f = rng.uniform(-1, 1, z.shape)
    return f.astype(np.float32).reshape(-1)


@pytest.mark.parametrize("kind,dims,iso", [("spheres", (40, 33, 29), 0.0), ("noise", (17, 13, 11), 0.1),
                                           ("noise", (65, 2, 9), 0.05), ("spheres", (103, 101, 99), 0.0)])
def test_marching_cubes_matches_oracle(kind, dims, iso):
    """Count, order and vertices against the oracle; the last grid has
    about a million cubes (about four thousand tiles of the tile scan)."""
    phi = _field(len(kind) + dims[0], dims, kind)
    origin, sp = np.array([-1.0, -0.5, 0.25], np.float32), np.float32(0.0625)
    tris, total = sph.marching_cubes(torch.from_numpy(phi).cuda(), dims, origin, float(sp), iso)
    got = tris.cpu().numpy().astype(np.float64)
    want, cube, case = osurf.marching_cubes(phi, dims, origin, sp, iso)
    assert total == len(want) and len(got) == total and total > 0
    span = float(np.abs(origin).max()) + float(sp) * max(dims)
    assert np.all(np.abs(got - want) <= 4 * np.finfo(np.float32).eps * span + 1e-6 * float(sp))


def test_marching_cubes_capacity_and_degenerate_grids():
    dims = (20, 20, 20)
    phi = _field(3, dims, "noise")
    d = torch.from_numpy(phi).cuda()
    full, total = sph.marching_cubes(d, dims, np.zeros(3, np.float32), 0.1, 0.0)
    part, total2 = sph.marching_cubes(d, dims, np.zeros(3, np.float32), 0.1, 0.0, max_tris=100)
    assert total2 == total > 100 and len(part) == 100
    assert torch.equal(part, full[:100])
    pos = torch.ones(20 * 20 * 20, device="cuda")
    none, t0 = sph.marching_cubes(pos, dims, np.zeros(3, np.float32), 0.1, 0.0)
    assert t0 == 0 and len(none) == 0
    flat, t1 = sph.marching_cubes(torch.zeros(20 * 20, device="cuda"), (20, 20, 1), np.zeros(3, np.float32), 0.1, 0.5)
    assert t1 == 0
    with pytest.raises(sph.SphError):
        sph.marching_cubes(d, dims, np.zeros(3, np.float32), -0.1, 0.0)


@pytest.mark.parametrize("cap", [1, 31, 33, 257, 777, 1025, 2600])
def test_marching_cubes_capacity_cuts_any_run(cap):
    """A capacity inside a warp's run of 32 triangles, across the emit
    blocks' runs of 256 and across tiles: the buffer holds exactly the
    first cap triangles of the full output."""
    dims = (40, 33, 29)
    phi = torch.from_numpy(_field(7, dims, "spheres")).cuda()
    origin = np.array([-1.0, -0.5, 0.25], np.float32)
    full, total = sph.marching_cubes(phi, dims, origin, 0.0625, 0.0)
    assert total > 2600
    part, total2 = sph.marching_cubes(phi, dims, origin, 0.0625, 0.0, max_tris=cap)
    assert total2 == total and len(part) == cap
    assert torch.equal(part, full[:cap])


def test_dam_break_surface_is_closed_and_oriented():
    """GPU voxel density then GPU marching cubes on the dam-break column:
    the corner grid extends past the box, so the mesh must be closed; the
    cubes sharing an edge compute its vertex from the same operands, so
    vertices match bit for bit; every mesh edge is traversed once in each
    direction; the enclosed volume (normals point inwards) is that of the
    column to within the particle radius."""
    sc = scenes.dam_break_small()
    p = lattice_params(sc)
    h = float(p["h"])
    sp, R, r = scenes.f32(h * 0.5), scenes.f32(h), scenes.f32(h * 0.25)
    s = _scene_state(sc, p)
    phi, _, origin, dims = s.voxel_density(sp, R, r, counts=False)
    tris, total = sph.marching_cubes(phi, dims, origin, float(sp), 0.0)
    T = tris.cpu().numpy()
    assert total == len(T) > 1000
    keys = {}
    idx = np.empty(T.shape[:2], np.int64)
    for t in range(len(T)):
        for k in range(3):
            idx[t, k] = keys.setdefault(T[t, k].tobytes(), len(keys))
    directed = {}
    for a, b, c in idx:
        for u, v in ((a, b), (b, c), (c, a)):
            directed[(u, v)] = directed.get((u, v), 0) + 1
    assert all(n == 1 and directed.get((v, u)) == 1 for (u, v), n in directed.items())
    T64 = T.astype(np.float64)
    vol = -np.einsum("ij,ij->i", T64[:, 0], np.cross(T64[:, 1], T64[:, 2])).sum() / 6.0
    lo, hi = sc["fluid_pos"][:, :3].min(0), sc["fluid_pos"][:, :3].max(0)
    box = np.prod(hi - lo)
    assert 0.5 * box < vol < np.prod(hi - lo + 2 * R)
