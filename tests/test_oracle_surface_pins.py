"""The surface oracle (voxel density, marching cubes) pinned to what the
paper prints and to what geometry fixes (CPU)."""
import math
import os

import numpy as np
import pytest

from oracle import surface as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_printed_values.txt")


def _golden():
    out = {}
    for line in open(GOLDEN):
        line = line.split("#", 1)[0].strip()
        if "=" in line:
            k, v = (t.strip() for t in line.split("=", 1))
            out[k] = v
    return out


# ------------------------------------------------------------------ tables

def test_paper_worked_example():
    """Section "Marching Cubes": vertex 3 alone below the isovalue gives cube
    index 8, edge mask 0x80c (edges 2, 3, 11) and the triangle 3, 11, 2."""
    g = _golden()
    et, tt = S.tables()
    ci = 1 << int(g["mc_example_vertex"])
    assert ci == int(g["mc_example_cube_index"])
    assert et[ci] == int(g["mc_example_edge_mask"], 16)
    assert [k for k in range(12) if (et[ci] >> k) & 1] == [int(x) for x in g["mc_example_cut_edges"].split()]
    tri = [int(x) for x in tt[ci] if x >= 0]
    want = [int(x) for x in g["mc_example_triangle"].split()]
    assert len(tri) == 3 and any(tri == want[k:] + want[:k] for k in range(3)), tri  # same triangle, same winding


def test_example_winding_points_below_the_isovalue():
    """The paper's triangle 3, 11, 2 in the cube's coordinates has its
    right-hand normal towards vertex 3, the corner below the isovalue."""
    mid = {e: S._mid(e) for e in range(12)}
    a, b, c = mid[3], mid[11], mid[2]
    n = np.cross(b - a, c - a)
    assert np.dot(n, S.VERTS[3] - (a + b + c) / 3.0) > 0


def test_edge_table_is_the_set_of_edges_with_differing_ends():
    et, tt = S.tables()
    for ci in range(256):
        inside = [(ci >> v) & 1 for v in range(8)]
        want = sum(1 << k for k, (u, v) in enumerate(S.EDGES) if inside[u] != inside[v])
        assert et[ci] == want
        used = {int(x) for x in tt[ci] if x >= 0}
        assert used == {k for k in range(12) if (want >> k) & 1}, ci
    assert et[0] == 0 and et[255] == 0 and (tt[0] < 0).all() and (tt[255] < 0).all()


def test_single_corner_cases_are_one_triangle_around_the_corner():
    et, tt = S.tables()
    for v in range(8):
        for ci in (1 << v, 255 ^ (1 << v)):
            tri = [int(x) for x in tt[ci] if x >= 0]
            assert len(tri) == 3
            assert all(v in S.EDGES[e] for e in tri)
            # winding: normal towards the side below the isovalue
            p = [S._mid(e) for e in tri]
            n = np.cross(p[1] - p[0], p[2] - p[0])
            towards = S.VERTS[v] - sum(p) / 3.0
            sign = 1 if ci == 1 << v else -1
            assert sign * np.dot(n, towards) > 0, (v, ci)


# ------------------------------------------------------- surfaces by MC

def _mesh(tris):
    """Vertices keyed by position (the shared edge vertices of neighbouring
    cubes are computed from the same operands), directed edges."""
    keys = {}
    idx = np.zeros(tris.shape[:2], dtype=np.int64)
    for t in range(len(tris)):
        for k in range(3):
            key = tuple(np.round(tris[t, k], 12))
            idx[t, k] = keys.setdefault(key, len(keys))
    return idx, len(keys)


def _closed_and_oriented(idx):
    directed = {}
    for a, b, c in idx:
        for u, v in ((a, b), (b, c), (c, a)):
            directed[(u, v)] = directed.get((u, v), 0) + 1
    for (u, v), n in directed.items():
        if n != 1 or directed.get((v, u), 0) != 1:
            return False
    return True


def _sample(fn, n, lo=-1.0, hi=1.0):
    s = (hi - lo) / (n - 1)
    origin = np.full(3, lo, np.float32)
    x, y, z = S.corner_positions(origin, s, (n, n, n))
    Z, Y, X = np.meshgrid(z.astype(np.float64), y.astype(np.float64), x.astype(np.float64), indexing="ij")
    return fn(X, Y, Z).astype(np.float32).reshape(-1), origin, np.float32(s)


def test_sphere_mesh_closed_area_volume_euler():
    r = 0.6
    phi, o, s = _sample(lambda X, Y, Z: np.sqrt(X * X + Y * Y + Z * Z) - r, 41)
    tris, cube, case = S.marching_cubes(phi, (41, 41, 41), o, s, 0.0)
    idx, nv = _mesh(tris)
    assert _closed_and_oriented(idx)
    edges = {tuple(sorted(e)) for a, b, c in idx for e in ((a, b), (b, c), (c, a))}
    assert nv - len(edges) + len(idx) == 2  # Euler characteristic of a sphere
    a, b, c = tris[:, 0], tris[:, 1], tris[:, 2]
    area = 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1).sum()
    vol = np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6.0
    assert area == pytest.approx(4 * math.pi * r * r, rel=0.01)
    # normals towards the inside: the signed volume is negative
    assert -vol == pytest.approx(4 / 3 * math.pi * r ** 3, rel=0.01)


def test_torus_has_euler_characteristic_zero():
    R, r = 0.55, 0.22
    phi, o, s = _sample(lambda X, Y, Z: np.sqrt((np.sqrt(X * X + Y * Y) - R) ** 2 + Z * Z) - r, 45)
    tris, _, _ = S.marching_cubes(phi, (45, 45, 45), o, s, 0.0)
    idx, nv = _mesh(tris)
    assert _closed_and_oriented(idx)
    edges = {tuple(sorted(e)) for a, b, c in idx for e in ((a, b), (b, c), (c, a))}
    assert nv - len(edges) + len(idx) == 0


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_noise_fields_give_closed_oriented_meshes(seed):
    """Random fields hit every ambiguous face configuration; with positive
    values on the grid's boundary every surface is closed, so every mesh
    edge must be shared by two triangles that traverse it in opposite
    directions (the face rule is the same in both cubes)."""
    rng = np.random.default_rng(seed)
    n = 14
    f = rng.uniform(-1, 1, (n, n, n)).astype(np.float32)
    f[0], f[-1], f[:, 0], f[:, -1], f[:, :, 0], f[:, :, -1] = 1, 1, 1, 1, 1, 1
    tris, cube, case = S.marching_cubes(f.reshape(-1), (n, n, n), np.zeros(3, np.float32), np.float32(0.1), 0.0)
    assert len(tris) > 500
    amb = 0
    for ci in set(case.tolist()):
        for cyc, _ in S.FACES:
            ins = [(ci >> v) & 1 for v in cyc]
            amb += ins in ([1, 0, 1, 0], [0, 1, 0, 1])
    assert amb > 0  # ambiguous faces occurred
    idx, _ = _mesh(tris)
    assert _closed_and_oriented(idx)


def test_vertices_interpolate_linearly_on_their_edges():
    """A field linear in x: each vertex lies where the linear function
    crosses the isovalue, on the cube edge between its corners."""
    n = 6
    phi, o, s = _sample(lambda X, Y, Z: X - 0.13 + 0 * Y + 0 * Z, n)
    tris, _, _ = S.marching_cubes(phi, (n, n, n), o, s, 0.0)
    assert len(tris) > 0
    assert np.allclose(tris[:, :, 0], 0.13, atol=1e-6)


def test_cube_order_and_counts():
    et, tt = S.tables()
    rng = np.random.default_rng(9)
    dims = (7, 5, 4)
    f = rng.uniform(-1, 1, dims[0] * dims[1] * dims[2]).astype(np.float32)
    tris, cube, case = S.marching_cubes(f, dims, np.zeros(3, np.float32), np.float32(1.0), 0.25)
    assert np.all(np.diff(cube) >= 0)
    F = f.reshape(dims[2], dims[1], dims[0])
    for c in range((dims[0] - 1) * (dims[1] - 1) * (dims[2] - 1)):
        ix, iy, iz = c % 6, (c // 6) % 4, c // 24
        ci = 0
        for v, (ox, oy, oz) in enumerate(S.VERTS):
            ci |= int(F[iz + oz, iy + oy, ix + ox] < np.float32(0.25)) << v
        assert (cube == c).sum() == (tt[ci] >= 0).sum() // 3


# ------------------------------------------------------------ voxel density

def test_voxel_density_single_particle_is_its_distance():
    """One particle: w = 1, xbar = x_1, so phi = |x - x_1| - r within R and
    phi = R (no neighbour) beyond."""
    p = np.array([[0.31, 0.42, 0.27, 0.0]], np.float32)
    dims, origin, sp, R, r = (9, 9, 9), np.zeros(3, np.float32), 0.1, 0.25, 0.05
    phi, cnt = S.voxel_density(p, origin, sp, dims, R, r)
    x, y, z = S.corner_positions(origin, sp, dims)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    d = np.sqrt((X.astype(np.float64) - p[0, 0]) ** 2 + (Y - p[0, 1]) ** 2.0 + (Z - p[0, 2]) ** 2.0).reshape(-1)
    inside = d < R - 1e-6
    outside = d > R + 1e-6
    assert np.all(cnt[inside] == 1) and np.all(cnt[outside] == 0)
    assert np.allclose(phi[inside], d[inside] - np.float32(r), atol=1e-12)
    assert np.all(phi[outside] == np.float32(R))


def test_voxel_density_symmetric_pair_and_weights():
    """Two particles at equal distance from a corner have equal weights:
    xbar is their midpoint; a farther particle gets the smaller weight
    (k decreasing), pulling xbar less."""
    c = np.float32(0.5)
    a = np.array([[0.5 - 0.06, 0.5, 0.5, 0], [0.5 + 0.06, 0.5, 0.5, 0]], np.float32)
    phi, cnt = S.voxel_density(a, np.full(3, c, np.float32), 0.1, (1, 1, 1), 0.2, 0.03)
    assert cnt[0] == 2 and phi[0] == pytest.approx(0.0 - np.float32(0.03), abs=1e-9)
    b = np.array([[0.5 - 0.05, 0.5, 0.5, 0], [0.5 + 0.10, 0.5, 0.5, 0]], np.float32)
    phi, cnt = S.voxel_density(b, np.full(3, c, np.float32), 0.1, (1, 1, 1), 0.2, 0.0)
    R = float(np.float32(0.2))
    k1 = (1 - ((float(c) - float(b[0, 0])) / R) ** 2) ** 3
    k2 = (1 - ((float(b[1, 0]) - float(c)) / R) ** 2) ** 3
    assert k1 > k2
    xbar = (k1 * float(b[0, 0]) + k2 * float(b[1, 0])) / (k1 + k2)
    assert phi[0] == pytest.approx(abs(float(c) - xbar), rel=1e-9)


def test_voxel_neighbour_counts_match_brute_force():
    rng = np.random.default_rng(4)
    P = rng.uniform(0, 1, (3000, 4)).astype(np.float32)
    dims, origin, sp, R = (11, 11, 11), np.zeros(3, np.float32), 0.1, 0.13
    phi, cnt = S.voxel_density(P, origin, sp, dims, R, 0.02)
    x, y, z = S.corner_positions(origin, sp, dims)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    C = np.stack([X.reshape(-1), Y.reshape(-1), Z.reshape(-1)], 1).astype(np.float64)
    d2 = ((C[:, None, :] - P[None, :, :3].astype(np.float64)) ** 2).sum(-1)
    R2 = float(np.float32(R) * np.float32(R))
    # float64 distances decide the same as the float32 predicate except within rounding of R^2
    clear = np.abs(d2 - R2) > 1e-5 * R2
    want = (d2 < R2).sum(1)
    ambiguous = (~clear).sum(1)
    assert np.all(np.abs(cnt - want) <= ambiguous)
    assert (ambiguous == 0).mean() > 0.9
    assert np.all((phi == np.float32(R)) == (cnt == 0))
