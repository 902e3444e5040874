"""Oracle of the surface stage -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py``
may import this module; the product library shares no code with it.

It restates, plainly and in float64 (numpy), the two passes of the paper's
surface reconstruction from particles:

* section "Voxel Density": at every corner x of a voxel grid,
  phi(x) = |x - xbar| - rbar with xbar = sum_i w_i x_i, rbar = sum_i w_i r_i,
  w_i = k(|x - x_i| / R) / sum_j k(|x - x_j| / R), k(s) = (1 - s^2)^3, over
  the particles within R of x;
* section "Marching Cubes": the cube index of each cube (bit i set when the
  value at vertex i is below the isovalue), the edges it cuts (edge table),
  the vertex on each cut edge by linear interpolation,
  p = p1 + (iso - v1) / (v2 - v1) (p2 - p1), and the triangles of the
  triangle table, appended cube by cube.

The edge and triangle tables are generated here from the cube's vertex and
edge numbering (the numbering of the paper's worked example: vertex 3 alone
below the isovalue gives cube index 8 and cuts edges 2, 3 and 11), not
copied from anywhere: see :func:`mc_tables`.

Readings (the paper leaves these open):

* neighbours of a corner are the fluid particles with |x - x_i| < R, the
  distance evaluated in float32 exactly as the particle-pair predicate of the
  step (d = x_i - x per component, r2 = fma(dz, dz, fma(dy, dy, dx dx)),
  r2 < fl(R R)); boid-attached particles are not fluid and do not count;
* all particles have the same radius r (rbar = r);
* a corner with no neighbour has phi = R (the listing divides by zero
  there; every particle is at least R away, so the corner is outside);
* corner (ix, iy, iz) lies at fl(origin + fl(i * spacing)) per axis (two
  float32 roundings) and has index ix + nx (iy + ny iz);
* cube (ix, iy, iz) has vertex v at corner (ix, iy, iz) + offset(v) with
  offsets v0 (0,0,0), v1 (1,0,0), v2 (1,1,0), v3 (0,1,0), v4 (0,0,1),
  v5 (1,0,1), v6 (1,1,1), v7 (0,1,1); edges e0 (v0 v1), e1 (v1 v2),
  e2 (v2 v3), e3 (v3 v0), e4 (v4 v5), e5 (v5 v6), e6 (v6 v7), e7 (v7 v4),
  e8 (v0 v4), e9 (v1 v5), e10 (v2 v6), e11 (v3 v7); a cut edge's vertex is
  interpolated from its endpoint with the smaller coordinate (p1, v1) to the
  other (p2, v2), so that the cubes sharing a grid edge compute its vertex
  from the same operands;
* a face with all four edges cut (two diagonal corners below the isovalue)
  is split so that each corner below the isovalue is cut off on its own,
  a rule decided by the face alone, so that the two cubes sharing the face
  agree and the surface is closed;
* triangles wind so that their right-hand normal points to the side below
  the isovalue (the winding of the paper's example triangle 3, 11, 2).
"""
from __future__ import annotations

import numpy as np

VERTS = np.array([(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0), (0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)],
                 dtype=np.int64)
EDGES = [(0, 1), (1, 2), (2, 3), (3, 0), (4, 5), (5, 6), (6, 7), (7, 4), (0, 4), (1, 5), (2, 6), (3, 7)]
# the six faces as vertex cycles, with their outward normals
FACES = [((0, 1, 2, 3), (0, 0, -1)), ((4, 5, 6, 7), (0, 0, 1)), ((0, 1, 5, 4), (0, -1, 0)),
         ((1, 2, 6, 5), (1, 0, 0)), ((2, 3, 7, 6), (0, 1, 0)), ((3, 0, 4, 7), (-1, 0, 0))]
MAX_TRI = 5  # triangles per cube (checked by mc_tables)


def _edge_id(a, b):
    for k, (u, v) in enumerate(EDGES):
        if {u, v} == {a, b}:
            return k
    raise KeyError((a, b))


def _mid(e):
    u, v = EDGES[e]
    return (VERTS[u] + VERTS[v]) / 2.0


def _faces_of(e):
    """The two faces (indices into FACES) that contain edge e."""
    u, v = EDGES[e]
    return {f for f, (cyc, _) in enumerate(FACES) if u in cyc and v in cyc}


def mc_tables():
    """Generate the edge table (256 masks) and the triangle table (256 x 16,
    -1 terminated) of marching cubes.

    For each cube index: every face contributes the segments that cut its
    corners below the isovalue off (one segment between its two cut edges,
    or, with four cut edges, one around each of its two corners below);
    each segment is directed so that (outward face normal) x (direction)
    points to the corners it cuts off; the directed segments chain into
    closed loops (each cut edge starts one segment and ends one); each loop
    is fanned into triangles from its smallest edge number, or from the next
    edge along the loop whose fan puts no triangle in a cube face; loops in
    order of their smallest edge."""
    edge_table = np.zeros(256, dtype=np.int64)
    tri_table = -np.ones((256, 3 * MAX_TRI + 1), dtype=np.int64)
    for ci in range(256):
        inside = [(ci >> v) & 1 == 1 for v in range(8)]
        mask = 0
        for k, (u, v) in enumerate(EDGES):
            if inside[u] != inside[v]:
                mask |= 1 << k
        edge_table[ci] = mask
        nxt = {}
        for cyc, normal in FACES:
            n = np.array(normal, dtype=float)
            cut = [_edge_id(cyc[i], cyc[(i + 1) % 4]) for i in range(4) if inside[cyc[i]] != inside[cyc[(i + 1) % 4]]]
            segs = []  # (edge, edge, the corners this segment cuts off)
            if len(cut) == 2:
                segs.append((cut[0], cut[1], [v for v in cyc if inside[v]]))
            elif len(cut) == 4:
                for i in range(4):
                    if inside[cyc[i]]:
                        a = _edge_id(cyc[(i - 1) % 4], cyc[i])
                        b = _edge_id(cyc[i], cyc[(i + 1) % 4])
                        segs.append((a, b, [cyc[i]]))
            for a, b, corners in segs:
                t = _mid(b) - _mid(a)
                side = np.mean([VERTS[v] for v in corners], axis=0) - (_mid(a) + _mid(b)) / 2.0
                if np.dot(np.cross(n, t), side) < 0:
                    a, b = b, a
                assert a not in nxt
                nxt[a] = b
        tris = []
        left = set(nxt)
        assert left == {k for k in range(12) if (mask >> k) & 1}
        while left:
            e0 = min(left)
            loop = [e0]
            e = nxt[e0]
            while e != e0:
                loop.append(e)
                e = nxt[e]
            left -= set(loop)
            # fan from the first rotation of the loop (from its smallest edge
            # on) whose triangles do not lie in a cube face: a triangle with
            # its three vertices on one face would lie in the face plane,
            # where the neighbouring cube's surface meets only the face's
            # segments
            for r in range(len(loop)):
                rot = loop[r:] + loop[:r]
                fan = [(rot[0], rot[i], rot[i + 1]) for i in range(1, len(rot) - 1)]
                if not any(_faces_of(a) & _faces_of(b) & _faces_of(c) for a, b, c in fan):
                    break
            else:
                raise AssertionError(f"case {ci}: every fan has a triangle in a face")
            for t in fan:
                tris += list(t)
        assert len(tris) <= 3 * MAX_TRI
        tri_table[ci, :len(tris)] = tris
    return edge_table, tri_table


_TABLES = None


def tables():
    global _TABLES
    if _TABLES is None:
        _TABLES = mc_tables()
    return _TABLES


# ----------------------------------------------------------- voxel density

def corner_positions(origin, spacing, dims):
    """float32 corner coordinates per axis: fl(origin + fl(i * spacing))."""
    o = np.asarray(origin, dtype=np.float32)
    s = np.float32(spacing)
    return [(np.arange(dims[a], dtype=np.float32) * s).astype(np.float32) + o[a] for a in range(3)]


def voxel_density(fluid_pos, origin, spacing, dims, radius, particle_radius):
    """phi (float64) and the neighbour count of every corner (index
    ix + nx (iy + ny iz)), from the C oracle's restatement of the section
    (the float32 predicate needs a true float32 fused multiply-add)."""
    import ctypes

    from . import lib

    L = lib()
    P = np.ascontiguousarray(np.asarray(fluid_pos, dtype=np.float32)[:, :3])
    o = np.ascontiguousarray(np.asarray(origin, dtype=np.float32))
    dm = np.ascontiguousarray(np.asarray(dims, dtype=np.int32))
    n = int(dm[0]) * int(dm[1]) * int(dm[2])
    phi = np.empty(n, dtype=np.float64)
    cnt = np.empty(n, dtype=np.int32)
    vp = ctypes.c_void_p
    rc = L.or_voxel_density(ctypes.c_int(len(P)), P.ctypes.data_as(vp), o.ctypes.data_as(vp),
                            ctypes.c_float(float(np.float32(spacing))), dm.ctypes.data_as(vp),
                            ctypes.c_float(float(np.float32(radius))),
                            ctypes.c_float(float(np.float32(particle_radius))),
                            phi.ctypes.data_as(vp), cnt.ctypes.data_as(vp))
    if rc != 0:
        raise ValueError("or_voxel_density: bad arguments")
    return phi, cnt.astype(np.int64)


# ---------------------------------------------------------- marching cubes

def marching_cubes(phi, dims, origin, spacing, iso):
    """Triangles of the iso-surface of a corner grid of float32 values.

    Returns (tris [T, 3, 3] float64, cube [T] int64: the cube index ix +
    (nx-1)(iy + (ny-1) iz) of each triangle, case [T] int64: its cube
    index in the table sense), cubes in ascending order, each cube's
    triangles in table order."""
    edge_table, tri_table = tables()
    nx, ny, nz = dims
    f = np.asarray(phi, dtype=np.float32).reshape(nz, ny, nx)
    isof = np.float32(iso)
    cx, cy, cz = corner_positions(origin, spacing, dims)
    if nx < 2 or ny < 2 or nz < 2:
        return np.zeros((0, 3, 3)), np.zeros(0, np.int64), np.zeros(0, np.int64)
    vals = []
    for (ox, oy, oz) in VERTS:
        vals.append(f[oz:nz - 1 + oz, oy:ny - 1 + oy, ox:nx - 1 + ox])
    ci = np.zeros((nz - 1, ny - 1, nx - 1), dtype=np.int64)
    for v in range(8):
        ci |= (vals[v] < isof).astype(np.int64) << v
    flat = ci.reshape(-1)
    ntri = (tri_table[flat] >= 0).sum(1) // 3
    cubes = np.nonzero(ntri)[0]
    out, cube_of, case_of = [], [], []
    for cube in cubes:
        c = int(flat[cube])
        ix = cube % (nx - 1)
        iy = (cube // (nx - 1)) % (ny - 1)
        iz = cube // ((nx - 1) * (ny - 1))
        pts = {}
        for e in range(12):
            if (edge_table[c] >> e) & 1:
                a, b = EDGES[e]
                if VERTS[a].sum() > VERTS[b].sum():  # from the lower end
                    a, b = b, a
                pa = np.array([cx[ix + VERTS[a][0]], cy[iy + VERTS[a][1]], cz[iz + VERTS[a][2]]], dtype=np.float64)
                pb = np.array([cx[ix + VERTS[b][0]], cy[iy + VERTS[b][1]], cz[iz + VERTS[b][2]]], dtype=np.float64)
                va = float(f[iz + VERTS[a][2], iy + VERTS[a][1], ix + VERTS[a][0]])
                vb = float(f[iz + VERTS[b][2], iy + VERTS[b][1], ix + VERTS[b][0]])
                pts[e] = pa + (float(isof) - va) / (vb - va) * (pb - pa)
        row = tri_table[c]
        for k in range(0, 3 * MAX_TRI, 3):
            if row[k] < 0:
                break
            out.append([pts[row[k]], pts[row[k + 1]], pts[row[k + 2]]])
            cube_of.append(cube)
            case_of.append(c)
    if not out:
        return np.zeros((0, 3, 3)), np.zeros(0, np.int64), np.zeros(0, np.int64)
    return np.array(out), np.array(cube_of, dtype=np.int64), np.array(case_of, dtype=np.int64)
