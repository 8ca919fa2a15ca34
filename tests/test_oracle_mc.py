"""Pins for the oracle's marching cubes (paper Sec. 2.2; Lorensen & Cline).

Checks from outside the oracle: hand-derived single cells, closed oriented
2-manifolds for all 256 cases and random grids, Euler characteristics of a
sphere (2), two spheres (4) and a torus (0), exact planes, the enclosed volume
of a sphere, normals that point up the gradient, hand-worked cells with
NaN and infinite corners, and for every case the patch's unshared sides on
its faces, matched in reverse by every neighbouring case across each face."""
import os
from collections import Counter, deque

import numpy as np
import pytest

import oracle
from paper_2408_05462_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _mesh_topology(mesh):
    """(V, E, F, directed-edge multiset) with vertices identified by edge id."""
    tri = mesh.edge_id
    directed = Counter()
    for a, b, c in tri:
        for u, v in ((a, b), (b, c), (c, a)):
            directed[(int(u), int(v))] += 1
    V = len(np.unique(tri))
    E = len({(min(u, v), max(u, v)) for (u, v) in directed})
    return V, E, tri.shape[0], directed


def _assert_closed_oriented(mesh):
    _, _, _, directed = _mesh_topology(mesh)
    for (u, v), n in directed.items():
        assert n == 1, f"directed edge {(u, v)} used {n} times"
        assert directed.get((v, u), 0) == 1, f"edge {(u, v)} has no opposite partner"


def _euler(mesh):
    V, E, F, _ = _mesh_topology(mesh)
    return V - E + F


def _components6(inside):
    nz, ny, nx = inside.shape
    seen = np.zeros_like(inside, bool)
    comps = 0
    for idx in zip(*np.nonzero(inside)):
        if seen[idx]:
            continue
        comps += 1
        dq = deque([idx])
        seen[idx] = True
        while dq:
            z, y, x = dq.popleft()
            for dz, dy, dx in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
                q = (z + dz, y + dy, x + dx)
                if 0 <= q[0] < nz and 0 <= q[1] < ny and 0 <= q[2] < nx and inside[q] and not seen[q]:
                    seen[q] = True
                    dq.append(q)
    return comps


def _read_golden():
    cases, edges = {}, {}
    with open(os.path.join(GOLDEN, "mc_single_cell.txt")) as fh:
        for line in fh:
            p = line.split()
            if not p or p[0].startswith("#"):
                continue
            if p[0] == "case":
                cases[int(p[1])] = [int(v) for v in p[3:]]
            elif p[0] == "edge":
                edges[int(p[1])] = [float(v) for v in p[2:]]
    return cases, edges


def test_golden_single_cells():
    cases, edges = _read_golden()
    for caseb, tri in cases.items():
        got = oracle.cell_triangles(caseb).ravel().tolist()
        assert got == tri, (caseb, got, tri)
        f = np.ones((2, 2, 2), np.float32)
        for j in range(8):
            if (caseb >> j) & 1:
                f[(j >> 2) & 1, (j >> 1) & 1, j & 1] = 0.0
        m = oracle.mc(f, 0.5)
        assert m.ntri == len(tri) // 3
        for t in range(m.ntri):
            for c in range(3):
                assert np.allclose(m.pos[t, c], edges[tri[3 * t + c]], atol=0, rtol=0)


def test_all_256_cases_closed_and_euler():
    # each corner pattern embedded in the middle cell of a 4^3 grid whose other
    # vertices are outside: the surface must close up across the neighbouring
    # cells (crack-free), be consistently oriented, and be one sphere per
    # 6-connected component of inside vertices.
    maxtri = 0
    for caseb in range(256):
        f = np.ones((4, 4, 4), np.float32)
        inside = np.zeros((4, 4, 4), bool)
        for j in range(8):
            if (caseb >> j) & 1:
                z, y, x = 1 + ((j >> 2) & 1), 1 + ((j >> 1) & 1), 1 + (j & 1)
                f[z, y, x] = -1.0
                inside[z, y, x] = True
        m = oracle.mc(f, 0.0)
        if caseb == 0:
            assert m.ntri == 0
            continue
        _assert_closed_oriented(m)
        assert _euler(m) == 2 * _components6(inside), caseb
        maxtri = max(maxtri, oracle.cell_triangles(caseb).shape[0])
    assert maxtri <= 5


def test_random_grids_closed_oriented():
    g = np.random.Generator(np.random.PCG64(3))
    for trial in range(40):
        n = int(g.integers(4, 8))
        f = g.uniform(-1, 1, size=(n, n, n)).astype(np.float32)
        f[0, :, :] = f[-1, :, :] = 1.0
        f[:, 0, :] = f[:, -1, :] = 1.0
        f[:, :, 0] = f[:, :, -1] = 1.0
        m = oracle.mc(f, 0.1)
        _assert_closed_oriented(m)
        assert _euler(m) % 2 == 0


def test_sphere_euler_volume_orientation():
    n = 32
    c = (15.3, 16.1, 14.7)
    r = 10.4
    f = synth.sphere_distance(n, c)
    m = oracle.mc(f, r)
    _assert_closed_oriented(m)
    assert _euler(m) == 2
    p = m.pos
    vol = np.einsum("ti,ti->t", p[:, 0], np.cross(p[:, 1], p[:, 2])).sum() / 6.0
    assert abs(vol - 4.0 / 3.0 * np.pi * r ** 3) < 0.01 * 4.0 / 3.0 * np.pi * r ** 3
    nrm = np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0])
    cen = p.mean(axis=1) - np.array(c)
    assert np.all(np.einsum("ti,ti->t", nrm, cen) > 0), "normals must point away from the inside"


def test_two_spheres_and_torus():
    n = 40
    f = np.minimum(synth.sphere_distance(n, (10.2, 12.1, 11.7)), synth.sphere_distance(n, (28.4, 27.3, 26.9)))
    m = oracle.mc(f, 7.3)
    _assert_closed_oriented(m)
    assert _euler(m) == 4
    t = synth.torus_field(n, (19.6, 20.2, 19.9), 10.0)
    m = oracle.mc(t, 3.5 ** 2)
    _assert_closed_oriented(m)
    assert _euler(m) == 0


def test_plane_exact():
    nx, ny, nz = 13, 9, 20
    f = synth.plane_field((nx, ny, nz), (0, 0, 1), 10.375)  # f = z - 10.375, exact in float32
    m = oracle.mc(f, 0.0)
    assert m.ntri == 2 * (nx - 1) * (ny - 1)
    assert np.all(m.pos[:, :, 2] == 10.375)
    nrm = np.cross(m.pos[:, 1] - m.pos[:, 0], m.pos[:, 2] - m.pos[:, 0])
    assert np.all(nrm[:, 2] > 0) and np.allclose(nrm[:, :2], 0)


def test_tilted_plane_normals_follow_gradient():
    grad = np.array([1.0, 2.0, 3.0])
    f = synth.plane_field(12, grad, 17.25)  # no vertex exactly on k
    m = oracle.mc(f, 0.0)
    assert m.ntri > 0
    nrm = np.cross(m.pos[:, 1] - m.pos[:, 0], m.pos[:, 2] - m.pos[:, 0])
    assert np.all(nrm @ grad > 0)
    # every vertex lies on the plane
    assert np.allclose(m.pos @ grad, 17.25, atol=1e-9)


def test_vertex_on_crossing_edge_and_order():
    f = synth.uniform_noise((7, 6, 5), 9)
    m = oracle.mc(f, 0.2)
    nz, ny, nx = f.shape
    flat = f.ravel()
    assert np.all(np.diff(m.cell) >= 0), "cells ascend"
    step = {0: 1, 1: nx, 2: nx * ny}
    for t in range(m.ntri):
        for c in range(3):
            eid = int(m.edge_id[t, c])
            i0, axis = divmod(eid, 3)
            f0, f1 = flat[i0], flat[i0 + step[axis]]
            assert (f0 < 0.2) != (f1 < 0.2)
            x0, y0, z0 = i0 % nx, (i0 // nx) % ny, i0 // (nx * ny)
            tt = (np.float64(np.float32(0.2)) - f0) / (np.float64(f1) - f0)
            assert 0 < tt <= 1
            exp = np.array([x0, y0, z0], float)
            exp[axis] += tt
            assert np.allclose(m.pos[t, c], exp, atol=1e-12)


def test_value_equal_to_isovalue_is_outside():
    f = np.ones((2, 2, 2), np.float32)
    f[0, 0, 0] = 0.5
    assert oracle.mc(f, 0.5).ntri == 0
    f[0, 0, 0] = np.nextafter(np.float32(0.5), np.float32(0))
    assert oracle.mc(f, 0.5).ntri == 1


def _cell_vertices(f, k):
    """{axis: position} of a one-cell mesh whose triangle sits on vertex 0's
    three edges."""
    m = oracle.mc(f, k)
    assert m.ntri == 1
    out = {}
    for c in range(3):
        i0, axis = divmod(int(m.edge_id[0, c]), 3)
        assert i0 == 0
        out[axis] = m.pos[0, c]
    assert sorted(out) == [0, 1, 2]
    return out


def test_nan_and_infinite_corners():
    # One cell, corner 0 inside (v < k), the rest outside.  A NaN corner is
    # outside (NaN < k is false) and the fraction t = (k - f0) / (f1 - f0)
    # on its edge is NaN; a +inf far end gives t = 0 (the vertex sits on the
    # inside corner); a -inf near end gives inf / inf = NaN on every edge.
    k = np.float32(0.5)
    f = np.ones((2, 2, 2), np.float32)
    f[0, 0, 0] = -1.0
    f[0, 0, 1] = np.nan                      # the +x neighbour of corner 0
    v = _cell_vertices(f, k)
    assert np.isnan(v[0][0]) and v[0][1] == 0.0 and v[0][2] == 0.0
    assert np.array_equal(v[1], [0.0, 0.75, 0.0]) and np.array_equal(v[2], [0.0, 0.0, 0.75])
    f[0, 0, 1] = np.inf
    v = _cell_vertices(f, k)
    assert np.array_equal(v[0], [0.0, 0.0, 0.0])
    f[0, 0, 1] = 1.0
    f[0, 0, 0] = -np.inf
    v = _cell_vertices(f, k)
    for axis in range(3):
        assert np.isnan(v[axis][axis])
        assert np.all(np.delete(v[axis], axis) == 0.0)


def test_body_diagonal_outside_pair_keeps_the_interior_inside():
    # Corners 0 and 7 outside, the other six inside: every face has exactly
    # one outside corner (three inside, no diagonal pair), so each face adds
    # one segment cutting off its outside corner, and the six segments close
    # into two triangles, one around each outside corner.  Edge numbers:
    # axis * 4 + the other two offset bits (lower axis first), so corner 0's
    # edges are 0, 4, 8 and corner 7's are 3, 7, 11.  The cell's interior
    # stays inside and joins the six inside corners, which under 6-adjacency
    # alone form a cycle: why the mesh's Euler characteristic is not twice
    # that of the 6-adjacency cubical complex of the inside vertices.
    caseb = 0xFF & ~(1 | (1 << 7))
    tris = oracle.cell_triangles(caseb)
    assert sorted(sorted(t) for t in tris.tolist()) == [[0, 4, 8], [3, 7, 11]]
    f = np.ones((4, 4, 4), np.float32)
    for j in range(8):
        if (caseb >> j) & 1:
            f[1 + ((j >> 2) & 1), 1 + ((j >> 1) & 1), 1 + (j & 1)] = -1.0
    m = oracle.mc(f, 0.0)
    _assert_closed_oriented(m)
    assert _euler(m) == 2  # one contractible inside region


def _edge_geom(e):
    """Local edge number -> (axis, [x, y, z] offsets, None along the axis):
    axis * 4 + the other two offset bits, lower axis first."""
    a = e >> 2
    others = [ax for ax in range(3) if ax != a]
    c = [None] * 3
    c[others[0]] = e & 1
    c[others[1]] = (e >> 1) & 1
    return a, c


def _edge_num(a, c):
    others = [ax for ax in range(3) if ax != a]
    return 4 * a + c[others[0]] + 2 * c[others[1]]


def _boundary_sides(caseb):
    """Directed sides of a cell's triangles not cancelled by their reverse
    inside the cell (fan diagonals are used twice, once each way)."""
    sides = Counter()
    for tri in oracle.cell_triangles(caseb).tolist():
        for u, v in ((tri[0], tri[1]), (tri[1], tri[2]), (tri[2], tri[0])):
            sides[(u, v)] += 1
    assert all(n == 1 for n in sides.values())
    return {s for s in sides if (s[1], s[0]) not in sides}


def _on_face(e, f, s):
    a, c = _edge_geom(e)
    return a != f and c[f] == s


def test_face_segments_and_shared_face_compatibility():
    # Every side of a cell's surface patch that is not shared inside the cell
    # lies on one of its faces.  Two cells meeting at a face (the +f face of
    # case A and the -f face of case B, with equal corner bits there) put the
    # same segments on it in opposite directions, so the surface continues
    # across the face without a crack: 256 x 3 x 16 pairs.
    bnd = {c: _boundary_sides(c) for c in range(256)}
    for c, sides in bnd.items():
        for u, v in sides:
            assert any(_on_face(u, f, s) and _on_face(v, f, s) for f in range(3) for s in (0, 1)), (c, u, v)
    pairs = 0
    for f in range(3):
        up = [j for j in range(8) if (j >> f) & 1]
        for ca in range(256):
            seg_a = set()
            for u, v in bnd[ca]:
                if _on_face(u, f, 1) and _on_face(v, f, 1):
                    mapped = []
                    for e in (u, v):
                        a, cc = _edge_geom(e)
                        cc[f] = 0
                        mapped.append(_edge_num(a, cc))
                    seg_a.add(tuple(mapped))
            for cb in range(256):
                if any(((ca >> j) & 1) != ((cb >> (j ^ (1 << f))) & 1) for j in up):
                    continue
                seg_b = {(v, u) for u, v in bnd[cb] if _on_face(u, f, 0) and _on_face(v, f, 0)}
                assert seg_a == seg_b, (f, ca, cb)
                pairs += 1
    assert pairs == 3 * 256 * 16
