"""Generate the marching-cubes case table ``mc_table.h`` (paper Sec. 2.2: the
surface in a cell is determined by its case; Lorensen & Cline marching cubes).

The table is derived geometrically here rather than copied from any published
table.  For every one of the 256 inside-corner patterns of a cell:

1. On each face, inside corners that are joined by a face edge form groups;
   a face with all four corners inside (or none) has no segment.  Each group
   is cut off by one segment between the two crossing points (edge midpoints
   suffice for the topology) on the face edges that leave the group.  Two
   diagonal inside corners are therefore kept apart.
2. The segment is directed so that the group lies to its right when the face
   is viewed from outside: ((B - A) x (P - A)) . n_out < 0 for a group corner P.
   This makes every triangle normal point away from the inside (v < k).
3. Segments chain into closed cycles; cycles are ordered by their smallest
   edge number and listed from it.
4. Each cycle is fanned from the first vertex none of whose diagonals joins
   two crossing points lying in one face plane (midpoints sharing a 0/1
   coordinate); the neighbouring cell could draw such a diagonal too.

Edge numbering: axis*4 + (offsets along the two other axes, lower axis in
bit 0); an edge runs from its corner with offset 0 along its axis.  Corner j
sits at (j&1, j>>1&1, j>>2&1).

Output: ``CHR_MC_CASE[256]`` 64-bit words; bits 12*t + 4*c .. +3 hold the
edge of corner c of triangle t, bits 60..63 the triangle count.

Run ``python gen_mc_table.py`` to rewrite mc_table.h next to this file.
"""
from __future__ import annotations

import os

import numpy as np

CORNERS = [np.array([(j >> 0) & 1, (j >> 1) & 1, (j >> 2) & 1], float) for j in range(8)]


def _edges():
    """edge number -> (corner a, corner b) with a the offset-0 end."""
    out = {}
    for axis in range(3):
        others = [a for a in range(3) if a != axis]
        for m in range(4):
            off = [0, 0, 0]
            off[others[0]] = m & 1
            off[others[1]] = (m >> 1) & 1
            ca = off[0] | (off[1] << 1) | (off[2] << 2)
            cb = ca | (1 << axis)
            out[axis * 4 + m] = (ca, cb)
    return out


EDGES = _edges()
EDGE_OF_PAIR = {frozenset(v): e for e, v in EDGES.items()}
MID = {e: (CORNERS[a] + CORNERS[b]) / 2 for e, (a, b) in EDGES.items()}


def _faces():
    faces = []
    for axis in range(3):
        for side in (0, 1):
            corners = [j for j in range(8) if ((j >> axis) & 1) == side]
            n = np.zeros(3)
            n[axis] = 1.0 if side else -1.0
            faces.append((corners, n))
    return faces


FACES = _faces()


def _face_segments(caseb, corners, n_out):
    inside = [j for j in corners if (caseb >> j) & 1]
    if len(inside) in (0, 4):
        return []
    # groups of inside corners joined by face edges (corners differing in one bit)
    groups, seen = [], set()
    for j in inside:
        if j in seen:
            continue
        grp, stack = [], [j]
        seen.add(j)
        while stack:
            c = stack.pop()
            grp.append(c)
            for d in inside:
                if d not in seen and bin(c ^ d).count("1") == 1:
                    seen.add(d)
                    stack.append(d)
        groups.append(grp)
    segs = []
    for grp in groups:
        leaving = []
        for c in grp:
            for d in corners:
                if bin(c ^ d).count("1") == 1 and not (caseb >> d) & 1:
                    leaving.append(EDGE_OF_PAIR[frozenset((c, d))])
        assert len(leaving) == 2, (caseb, grp, leaving)
        a, b = leaving
        P = CORNERS[grp[0]]
        side = np.dot(np.cross(MID[b] - MID[a], P - MID[a]), n_out)
        assert side != 0
        segs.append((a, b) if side < 0 else (b, a))
    return segs


def _share_face_plane(ea, eb):
    pa, pb = MID[ea], MID[eb]
    return any(pa[i] == pb[i] and pa[i] in (0.0, 1.0) for i in range(3))


def case_triangles(caseb: int):
    nxt = {}
    for corners, n in FACES:
        for a, b in _face_segments(caseb, corners, n):
            assert a not in nxt
            nxt[a] = b
    tris, done = [], set()
    for start in sorted(nxt):
        if start in done:
            continue
        cyc, e = [], start
        while True:
            cyc.append(e)
            done.add(e)
            e = nxt[e]
            if e == start:
                break
        L = len(cyc)
        apex = None
        for i in range(L):
            bad = any(_share_face_plane(cyc[i], cyc[j]) for j in range(L)
                      if j not in (i, (i + 1) % L, (i - 1) % L))
            if not bad:
                apex = i
                break
        assert apex is not None, (caseb, cyc)
        ring = cyc[apex:] + cyc[:apex]
        for i in range(1, L - 1):
            tris.append((ring[0], ring[i], ring[i + 1]))
    return tris


def build_table():
    table = []
    for caseb in range(256):
        tris = case_triangles(caseb)
        assert len(tris) <= 5
        word = len(tris) << 60
        for t, tri in enumerate(tris):
            for c, e in enumerate(tri):
                word |= e << (12 * t + 4 * c)
        table.append(word)
    return table


def render(table) -> str:
    lines = [
        "/* Generated by gen_mc_table.py: marching-cubes case table (see the",
        "   generator for the face rule, orientation and fan order).  Entry",
        "   [case]: bits 12*t + 4*c hold the edge of corner c of triangle t,",
        "   bits 60..63 the triangle count.  Do not edit by hand. */",
        "#pragma once",
        "#include <stdint.h>",
        "#define CHR_MC_MAX_TRI 5",
        "#define CHR_MC_CASE_INIT \\",
        "    { \\",
    ]
    for i in range(0, 256, 4):
        lines.append("        " + ", ".join(f"0x{w:016x}ull" for w in table[i:i + 4]) + ", \\")
    lines.append("    }")
    lines.append("static const uint64_t CHR_MC_CASE[256] = CHR_MC_CASE_INIT;")
    return "\n".join(lines) + "\n"


def main():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "mc_table.h")
    with open(path, "w") as fh:
        fh.write(render(build_table()))
    print("wrote", path)


if __name__ == "__main__":
    main()
