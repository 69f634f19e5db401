"""Cube-cell topology for ODC (test infrastructure only).

Paper: each crossing cell's crossing edges are partitioned into groups
E^S_{c,1..4}, one per primal face, as in Dual Marching Cubes / MC'03; around
each group 1D and 2D points alternate, so every crossing edge is adjacent to
two 2D points (A.1.1, Fig. A1).  One 3D point is placed per group (Sec. 4
"3D Point Identification").  A manifold fix removes the non-manifold edges
that appear when the ambiguities of two neighbouring cells coincide (A.1.1).

Conventions (shared with the CUDA path as a *definition*, not as code):
  * corner index = dx + 2 dy + 4 dz, config bit i = label of corner i.
  * local edge (axis a, o1, o2) has index 4a + o1 + 2 o2, where o1 is the
    offset along axis (a+1)%3 and o2 along (a+2)%3.
  * local face (a, s) has index 2a + s: the face perpendicular to axis a at
    side s, spanning u = axis (a+1)%3 and v = axis (a+2)%3.  Its corners in
    face order are (u,v) = (0,0), (1,0), (1,1), (0,1); face edge i joins face
    corners i and i+1.

Readings (the paper is silent):
  * A face with 4 crossing edges (two diagonal inside corners) pairs each
    crossing edge with its neighbour around an inside corner, i.e. the
    segments cut off the inside corners.  The rule depends only on the face's
    four labels, so both cells sharing the face agree.  A "flipped" face uses
    the other pairing (segments around the outside corners).
  * Segment slot 0 of a face is the segment holding the lowest crossing face
    edge; slot 1 (ambiguous faces only) is the other.
  * Cycles of a cell are numbered by increasing smallest local edge index.
  * Manifold fix (reading of the cited Wenger 2013 fix): an interior face with
    two segments is flipped when, in *both* cells sharing it, the two segments
    lie on the same cycle (then the dual edge between the two cells' vertices
    would be shared by four quads).  Flips are applied simultaneously in
    rounds until no face qualifies.  A single cycle through both segments of
    a face always splits in two when the face is flipped (the cycle is a
    Jordan curve on the cube's surface, so its two arcs off the face join the
    face's crossing edges without crossing), so the rounds terminate.
"""
from __future__ import annotations

from functools import lru_cache

import numpy as np


def corner_offset(idx: int):
    return (idx & 1, (idx >> 1) & 1, (idx >> 2) & 1)


def corner_index(d) -> int:
    return int(d[0]) + 2 * int(d[1]) + 4 * int(d[2])


def edge_index(a: int, o1: int, o2: int) -> int:
    return 4 * a + o1 + 2 * o2


def edge_axis_offsets(le: int):
    """(axis, o1, o2) of local edge ``le``."""
    a = le // 4
    r = le % 4
    return a, r & 1, r >> 1


def edge_start(le: int):
    """Offset (dx, dy, dz) of the lower corner of local edge ``le``."""
    a, o1, o2 = edge_axis_offsets(le)
    d = [0, 0, 0]
    d[(a + 1) % 3] = o1
    d[(a + 2) % 3] = o2
    return tuple(d)


def edge_corners(le: int):
    a, _, _ = edge_axis_offsets(le)
    d0 = list(edge_start(le))
    d1 = list(d0)
    d1[a] = 1
    return corner_index(d0), corner_index(d1)


def face_edges(f: int):
    """Local edges of local face ``f`` in face-edge order 0..3."""
    a, s = f // 2, f % 2
    b, c = (a + 1) % 3, (a + 2) % 3
    return (edge_index(b, 0, s), edge_index(c, s, 1), edge_index(b, 1, s), edge_index(c, s, 0))


def face_corners(f: int):
    """Local corners of local face ``f`` in face-corner order 0..3."""
    a, s = f // 2, f % 2
    b, c = (a + 1) % 3, (a + 2) % 3
    out = []
    for (u, v) in ((0, 0), (1, 0), (1, 1), (0, 1)):
        d = [0, 0, 0]
        d[a], d[b], d[c] = s, u, v
        out.append(corner_index(d))
    return tuple(out)


def edge_faces(le: int):
    """The two local faces containing local edge ``le``: ((a+1)%3, o1) and ((a+2)%3, o2)."""
    a, o1, o2 = edge_axis_offsets(le)
    return (2 * ((a + 1) % 3) + o1, 2 * ((a + 2) % 3) + o2)


def face_segments(lab4, flip: bool):
    """Segments (pairs of face-edge indices) of a face with corner labels ``lab4``.

    Returned in slot order.  An empty list for a face without crossings.
    """
    cross = [bool(lab4[i]) != bool(lab4[(i + 1) % 4]) for i in range(4)]
    idx = [i for i in range(4) if cross[i]]
    if not idx:
        return []
    if len(idx) == 2:
        return [(idx[0], idx[1])]
    # checkerboard face: corner i is shared by face edges i-1 and i
    want = (not flip)
    corners = [i for i in range(4) if bool(lab4[i]) == want]
    segs = sorted(tuple(sorted(((i - 1) % 4, i))) for i in corners)
    return segs


def _cell_face_labels(config: int, f: int):
    return tuple((config >> c) & 1 for c in face_corners(f))


@lru_cache(maxsize=None)
def cell_cycles(config: int, flips: int = 0):
    """Cycles of a cell: (cycle index per local edge, -1 if not crossing; count).

    ``flips`` has bit f set when local face f uses the flipped pairing.
    """
    partners = {}
    for f in range(6):
        fe = face_edges(f)
        for (i, j) in face_segments(_cell_face_labels(config, f), bool((flips >> f) & 1)):
            partners.setdefault(fe[i], []).append(fe[j])
            partners.setdefault(fe[j], []).append(fe[i])
    cyc = [-1] * 12
    crossing = sorted(partners)
    for le in crossing:
        assert len(partners[le]) == 2, (config, flips, le)
    n = 0
    for le in crossing:            # increasing index -> cycles numbered by min edge
        if cyc[le] >= 0:
            continue
        prev, cur = None, le
        while cyc[cur] < 0:
            cyc[cur] = n
            p0, p1 = partners[cur]
            nxt = p0 if p0 != prev else p1
            if p0 == p1:           # degenerate 2-cycle cannot happen on a cube
                nxt = p0
            prev, cur = cur, nxt
        n += 1
    return tuple(cyc), n


@lru_cache(maxsize=None)
def mc_successors(config: int, flips: int = 0):
    """Oriented order of every cycle of a cell, for marching-cubes polygons
    (Tab. A8's MC variants): successor of each crossing local edge, -1 if not
    crossing.

    Each face boundary is walked counter-clockwise as seen from outside the
    cell (face order for side 1, reversed for side 0: the face spans
    u = (a+1)%3, v = (a+2)%3 with u x v along +a).  A segment runs from the
    face's out->in crossing to its in->out crossing; the surface polygon then
    turns counter-clockwise about its outward normal (inside corners on its
    right when walked on the face from outside).  A crossing edge is an
    out->in crossing on exactly one of its two faces (the faces walk their
    shared edge in opposite directions), where its successor is the other end
    of its segment."""
    nxt = [-1] * 12
    for f in range(6):
        lab4 = _cell_face_labels(config, f)
        fe = face_edges(f)
        side = f % 2
        for (i, j) in face_segments(lab4, bool((flips >> f) & 1)):
            for (x, y) in ((i, j), (j, i)):
                a, b = (x, (x + 1) % 4) if side else ((x + 1) % 4, x)   # walk from corner a to b
                if not lab4[a] and lab4[b]:
                    nxt[fe[x]] = fe[y]
    return tuple(nxt)


def cell_crossing_edges(config: int):
    out = []
    for le in range(12):
        c0, c1 = edge_corners(le)
        if ((config >> c0) & 1) != ((config >> c1) & 1):
            out.append(le)
    return out


def face_slot_of_edge(config: int, flips: int, f: int, le: int) -> int:
    """Slot of the segment of local face ``f`` that contains local edge ``le``."""
    fe = face_edges(f)
    k = fe.index(le)
    for slot, (i, j) in enumerate(face_segments(_cell_face_labels(config, f), bool((flips >> f) & 1))):
        if k in (i, j):
            return slot
    raise ValueError("edge not crossing on face")


def face_same_cycle(config: int, flips: int, f: int) -> bool:
    """True when local face ``f`` has two segments that lie on one cycle."""
    segs = face_segments(_cell_face_labels(config, f), bool((flips >> f) & 1))
    if len(segs) != 2:
        return False
    cyc, _ = cell_cycles(config, flips)
    fe = face_edges(f)
    return cyc[fe[segs[0][0]]] == cyc[fe[segs[1][0]]]


# ---- symmetry group of the cube (for the 22-class check) -------------------

def cube_symmetries():
    """The 48 maps of the cube onto itself, as permutations of the 8 corners."""
    import itertools
    perms = []
    for axes in itertools.permutations(range(3)):
        for flip in itertools.product((0, 1), repeat=3):
            p = []
            for c in range(8):
                d = corner_offset(c)
                nd = [d[axes[k]] ^ flip[k] for k in range(3)]
                p.append(corner_index(nd))
            perms.append(tuple(p))
    return perms


def config_classes():
    """Equivalence classes of the 256 configurations under the 48 symmetries."""
    syms = cube_symmetries()
    seen = {}
    classes = []
    for cfg in range(256):
        if cfg in seen:
            continue
        orbit = set()
        for p in syms:
            img = 0
            for c in range(8):
                if (cfg >> c) & 1:
                    img |= 1 << p[c]
            orbit.add(img)
        for o in orbit:
            seen[o] = len(classes)
        classes.append(sorted(orbit))
    return classes
