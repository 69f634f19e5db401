"""Pins of the oracle's IC quad split (A.1.5, Eqs. A1, A2) against geometry.

The split case rule is checked against what it is for, not against a retyped
formula:

  * A.1.5 defines the envelope of a crossing edge as the union of the four
    tetrahedra (v_in, v_out, c_k, c_k+1); case 1 is valid when its diagonal
    c1 c3 stays inside the envelope, case 2 when c2 c4 does.  A brute-force
    test samples each diagonal and asks for barycentric containment in one of
    the four tetrahedra.  On random quads whose 3D points lie in their own
    cells, the oracle's concavity tests must give exactly the valid cases the
    containment test finds (case 1 when both are valid, case 3 when neither
    is).
  * Mistakes planted in a copy of the oracle's rule (one inequality flipped,
    the ring neighbours swapped, the two cases' tests crossed, the tie broken
    the other way) must each disagree with the containment test.
  * A.1.5: with one 3D point per cell the split is intersection-free.  On
    shapes whose every crossing cell holds one cycle, the oracle's rule applied
    to the 3D points held in their cells gives meshes without a single
    intersecting triangle pair (oracle/quality.py's counter), while the plain
    diagonal of Sec. 4 intersects on the same points.
"""
import inspect
import math
import textwrap

import numpy as np
import pytest

from oracle import odc, quality
from paper_2409_13418_gb300 import inputs as I

# 3D-point cells around an edge along +x, in the ring order A.1.5 asks for
# when v_in is the edge's lower end (the normal of the centres c1, c2, c3
# points along v_in -> v_out): (y, z) quadrants (+,+), (-,+), (-,-), (+,-).
_QUAD = np.array([(0, 0), (-1, 0), (-1, -1), (0, -1)], np.float64)


def _rotation(rng):
    q = rng.normal(size=4)
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def random_quads(n, seed):
    """n quads with each 3D point uniform in its own cell, edge ends at x = 0
    and x = 1 (either one inside), rigidly rotated at random."""
    rng = np.random.default_rng(seed)
    P = np.zeros((n, 4, 3))
    P[:, :, 0] = rng.uniform(0, 1, (n, 4))
    P[:, :, 1:] = _QUAD[None] + rng.uniform(0, 1, (n, 4, 2))
    lower_in = rng.random(n) < 0.5
    p_in = np.where(lower_in[:, None], 0.0, np.array([1.0, 0, 0]))
    p_out = np.where(lower_in[:, None], np.array([1.0, 0, 0]), 0.0)
    # with v_in at the upper end the ring runs the other way round
    P[~lower_in] = P[~lower_in][:, [0, 3, 2, 1]]
    for q in range(n):
        R = _rotation(rng)
        P[q] = P[q] @ R.T
        p_in[q] = R @ p_in[q]
        p_out[q] = R @ p_out[q]
    return P, p_in, p_out


def diagonal_depth(P, p_in, p_out, i, j, n_samples=256):
    """How deep the open segment P_i P_j stays inside the envelope (the union
    of the tetrahedra (v_in, v_out, c_k, c_k+1)): over samples x(t), the
    largest smallest-barycentric-coordinate among the four tetrahedra,
    divided by the distance in t to the nearer end (the segment ends on the
    envelope's vertices), minimised over t.  > 0: inside, < 0: it leaves."""
    Q = P.shape[0]
    M = np.zeros((Q, 4, 3, 3))
    for k in range(4):
        M[:, k, :, 0] = p_out - p_in
        M[:, k, :, 1] = P[:, k] - p_in
        M[:, k, :, 2] = P[:, (k + 1) % 4] - p_in
    Minv = np.linalg.inv(M)
    t = np.linspace(0.01, 0.99, n_samples)
    x = P[:, i, None, :] + t[None, :, None] * (P[:, j] - P[:, i])[:, None, :]       # (Q, S, 3)
    lam = np.einsum("qkab,qsb->qksa", Minv, x[:, :, :] - p_in[:, None, :])         # (Q, 4, S, 3)
    lam0 = 1.0 - lam.sum(axis=3)
    depth = np.minimum(lam0, lam.min(axis=3)).max(axis=1)                           # (Q, S)
    return (depth / np.minimum(t, 1 - t)[None]).min(axis=1)


def _expected_case(d13, d24):
    ok1, ok2 = d13 > 0, d24 > 0
    return np.where(ok1, 1, np.where(ok2, 2, 3))


def _clear(d13, d24, mindet):
    return (np.abs(d13) > 1e-3) & (np.abs(d24) > 1e-3) & (mindet > 1e-4)


def test_ic_case_equals_envelope_containment():
    P, p_in, p_out = random_quads(2000, seed=11)
    case, mindet = odc.ic_cases(P, p_in, p_out)
    d13 = diagonal_depth(P, p_in, p_out, 0, 2)
    d24 = diagonal_depth(P, p_in, p_out, 1, 3)
    keep = _clear(d13, d24, mindet)
    assert keep.sum() > 1500
    exp = _expected_case(d13, d24)
    assert np.array_equal(case[keep], exp[keep])
    # every case occurs, with both diagonals valid, one of them, or neither
    ok1, ok2 = d13[keep] > 0, d24[keep] > 0
    assert np.sum(ok1 & ok2) > 300 and np.sum(ok1 & ~ok2) > 50 and np.sum(~ok1 & ok2) > 50
    assert np.sum(~ok1 & ~ok2) > 30


# Quads with known geometry (edge v_in = 0 -> v_out = (1, 0, 0)).  In the
# first, c1 and c3 sit near the borders of c2's quadrant, so the diagonal
# c1 c3 runs through c2's quadrant farther from the edge than c2 itself: c2
# lies below (c1, c3, v_out) (Eq. A1) and above (c1, c3, v_in) (Eq. A2),
# the diagonal leaves the envelope and case 2 must be taken.  The others are
# the same quad turned by a quarter around the edge (the concave vertex moves
# to c3, c4, c1) and a quad with every vertex convex (both cases valid:
# case 1 by the tie-break reading).
_C2_CONCAVE = [(0.5, 0.1, 0.9), (0.5, -0.1, 0.1), (0.5, -0.9, -0.1), (0.5, 0.5, -0.4)]


def _turn(P, k):
    """The quad turned by k quarter turns about the edge (+y -> +z), the
    ring relabelled so that c1 stays in the (+, +) quadrant."""
    P = np.asarray(P, np.float64)
    R = np.array([[1, 0, 0], [0, 0, -1], [0, 1, 0]], np.float64)
    for _ in range(k):
        P = P @ R.T
    return np.roll(P, k, axis=0)


@pytest.mark.parametrize("quad,expect", [
    (_turn(_C2_CONCAVE, 0), 2),   # c2 concave: case 1 invalid
    (_turn(_C2_CONCAVE, 1), 1),   # c3 concave: case 2 invalid
    (_turn(_C2_CONCAVE, 2), 2),   # c4 concave
    (_turn(_C2_CONCAVE, 3), 1),   # c1 concave
    ([(0.5, 0.6, 0.4), (0.5, -0.4, 0.6), (0.5, -0.5, -0.4), (0.5, 0.4, -0.6)], 1),   # all convex
])
def test_ic_case_hand_built(quad, expect):
    P = np.asarray(quad, np.float64)[None]
    p_in, p_out = np.zeros((1, 3)), np.array([[1.0, 0, 0]])
    case, _ = odc.ic_cases(P, p_in, p_out)
    assert int(case[0]) == expect
    d13 = diagonal_depth(P, p_in, p_out, 0, 2)[0]
    d24 = diagonal_depth(P, p_in, p_out, 1, 3)[0]
    if expect == 1:
        assert d13 > 0
    else:
        assert d13 < -0.1 and d24 > 0


def test_ic_case_three_when_both_diagonals_leave():
    P, p_in, p_out = random_quads(4000, seed=5)
    case, mindet = odc.ic_cases(P, p_in, p_out)
    d13 = diagonal_depth(P, p_in, p_out, 0, 2)
    d24 = diagonal_depth(P, p_in, p_out, 1, 3)
    both_out = (d13 < -0.05) & (d24 < -0.05) & (mindet > 1e-3)
    assert both_out.sum() >= 20
    assert np.all(case[both_out] == 3)


def _planted(replace_from, replace_to):
    """A copy of the oracle's case rule with one planted mistake."""
    src = textwrap.dedent(inspect.getsource(odc.ic_cases))
    assert replace_from in src, replace_from
    ns = {"np": np}
    exec(src.replace(replace_from, replace_to), ns)
    return ns["ic_cases"]


@pytest.mark.parametrize("frm,to", [
    ("(d_out < 0)", "(d_out > 0)"),                        # Eq. A1 flipped
    ("(d_in > 0)", "(d_in < 0)"),                          # Eq. A2 flipped
    ("pp, pn = P[:, kq], P[:, (kq - 1) % 4], P[:, (kq + 1) % 4]",
     "pp, pn = P[:, kq], P[:, (kq + 1) % 4], P[:, (kq - 1) % 4]"),   # ring neighbours swapped
    ("ok1 = ~(conc[:, 1] | conc[:, 3])", "ok1 = ~(conc[:, 0] | conc[:, 2])"),   # cases' tests crossed
    ("np.where(ok1, 1, np.where(ok2, 2, 3))", "np.where(ok2, 2, np.where(ok1, 1, 3))"),   # tie broken to case 2
])
def test_ic_pin_detects_planted_mistakes(frm, to):
    rule = _planted(frm, to)
    P, p_in, p_out = random_quads(600, seed=3)
    case, mindet = rule(P, p_in, p_out)
    d13 = diagonal_depth(P, p_in, p_out, 0, 2)
    d24 = diagonal_depth(P, p_in, p_out, 1, 3)
    keep = _clear(d13, d24, mindet)
    assert np.sum(case[keep] != _expected_case(d13, d24)[keep]) > 10


def _rot(axis, ang):
    a = np.asarray(axis, float) / np.linalg.norm(axis)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * K @ K


def split_mesh_in_cells(src, grid, k=10, split=True):
    """The oracle's quads on ``grid`` with every 3D point moved into its own
    cell (the premise of the intersection-free guarantee: one point per
    cell, inside it), split by the oracle's case rule (split=True) or along
    c1 c3 everywhere (Sec. 4's plain diagonal)."""
    r = odc.extract(src, grid, steps_1d=k, ic_split=False)
    assert r.cell_ncyc.max() == 1, "the guarantee needs one 3D point per cell"
    X = odc.grid_coords(grid)
    geo = odc._Geo(grid.res)
    C = len(r.cells)
    ci, cj, ck = geo.cijk(r.cells)
    lo = np.stack([X[0][ci], X[1][cj], X[2][ck]], 1)
    hi = np.stack([X[0][ci + 1], X[1][cj + 1], X[2][ck + 1]], 1)
    V = np.clip(r.vertices[:C], lo, hi)
    tri = r.triangles.reshape(-1, 2, 3)          # case 1 everywhere: (c1, c2, c3), (c1, c3, c4)
    Q = tri.shape[0]
    assert Q == len(r.quad_edges)
    ring = np.stack([tri[:, 0, 0], tri[:, 0, 1], tri[:, 0, 2], tri[:, 1, 2]], 1)
    e = r.edges[r.quad_edges]
    v, a = e // 3, e % 3
    ijk = np.stack(geo.vijk(v), 1)
    p0 = np.stack([X[0][ijk[:, 0]], X[1][ijk[:, 1]], X[2][ijk[:, 2]]], 1)
    p1 = p0.copy()
    for ax in range(3):
        m = a == ax
        p1[m, ax] = X[ax][ijk[m, ax] + 1]
    lower_in = r.labels[ijk[:, 2], ijk[:, 1], ijk[:, 0]]
    p_in = np.where(lower_in[:, None], p0, p1)
    p_out = np.where(lower_in[:, None], p1, p0)
    case = odc.ic_cases(V[ring], p_in, p_out)[0] if split else np.ones(Q, np.int64)
    pe = p0 + (p1 - p0) * (r.T[r.quad_edges] / 2.0 ** (k + 1))[:, None]
    verts, tris = [V], []
    for q in range(Q):
        c1, c2, c3, c4 = ring[q]
        if case[q] == 1:
            tris += [(c1, c2, c3), (c1, c3, c4)]
        elif case[q] == 2:
            tris += [(c1, c2, c4), (c2, c3, c4)]
        else:
            pid = C + len(verts) - 1
            verts.append(pe[q:q + 1])
            tris += [(pid, c1, c2), (pid, c2, c3), (pid, c3, c4), (pid, c4, c1)]
    return np.concatenate(verts), np.asarray(tris, np.int64)


@pytest.mark.parametrize("name,src,res", [
    ("two spheres", I.csg_from_list([(I.PRIM_SPHERE, I.OP_UNION, (-0.2, 0, 0), None, (0.45,)),
                                     (I.PRIM_SPHERE, I.OP_UNION, (0.25, 0.04, 0.05), None, (0.38,))]), 28),
    ("sphere minus sphere", I.csg_from_list([(I.PRIM_SPHERE, I.OP_UNION, (0, 0, 0), None, (0.6,)),
                                             (I.PRIM_SPHERE, I.OP_DIFFERENCE, (0.4, 0.35, 0.45), None, (0.35,))]), 20),
    ("sphere minus sphere", I.csg_from_list([(I.PRIM_SPHERE, I.OP_UNION, (0, 0, 0), None, (0.6,)),
                                             (I.PRIM_SPHERE, I.OP_DIFFERENCE, (0.4, 0.35, 0.45), None, (0.35,))]), 28),
    ("sphere", I.single_prim(I.PRIM_SPHERE, (0.03, -0.02, 0.01), params=(0.6,)), 32),
])
def test_ic_split_intersection_free_with_one_point_per_cell(name, src, res):
    g = I.cube_grid(res)
    v1, t1 = split_mesh_in_cells(src, g, split=True)
    n1, _ = quality.self_intersections(v1, t1)
    assert n1 == 0, f"{name} {res}^3: {n1} intersecting pairs after the IC split"
    if name != "sphere":
        v0, t0 = split_mesh_in_cells(src, g, split=False)
        n0, _ = quality.self_intersections(v0, t0)
        assert n0 > 0, f"{name} {res}^3: the plain diagonal should intersect on these points"
