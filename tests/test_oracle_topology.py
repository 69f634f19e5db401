"""Pins of the oracle's cell topology (A.1.1, Fig. A1) against brute force.

The paper prints no worked example, so the topology is pinned by what the
mathematics fixes: the 22 classes of Fig. A1, the degree-2 structure of the
cycles around every cell, and closed oriented 2-manifold output on every sign
pattern of a small grid (the manifoldness guarantee of A.1.1).
"""
import multiprocessing as mp

import numpy as np
import pytest

from oracle import bruteforce, meshcheck, odc, topology as topo


def test_22_classes_under_cube_symmetry():
    # Fig. A1: 256 configurations, 22 classes under rotation and mirroring
    assert len(topo.config_classes()) == 22


def test_face_and_edge_tables_are_consistent():
    for f in range(6):
        fe = topo.face_edges(f)
        fc = topo.face_corners(f)
        for i in range(4):
            # face edge i joins face corners i and i+1
            assert set(topo.edge_corners(fe[i])) == {fc[i], fc[(i + 1) % 4]}
        for le in fe:
            assert f in topo.edge_faces(le)
    for le in range(12):
        f1, f2 = topo.edge_faces(le)
        assert le in topo.face_edges(f1) and le in topo.face_edges(f2) and f1 != f2


@pytest.mark.parametrize("flips", [0, 0b111111])
def test_every_config_partitions_its_crossing_edges_into_cycles(flips):
    for cfg in range(256):
        cyc, n = topo.cell_cycles(cfg, flips)
        crossing = topo.cell_crossing_edges(cfg)
        assert sorted(le for le in range(12) if cyc[le] >= 0) == crossing
        if cfg in (0, 255):
            assert n == 0
            continue
        assert 1 <= n <= 4
        sizes = np.bincount([cyc[le] for le in crossing], minlength=n)
        assert np.all(sizes >= 3)            # a primal face has >= 3 sides
        # cycles are numbered by their smallest edge
        firsts = [min(le for le in crossing if cyc[le] == c) for c in range(n)]
        assert firsts == sorted(firsts)


def test_single_corner_is_a_triangle_and_tetrahedral_config_has_four():
    cyc, n = topo.cell_cycles(0b00000001)
    assert n == 1 and sum(c >= 0 for c in cyc) == 3
    # corners 0, 3, 5, 6 inside: every face is ambiguous, inside corners separated
    cyc, n = topo.cell_cycles((1 << 0) | (1 << 3) | (1 << 5) | (1 << 6))
    assert n == 4 and sum(c >= 0 for c in cyc) == 12


def test_ambiguous_pairing_separates_inside_corners():
    # checkerboard face, corners 0 and 2 inside -> segments around corners 0 and 2
    assert topo.face_segments((1, 0, 1, 0), False) == [(0, 3), (1, 2)]
    assert topo.face_segments((1, 0, 1, 0), True) == [(0, 1), (2, 3)]
    assert topo.face_segments((0, 1, 0, 1), False) == [(0, 1), (2, 3)]
    assert topo.face_segments((1, 1, 0, 0), False) == [(1, 3)]


def _run_bruteforce(disable_fix: bool):
    chunks = [(i, min(i + 8192, 1 << 18), disable_fix) for i in range(0, 1 << 18, 8192)]
    with mp.get_context("spawn").Pool(min(8, mp.cpu_count())) as pool:
        res = pool.map(bruteforce.check_range, chunks)
    bad = sum((r[0] for r in res), [])
    return bad, sum(r[1] for r in res), max(r[2] for r in res)


def test_exhaustive_small_grid_is_closed_manifold():
    """All 2^18 inner sign patterns of a 5x5x4 grid mesh to closed 2-manifolds."""
    bad, nflip, rounds = _run_bruteforce(False)
    assert bad == []
    assert nflip > 0 and rounds >= 1


def test_manifold_fix_is_needed():
    """Without the fix some patterns give non-manifold edges (the C12/C18 case)."""
    bad, _, _ = bruteforce.check_range((3645, 3645 + 1024, True))
    assert len(bad) > 0
    bad_fixed, nflip, _ = bruteforce.check_range((3645, 3645 + 1024, False))
    assert bad_fixed == [] and nflip == len(bad)


@pytest.mark.parametrize("density", [0.3, 0.5, 0.7])
def test_random_voxel_grids_are_closed_manifold(density):
    rng = np.random.default_rng(int(density * 100))
    for _ in range(12):
        lab = np.zeros((9, 9, 9), bool)
        lab[1:-1, 1:-1, 1:-1] = rng.random((7, 7, 7)) < density
        tris, t = odc.topology_triangles(lab)
        chk = meshcheck.check_closed_manifold(tris)
        assert chk["ok"], chk


# ---- marching-cubes polygons (Tab. A8's MC variants) ------------------------

def _label_source(lab, lo=-1.0, h=0.5):
    """Occupancy of a label grid: the label of the nearest grid vertex (ties
    to the upper one), so every crossing edge's bisection ends at its middle."""
    nz, ny, nx = lab.shape

    def phi(x):
        idx = np.floor((x - lo) / h + 0.5).astype(np.int64)
        i = np.clip(idx[:, 0], 0, nx - 1)
        j = np.clip(idx[:, 1], 0, ny - 1)
        k = np.clip(idx[:, 2], 0, nz - 1)
        return lab[k, j, i], np.full(x.shape[0], np.inf)
    return phi


def test_mc_polygons_close_and_face_outward_for_every_cell_configuration():
    from oracle import meshcheck, odc
    from paper_2409_13418_gb300 import inputs as I
    g = I.Grid((-1.0, -1.0, -1.0), (0.5, 0.5, 0.5), (3, 3, 3))
    for cfg in range(1, 256):
        lab = np.zeros((4, 4, 4), bool)
        for c in range(8):
            lab[1 + (c >> 2), 1 + ((c >> 1) & 1), 1 + (c & 1)] = (cfg >> c) & 1
        r = odc.extract(_label_source(lab), g, steps_1d=4, mc=True)
        assert meshcheck.check_closed_manifold(r.triangles)["ok"], cfg
        assert meshcheck.signed_volume(r.vertices, r.triangles) > 0, cfg


def test_mc_polygons_on_random_label_grids():
    from oracle import meshcheck, odc
    from paper_2409_13418_gb300 import inputs as I
    rng = np.random.default_rng(11)
    g = I.Grid((-1.0, -1.0, -1.0), (1.0, 1.0, 1.0), (4, 4, 4))
    for _ in range(300):
        lab = np.zeros((5, 5, 5), bool)
        lab[1:4, 1:4, 1:4] = rng.random((3, 3, 3)) < 0.5
        if not lab.any():
            continue
        r = odc.extract(_label_source(lab), g, steps_1d=4, mc=True)
        assert meshcheck.check_closed_manifold(r.triangles)["ok"]
        # the surface bounds the union of the inside vertices' half-cell
        # neighbourhoods: positive volume
        assert meshcheck.signed_volume(r.vertices, r.triangles) > 0


def test_mc_around_a_single_inside_vertex_is_an_octahedron():
    """A sphere of radius 0.3 h around one grid vertex: six crossing edges,
    eight triangles, vertices within 2^-(k+1) h of distance 0.3 h, volume
    (4/3) r^3 of the octahedron with those vertices."""
    from oracle import meshcheck, odc
    from paper_2409_13418_gb300 import inputs as I
    h = 0.25
    src = I.single_prim(I.PRIM_SPHERE, (0.0, 0.0, 0.0), params=(0.3 * h,))
    k = 12
    r = odc.extract(src, I.cube_grid(8), steps_1d=k, mc=True)
    assert r.vertices.shape == (6, 3) and r.triangles.shape == (8, 3)
    d = np.linalg.norm(r.vertices, axis=1)
    assert np.all(np.abs(d - 0.3 * h) <= h * 2.0 ** -(k + 1) + 1e-7)
    vol = meshcheck.signed_volume(r.vertices, r.triangles)
    lo, hi = (4 / 3) * d.min() ** 3, (4 / 3) * d.max() ** 3
    assert lo * (1 - 1e-6) <= vol <= hi * (1 + 1e-6)
