"""Pins of the FP64 oracle against closed forms and invariants.

Each pin is chosen so that a plausible slip in the oracle (a wrong sign, a
dropped term, a transposed operand, an off-by-one in a search) fails it:
  * 1D points on a sphere lie within 2^-(k+1) cell of the analytic crossing
    (Sec. 5.1; midpoint output reading).
  * Line-binary search output brackets an analytic half-plane crossing
    (A.1.3).
  * Lemma 1 (Sec. 5.2, A.1.2): on a face pierced by the crease of a wedge the
    2D point is the corner u of the two isolines.
  * Planar occupancy gives coplanar 3D points; a single axis-aligned plane
    gives the textbook QEF answer (mass point projected onto the plane).
  * The box corners of the sphere+box union are recovered (QEF, Eq. 2).
  * Euler characteristic 2 for spheres, 0 for a torus, closed manifold
    output, outward orientation and the enclosed volume.
  * The IC split (A.1.5) keeps the Euler characteristic: case 3 adds one
    vertex and two triangles.
  * The MLP evaluator equals a closed form for hand-built weights.
"""
import math

import numpy as np
import pytest

from oracle import meshcheck, odc
from oracle.occupancy import Occupancy, mlp_logit, csg_eval
from paper_2409_13418_gb300 import inputs as I


def _edge_points(r, grid):
    X = odc.grid_coords(grid)
    geo = odc._Geo(grid.res)
    out = []
    for eid in r.edges:
        v, a = int(eid // 3), int(eid % 3)
        ijk = np.array(geo.vijk(v))
        p0 = np.array([X[0][ijk[0]], X[1][ijk[1]], X[2][ijk[2]]])
        p1 = p0.copy()
        p1[a] = X[a][ijk[a] + 1]
        out.append((p0, p1))
    return out


def test_1d_points_on_sphere_within_half_final_interval():
    k = 10
    src = I.single_prim(I.PRIM_SPHERE, (0.03, -0.02, 0.01), params=(0.6,))
    g = I.cube_grid(32)
    r = odc.extract(src, g, steps_1d=k)
    c = src.centers[0].astype(np.float64)
    R = float(src.params[0, 0])
    assert len(r.edges) > 1000
    worst = 0.0
    for (p0, p1), T in zip(_edge_points(r, g), r.T):
        d, f = p1 - p0, p0 - c
        A, B, Cc = d @ d, 2 * f @ d, f @ f - R * R
        disc = math.sqrt(B * B - 4 * A * Cc)
        ts = [t for t in ((-B - disc) / (2 * A), (-B + disc) / (2 * A)) if 0 <= t <= 1]
        assert len(ts) == 1
        worst = max(worst, abs(T / 2 ** (k + 1) - ts[0]))
        assert T % 2 == 1
    # the crossing lies in the final interval of width 2^-k; its midpoint is
    # within 2^-(k+1) (plus the FP32 rounding of query points, < 1e-6 cell)
    assert worst <= 2.0 ** -(k + 1) + 1e-6


def test_1d_dense_scan_brute_force():
    """On a tiny grid the final interval contains the crossing found by a dense scan."""
    k = 8
    src = I.single_prim(I.PRIM_TORUS, (0.01, 0.02, -0.03),
                        rot=I._frame_from_axis((0.3, 0.5, 0.8)), params=(0.45, 0.2))
    g = I.cube_grid(6)
    r = odc.extract(src, g, steps_1d=k)
    phi = Occupancy(src)
    ts = np.linspace(0.0, 1.0, 200001)
    for (p0, p1), T in zip(_edge_points(r, g), r.T):
        lab, _ = phi(p0[None, :] + ts[:, None] * (p1 - p0)[None, :])
        flips = np.nonzero(lab[1:] != lab[:-1])[0]
        lo = (T - 1) / 2 ** (k + 1)
        hi = (T + 1) / 2 ** (k + 1)
        # some sign change of the dense scan lies in the final interval
        locs = (flips + 0.5) / 200000.0
        assert np.any((locs >= lo - 1e-5) & (locs <= hi + 1e-5))


def test_axis_plane_1d_points_are_dyadic_exact():
    # half-space z < 0.3 + 5/1024 (a big box); every z-edge crossing is at the plane
    zc = 0.3 + 5.0 / 1024.0
    src = I.single_prim(I.PRIM_AABB, (0.0, 0.0, zc - 10.0), params=(10.0, 10.0, 10.0))
    g = I.cube_grid(16)
    k = 12
    r = odc.extract(src, g, steps_1d=k)
    X = odc.grid_coords(g)
    zplane = float(np.float32(zc - 10.0)) + float(np.float32(10.0))
    geo = odc._Geo(g.res)
    for eid, T in zip(r.edges, r.T):
        v, a = int(eid // 3), int(eid % 3)
        assert a == 2
        kz = geo.vijk(v)[2]
        t_true = (zplane - X[2][kz]) / (X[2][kz + 1] - X[2][kz])
        assert abs(T / 2 ** (k + 1) - t_true) <= 2.0 ** -(k + 1)
    # all 3D points on the plane within the dyadic bound
    assert np.max(np.abs(r.vertices[:, 2] - zplane)) <= 2.0 ** -(k + 1) * (2 / 16) + 1e-9


def test_single_plane_qef_is_mass_point_projection():
    """Textbook case of Eq. 2: one plane -> mass point projected onto it."""
    src = I.single_prim(I.PRIM_AABB, (0.0, 0.0, -10.0 + 0.2), params=(10.0, 10.0, 10.0))
    g = I.cube_grid(8)
    r = odc.extract(src, g, steps_1d=12)
    X = odc.grid_coords(g)
    geo = odc._Geo(g.res)
    for n, c in enumerate(r.cells):
        ci = geo.cijk(int(c))
        pes = []
        for le in range(12):
            if r.cell_cyc[n, le] < 0:
                continue
            from oracle import topology as topo
            a, _, _ = topo.edge_axis_offsets(le)
            d0 = np.array(topo.edge_start(le))
            gid = 3 * geo.vid(*(np.array(ci) + d0)) + a
            T = r.T[np.searchsorted(r.edges, gid)]
            p = d0.astype(float)
            p[a] = T / 2 ** 13
            pes.append(p)
        cbar = np.mean(pes, axis=0)
        x = r.verts_local[r.vbase[n]]
        assert abs(x[0] - cbar[0]) < 1e-9 and abs(x[1] - cbar[1]) < 1e-9
        assert abs(x[2] - cbar[2]) < 1e-9      # all z equal on a z-plane


def test_line_binary_search_brackets_half_plane():
    """A.1.3: the output keeps p's label and is within one bisection step of
    the crossing along the ray; the q == m case appears when the crossing is
    closer than one step."""
    # a plane crossing a z-face at u = const: inside for x < x0
    for x0 in (0.13, 0.37, 0.51, 0.5002):
        src = I.single_prim(I.PRIM_AABB, (x0 - 10.0, 0.0, 0.0), params=(10.0, 10.0, 10.0))
        g = I.Grid((0.0, -0.5, -0.5), (1.0, 0.5, 0.5), (1, 1, 1))
        r = odc.extract(src, g, steps_1d=14)
        # the plane is parallel to the face's v axis: both 1D points at u = x0,
        # the segment lies on the isoline, Lemma 1's identical case -> p_f = m
        for n in range(len(r.faces)):
            if r.faces[n, 0] % 3 == 2:
                assert abs(r.face_pts[n, 0] - x0) < 2 ** -14


@pytest.mark.parametrize("theta,off", [(0.3, (0.013, 0.021)), (0.7, (0.031, -0.017)),
                                       (1.1, (0.031, -0.017)), (0.05, (0.013, 0.021))])
def test_lemma1_wedge_corner(theta, off):
    """Lemma 1: two isolines through the 1D points meet at u -> p_f = u."""
    Rz = np.array([[math.cos(theta), math.sin(theta), 0], [-math.sin(theta), math.cos(theta), 0], [0, 0, 1]])
    ex = 0.4
    c = np.array([off[0], off[1], 0.0]) - Rz.T @ np.array([ex, ex, 0.0])
    src = I.single_prim(I.PRIM_OBOX, c, rot=Rz, params=(ex, ex, 10.0))
    g = I.cube_grid(16, -0.5, 0.5)
    r = odc.extract(src, g, steps_1d=12)
    M = src.rot[0].astype(np.float64)
    e = src.params[0].astype(np.float64)
    u = src.centers[0].astype(np.float64) + M.T @ np.array([e[0], e[1], 0.0])
    X = odc.grid_coords(g)
    h = 1.0 / 16
    geo = odc._Geo(g.res)
    checked = 0
    for n, (fid, slot) in enumerate(r.faces):
        v, a = int(fid // 3), int(fid % 3)
        if a != 2:
            continue
        i, j, _ = geo.vijk(v)
        fu, fv = (u[0] - X[0][i]) / h, (u[1] - X[1][j]) / h
        if 0.05 < fu < 0.95 and 0.05 < fv < 0.95:
            checked += 1
            # search resolutions: 0.8/4/2^11 ~ 1e-4 (step 1), 0.71/3/2^12 ~ 6e-5 (step 2)
            assert math.hypot(r.face_pts[n, 0] - fu, r.face_pts[n, 1] - fv) < 3e-4
            assert not (r.face_flags[n] & 1)
    assert checked >= 10


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_planar_occupancy_gives_coplanar_3d_points(seed):
    rng = np.random.default_rng(seed)
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    Rm = I._quat_to_rows(q)
    g = I.cube_grid(16, -0.5, 0.5)
    h = 1.0 / 16
    src = I.single_prim(I.PRIM_OBOX, tuple(rng.uniform(-0.05, 0.05, 3) - 0.7 * Rm[2]), rot=Rm,
                        params=(5.0, 5.0, 0.7))
    r = odc.extract(src, g, steps_1d=12)
    M = src.rot[0].astype(np.float64)
    dist = (r.vertices @ M[2] - M[2] @ src.centers[0].astype(np.float64) - float(src.params[0, 2])) / h
    assert len(r.vertices) > 100
    # Lemma 1, identical-lines case: the ray from m crosses the plane within
    # one bisection step, so (almost) every 2D point is the midpoint m
    assert np.mean(r.face_flags & 1) > 0.9
    # 1D points lie within 2^-13 cell of the plane; a normal built from a
    # segment of length L tilts by ~2^-13 / L, so short corner-cutting
    # segments give the tail
    assert np.percentile(np.abs(dist), 95) < 1e-3
    assert np.max(np.abs(dist)) < 1e-2


def test_config1_box_corners_recovered():
    src = I.config1_csg()
    g = I.cube_grid(32)
    k = 10
    r = odc.extract(src, g, steps_1d=k)
    bc = src.centers[1].astype(np.float64)
    be = src.params[1, :3].astype(np.float64)
    sc = src.centers[0].astype(np.float64)
    sr = float(src.params[0, 0])
    h = 1.0 / 16
    n_out = 0
    for sx in (-1, 1):
        for sy in (-1, 1):
            for sz in (-1, 1):
                cor = bc + np.array([sx, sy, sz]) * be
                if np.linalg.norm(cor - sc) <= sr:
                    continue
                n_out += 1
                d = np.min(np.linalg.norm(r.vertices - cor, axis=1)) / h
                # three planes, each offset by at most 2^-(k+1) cell
                assert d <= math.sqrt(3) * 2.0 ** -k
    assert n_out == 6
    chk = meshcheck.check_closed_manifold(r.triangles)
    assert chk["ok"], chk
    assert meshcheck.euler_characteristic(r.triangles) == 2
    assert meshcheck.signed_volume(r.vertices, r.triangles) > 0


def test_sphere_euler_volume_orientation():
    R = 0.6
    src = I.single_prim(I.PRIM_SPHERE, (0.03, -0.02, 0.01), params=(R,))
    g = I.cube_grid(32)
    h = 2.0 / 32
    r = odc.extract(src, g, steps_1d=10)
    assert meshcheck.check_closed_manifold(r.triangles)["ok"]
    assert meshcheck.euler_characteristic(r.triangles) == 2
    vol = meshcheck.signed_volume(r.vertices, r.triangles)
    exact = 4.0 / 3.0 * math.pi * float(src.params[0, 0]) ** 3
    # chords of length ~h on a sphere of radius R cut ~h^2/(8R) deep: the
    # volume deficit is below area * h^2 / (4R)
    assert vol > 0
    assert abs(vol - exact) < 4 * math.pi * R * R * h * h / (4 * R)
    # vertices lie near the sphere
    dist = np.abs(np.linalg.norm(r.vertices - src.centers[0], axis=1) - float(src.params[0, 0])) / h
    assert np.max(dist) < 0.05


def test_torus_has_euler_zero():
    src = I.single_prim(I.PRIM_TORUS, (0.02, -0.01, 0.03), rot=I._frame_from_axis((0.2, 0.3, 0.9)),
                        params=(0.5, 0.22))
    g = I.cube_grid(32)   # minor radius 0.22 = 3.5 h
    r = odc.extract(src, g, steps_1d=10)
    chk = meshcheck.check_closed_manifold(r.triangles)
    assert chk["ok"], chk
    assert meshcheck.euler_characteristic(r.triangles) == 0
    assert meshcheck.components(r.triangles) == 1


def test_two_spheres_euler_four():
    src = I.csg_from_list([(I.PRIM_SPHERE, I.OP_UNION, (-0.45, 0, 0), None, (0.3,)),
                           (I.PRIM_SPHERE, I.OP_UNION, (0.45, 0.05, 0), None, (0.3,))])
    r = odc.extract(src, I.cube_grid(24), steps_1d=10)
    assert meshcheck.euler_characteristic(r.triangles) == 4
    assert meshcheck.components(r.triangles) == 2


def test_ic_split_preserves_euler_and_counts():
    """A.1.5: case 3 adds one vertex (p_e) and turns 2 triangles into 4."""
    src = I.random_csg(5, n_prims=12)
    g = I.cube_grid(24)
    r1 = odc.extract(src, g, steps_1d=10, ic_split=True)
    r0 = odc.extract(src, g, steps_1d=10, ic_split=False)
    n3 = int(np.sum(r1.quad_case == 3))
    assert len(r1.vertices) == len(r0.vertices) + n3
    assert len(r1.triangles) == len(r0.triangles) + 2 * n3
    assert meshcheck.euler_characteristic(r1.triangles) == meshcheck.euler_characteristic(r0.triangles)
    assert meshcheck.check_closed_manifold(r1.triangles)["ok"]
    assert np.all(r0.quad_case == 1)


def test_difference_and_union_semantics():
    src = I.csg_from_list([(I.PRIM_SPHERE, I.OP_UNION, (0, 0, 0), None, (0.5,)),
                           (I.PRIM_SPHERE, I.OP_DIFFERENCE, (0.3, 0, 0), None, (0.3,)),
                           (I.PRIM_SPHERE, I.OP_UNION, (0.3, 0, 0), None, (0.1,))])
    pts = np.array([[-0.3, 0, 0], [0.3, 0, 0], [0.15, 0, 0], [0.45, 0.0, 0.0], [0.9, 0, 0]])
    lab, _ = csg_eval(src, pts)
    assert list(lab) == [True, True, False, False, False]


def test_mlp_closed_form():
    """Hand-built weights make f(x) = sin(2 pi b.x): pins feature order, layer
    order and transposes of the MLP evaluator."""
    b = np.array([[1.25, -0.5, 0.75]], np.float32)
    W1 = np.array([[1, 0], [-1, 0]], np.float32)     # [sin, cos] -> (relu(s), relu(-s))
    Wid = np.eye(2, dtype=np.float32)
    W5 = np.array([[1, -1]], np.float32)
    src = I.MLPSource(B=b, weights=[W1, Wid, Wid, Wid, W5],
                      biases=[np.zeros(2, np.float32)] * 4 + [np.zeros(1, np.float32)])
    rng = np.random.default_rng(0)
    x = rng.uniform(-1, 1, (50, 3)).astype(np.float32).astype(np.float64)
    f = np.sin(2 * np.pi * (x @ b[0].astype(np.float64)))
    z = mlp_logit(src, x)
    expect = 20.0 * ((0.5 - np.linalg.norm(x, axis=1)) + float(np.float32(0.15)) * f)
    assert np.allclose(z, expect, rtol=0, atol=1e-12)
    # with the cos branch selected instead
    W1c = np.array([[0, 1], [0, -1]], np.float32)
    src.weights[0] = W1c
    fc = np.cos(2 * np.pi * (x @ b[0].astype(np.float64)))
    z = mlp_logit(src, x)
    assert np.allclose(z, 20.0 * ((0.5 - np.linalg.norm(x, axis=1)) + float(np.float32(0.15)) * fc), atol=1e-12)


def test_mlp_envelope_sphere_1d_points():
    """With zero network amplitude the envelope is the sphere |x| = 0.5."""
    src = I.envelope_mlp(0, hidden=16, n_freq=8)
    src.env_amp = 0.0
    k = 10
    g = I.cube_grid(16)
    r = odc.extract(src, g, steps_1d=k)
    for (p0, p1), T in zip(_edge_points(r, g), r.T):
        d = p1 - p0
        A, B, Cc = d @ d, 2 * p0 @ d, p0 @ p0 - 0.25
        disc = math.sqrt(B * B - 4 * A * Cc)
        ts = [t for t in ((-B - disc) / (2 * A), (-B + disc) / (2 * A)) if 0 <= t <= 1]
        assert abs(T / 2 ** (k + 1) - ts[0]) <= 2.0 ** -(k + 1) + 1e-6
    assert meshcheck.euler_characteristic(r.triangles) == 2


def test_query_points_are_fp32_rounded():
    src = I.single_prim(I.PRIM_AABB, (0.0, 0.0, 0.0), params=(0.1, 0.1, 0.1))
    e = float(np.float32(0.1))
    p = np.array([[e + 1e-12, 0, 0], [e - 1e-8, 0, 0]])
    lab, _ = csg_eval(src, p)
    # e + 1e-12 rounds to e itself (on the boundary: out); e - 1e-8 (more than
    # half an FP32 ulp of 0.1) rounds below e
    assert list(lab) == [False, True]


def test_replay_of_own_decisions_is_exact_and_detects_planted_errors():
    """Replaying the oracle's own decisions reproduces it with no violation;
    a planted wrong decision (one flipped bisection bit, one flipped label of
    m) is reported as a violation."""
    src = I.random_csg(6, n_prims=10)
    g = I.cube_grid(20)
    r = odc.extract(src, g, steps_1d=10)
    rep = dict(T=r.T, **r.search)
    r2 = odc.extract(src, g, steps_1d=10, replay=rep, replay_margin=1e-12)
    assert r2.stats["edge_violations"] == 0 and r2.stats["face_violations"] == 0
    assert np.array_equal(r2.triangles, r.triangles)
    assert np.array_equal(r2.face_pts, r.face_pts) and np.array_equal(r2.verts_local, r.verts_local)
    bad = dict(rep)
    bad["T"] = r.T.copy()
    bad["T"][5] ^= 1 << 6                      # flip one bisection decision
    bad["lab_m"] = r.search["lab_m"].copy()
    bad["lab_m"][7] = ~bad["lab_m"][7]         # flip the label of one midpoint
    r3 = odc.extract(src, g, steps_1d=10, replay=bad, replay_margin=1e-12)
    assert r3.stats["edge_violations"] == 1
    assert r3.stats["face_violations"] >= 1


def test_serving_trace_is_poisson_with_the_resolution_mix():
    """The serving workload generator: Poisson arrivals (exponential gaps of
    mean 1/rate) and the 0.4/0.3/0.2/0.1 resolution mix."""
    import numpy as np
    from paper_2409_13418_gb300 import inputs as I
    tr = I.serving_trace(0, 40.0, 300.0)
    t = np.array([a for a, _, _ in tr])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(len(tr) / 300.0 - 40.0) < 1.5
    assert abs(gaps.mean() - 1 / 40.0) < 1.5e-3 and abs(gaps.std() / gaps.mean() - 1.0) < 0.05
    res = np.array([r for _, r, _ in tr])
    for r, w in zip((64, 128, 256, 512), (0.4, 0.3, 0.2, 0.1)):
        assert abs(np.mean(res == r) - w) < 0.02
    assert I.serving_trace(0, 40.0, 300.0) == tr


# ---- dense voxel-grid occupancy source ----------------------------------------

def test_voxel_trilinear_reproduces_samples_and_multilinear_fields():
    from oracle import occupancy as O
    from paper_2409_13418_gb300 import inputs as I
    dims = (7, 5, 9)
    lo, hi = (-0.75, -1.0, -0.5), (0.75, 0.5, 1.0)
    xs = [np.linspace(lo[a], hi[a], dims[a]) for a in range(3)]
    zz, yy, xx = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    f = lambda x, y, z: 0.3 * x - 0.2 * y + 0.1 * z + 0.25 * x * y - 0.5 * x * y * z + 0.4   # multilinear
    src = I.VoxelSource(values=f(xx, yy, zz).astype(np.float32), lo=lo, hi=hi)
    vals = src.values.astype(np.float64)
    # at the sample positions: the samples themselves
    idx = np.array([[0, 0, 0], [6, 4, 8], [3, 2, 5], [1, 3, 7]])
    pts = np.stack([xs[0][idx[:, 0]], xs[1][idx[:, 1]], xs[2][idx[:, 2]]], axis=1)
    assert np.allclose(O.voxel_value(src, pts), vals[idx[:, 2], idx[:, 1], idx[:, 0]], rtol=0, atol=1e-6)
    # inside every cell, trilinear interpolation reproduces a multilinear field
    rng = np.random.default_rng(3)
    p = np.stack([rng.uniform(lo[a], hi[a], 2000) for a in range(3)], axis=1).astype(np.float32).astype(np.float64)
    ref = f(p[:, 0], p[:, 1], p[:, 2])
    assert np.max(np.abs(O.voxel_value(src, p) - ref)) < 1e-6      # float32 samples
    # outside the box the value of the nearest face point (clamped)
    q = np.array([[5.0, 0.0, 0.0], [-5.0, -5.0, 5.0]])
    qc = np.clip(q, lo, hi)
    assert np.allclose(O.voxel_value(src, q), f(qc[:, 0], qc[:, 1], qc[:, 2]), atol=1e-6)


def test_voxel_plane_gives_coplanar_points():
    """A linear volume's iso-surface is a plane: every 1D point lies on it to
    the bisection bound and every 3D point on it within the search error."""
    from oracle import odc as oracle
    from paper_2409_13418_gb300 import inputs as I
    n = np.array([0.31, -0.62, 0.72])
    n /= np.linalg.norm(n)
    dims = (9, 9, 9)
    xs = np.linspace(-1, 1, 9)
    zz, yy, xx = np.meshgrid(xs, xs, xs, indexing="ij")
    src = I.VoxelSource(values=(0.5 + 0.4 * (n[0] * xx + n[1] * yy + n[2] * zz - 0.05)).astype(np.float32))
    k = 14
    g = I.cube_grid(16)
    r = oracle.extract(src, g, steps_1d=k)
    h = 2.0 / 16
    d = r.vertices @ n - 0.05
    assert np.max(np.abs(d)) < 2e-3 * h
