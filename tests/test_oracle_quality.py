"""Pins of the oracle's mesh-quality measures (Sec. 6.1 metrics): the
SplitMix64 stream against its published first outputs, area-uniform sampling
against areas and centroids, the occupancy deviation against closed-form
bounds on a sphere, and the self-intersection count on hand-built cases."""
import math

import numpy as np

from oracle import meshcheck, quality as Q
from oracle import odc as oracle
from paper_2409_13418_gb300 import inputs as I


def test_splitmix64_first_outputs_of_seed_zero():
    # the generator's published reference sequence for state 0
    r = Q.splitmix64(0, np.arange(3))
    assert [int(x) for x in r] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    u = Q.uniforms(7, 100000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.003 and abs(u.var() - 1 / 12) < 0.002


def test_samples_are_uniform_by_area():
    # a 3 x 1 rectangle split into triangles of areas 1.5 and 1.5, plus a unit
    # right triangle elsewhere (area 0.5): fractions 3/7, 3/7, 1/7
    v = np.array([[0, 0, 0], [3, 0, 0], [3, 1, 0], [0, 1, 0], [10, 0, 0], [11, 0, 0], [10, 1, 0]], np.float32)
    t = np.array([[0, 1, 2], [0, 2, 3], [4, 5, 6]])
    n = 200000
    p = Q.surface_samples(v, t, n, seed=3).astype(np.float64)
    far = p[:, 0] >= 9.5
    assert abs(far.mean() - 1 / 7) < 0.004
    rect = p[~far]
    assert abs(rect[:, 0].mean() - 1.5) < 0.01 and abs(rect[:, 1].mean() - 0.5) < 0.005
    # in the unit triangle: centroid (10 + 1/3, 1/3) and 1/4 of the mass in the
    # half-scale corner triangle at (10, 0)
    tri = p[far] - np.array([10.0, 0.0, 0.0])
    assert abs(tri[:, 0].mean() - 1 / 3) < 0.005 and abs(tri[:, 1].mean() - 1 / 3) < 0.005
    corner = (tri[:, 0] + tri[:, 1]) <= 0.5
    assert abs(corner.mean() - 0.25) < 0.01


def _icosphere(r, level):
    t = (1 + 5 ** 0.5) / 2
    v = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
         (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    f = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6),
         (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10),
         (8, 6, 7), (9, 8, 1)]
    v = [np.array(x, float) / np.linalg.norm(x) for x in v]
    for _ in range(level):
        mid, nf = {}, []
        for a, b, c in f:
            m = []
            for i, j in ((a, b), (b, c), (c, a)):
                k = (min(i, j), max(i, j))
                if k not in mid:
                    x = v[i] + v[j]
                    v.append(x / np.linalg.norm(x))
                    mid[k] = len(v) - 1
                m.append(mid[k])
            nf += [(a, m[0], m[2]), (b, m[1], m[0]), (c, m[2], m[1]), (m[0], m[1], m[2])]
        f = nf
    return (np.array(v) * r).astype(np.float32), np.array(f)


def test_occupancy_deviation_on_a_sphere_lies_within_closed_form_bounds():
    # amp = 0: occ(x) = sigmoid(20 (0.5 - |x|)); a sphere mesh of radius 0.6
    # has every surface point at |x| in [r_in, 0.6], r_in its inradius; the
    # deviation 1/2 - sigmoid(20 (0.5 - |x|)) grows with |x| beyond 0.5, so it
    # lies in [1/2 - sigmoid(-20 (r_in - 0.5)), 1/2 - sigmoid(-20 (0.6 - 0.5))]
    mlp = I.envelope_mlp(0)
    mlp.env_amp = 0.0
    v, t = _icosphere(0.6, 3)
    vv = v.astype(np.float64)
    n = np.cross(vv[t[:, 1]] - vv[t[:, 0]], vv[t[:, 2]] - vv[t[:, 0]])
    r_in = float(np.min(np.abs(np.einsum("ij,ij->i", n / np.linalg.norm(n, axis=1)[:, None], vv[t[:, 0]]))))
    lo = 0.5 - 1 / (1 + math.exp(20 * (r_in - 0.5)))
    hi = 0.5 - 1 / (1 + math.exp(20 * (0.6 - 0.5)))
    mean, mx = Q.occupancy_deviation(mlp, v, t, 20000, seed=1)
    assert lo - 1e-6 <= mean <= hi + 1e-6 and mx <= hi + 1e-6
    assert 0.59 < r_in < 0.6 and abs(hi - 0.3807970779778823) < 1e-12       # 1/2 - 1/(1 + e^2)


def _tri_pair(a, b):
    v = np.array(a + b, np.float32)
    return v, np.array([[0, 1, 2], [3, 4, 5]])


def test_self_intersection_cases():
    # crossing (X), disjoint parallel, coplanar overlap, coplanar disjoint
    v, t = _tri_pair([(0, 0, 0), (2, 0, 0), (0, 2, 0)], [(0.5, 0.5, -1), (0.5, 0.5, 1), (3, 3, 0.5)])
    assert Q.self_intersections(v, t)[0] == 1
    v, t = _tri_pair([(0, 0, 0), (2, 0, 0), (0, 2, 0)], [(0, 0, 1), (2, 0, 1), (0, 2, 1)])
    assert Q.self_intersections(v, t)[0] == 0
    v, t = _tri_pair([(0, 0, 0), (2, 0, 0), (0, 2, 0)], [(0.5, 0.5, 0), (3, 0.5, 0), (0.5, 3, 0)])
    assert Q.self_intersections(v, t)[0] == 1
    v, t = _tri_pair([(0, 0, 0), (1, 0, 0), (0, 1, 0)], [(2, 2, 0), (3, 2, 0), (2, 3, 0)])
    assert Q.self_intersections(v, t)[0] == 0
    # one shared vertex: touching only there (0) / the second folded through the first (1)
    v = np.array([(0, 0, 0), (2, 0, 0), (0, 2, 0), (-1, 0, 1), (0, -1, 1)], np.float32)
    assert Q.self_intersections(v, np.array([[0, 1, 2], [0, 3, 4]]))[0] == 0
    v = np.array([(0, 0, 0), (2, 0, 0), (0, 2, 0), (1, 1, -1), (1, 1, 1)], np.float32)
    assert Q.self_intersections(v, np.array([[0, 1, 2], [0, 3, 4]]))[0] == 1
    # a shared edge never counts, even folded flat onto the other triangle
    v = np.array([(0, 0, 0), (2, 0, 0), (0, 2, 0), (1, 1, 0)], np.float32)
    assert Q.self_intersections(v, np.array([[0, 1, 2], [1, 0, 3]]))[0] == 0
    # a closed convex mesh has none
    v, t = _icosphere(1.0, 2)
    assert Q.self_intersections(v, t)[0] == 0


def _moller_trumbore_hit(o, d, tri):
    """Segment o + s d, s in [0, 1], meets triangle tri (Moller-Trumbore ray
    test with barycentric (u, v) and segment parameter s)."""
    e1, e2 = tri[1] - tri[0], tri[2] - tri[0]
    p = np.cross(d, e2)
    det = e1 @ p
    if det == 0.0:
        return False
    s0 = o - tri[0]
    u = (s0 @ p) / det
    q = np.cross(s0, e1)
    v = (d @ q) / det
    t = (e2 @ q) / det
    return u >= 0 and v >= 0 and u + v <= 1 and 0 <= t <= 1


def _brute_si(v, t):
    """Independent count: every bounding-box-overlapping pair, edges tested by
    Moller-Trumbore (unreliable for nearly coplanar pairs, so used on meshes
    of curved shapes only)."""
    P = v[t]
    lo, hi = P.min(1), P.max(1)
    cnt = 0
    for i in range(len(t) - 1):
        js = np.arange(i + 1, len(t))
        js = js[np.all(lo[js] <= hi[i], 1) & np.all(lo[i] <= hi[js], 1)]
        for j in js:
            sh = set(t[i]) & set(t[j])
            if len(sh) >= 2:
                continue
            if not sh:
                hit = any(_moller_trumbore_hit(P[i][a], P[i][(a + 1) % 3] - P[i][a], P[j]) for a in range(3)) or \
                    any(_moller_trumbore_hit(P[j][a], P[j][(a + 1) % 3] - P[j][a], P[i]) for a in range(3))
            else:
                s = sh.pop()
                ki, kj = list(t[i]).index(s), list(t[j]).index(s)
                hit = _moller_trumbore_hit(P[i][(ki + 1) % 3], P[i][(ki + 2) % 3] - P[i][(ki + 1) % 3], P[j]) or \
                    _moller_trumbore_hit(P[j][(kj + 1) % 3], P[j][(kj + 2) % 3] - P[j][(kj + 1) % 3], P[i])
            cnt += hit
    return cnt


def test_self_intersection_count_matches_an_independent_test_on_odc_meshes():
    """The orientation-predicate counter against Moller-Trumbore on ODC meshes
    of a coarse random MLP and a random CSG tree, with and without IC quad
    splitting (Sec. 5.4); all four meshes are closed manifolds.  Coarse grids
    of bumpy shapes do self-intersect (several 3D points per cell, QEF points
    outside their cells), so the counts are far from zero."""
    for src, n, k in ((I.envelope_mlp(0), 16, 12), (I.random_csg(4, n_prims=12), 20, 10)):
        for ic in (False, True):
            r = oracle.extract(src, I.cube_grid(n), steps_1d=k, ic_split=ic)
            v, t = np.asarray(r.vertices, np.float64), np.asarray(r.triangles)
            assert meshcheck.check_closed_manifold(t)["ok"]
            c, flag = Q.self_intersections(v, t)
            assert c > 0 and c == _brute_si(v, t)
            assert flag.sum() <= 2 * c


def test_csg_gradient_matches_finite_differences_and_psi32_matches_fp64():
    from oracle import occupancy as O
    src = I.random_csg(2, n_prims=64)
    rng = np.random.default_rng(5)
    x = rng.uniform(-0.9, 0.9, (4000, 3)).astype(np.float32).astype(np.float64)
    psi = Q.implicit_psi(src, x)
    g = O.csg_grad(src, x)          # x is FP32-representable: no rounding inside

    def psi64(y):                   # the fold in FP64 at unrounded points
        v, _ = O.prim_g(src, 0, y)
        for i in range(1, src.n_prims):
            gi, _ = O.prim_g(src, i, y)
            v = np.minimum(v, gi) if int(src.ops[i]) == 0 else np.maximum(v, -gi)
        return v
    h = 1e-6
    fd = np.stack([(psi64(x + h * e) - psi64(x - h * e)) / (2 * h) for e in np.eye(3)], axis=1)
    # away from kinks of the min/max fold and of the box and cylinder maxima
    # the central difference sees one smooth branch
    err = np.linalg.norm(fd - g, axis=1) / np.maximum(np.linalg.norm(g, axis=1), 1e-12)
    assert np.mean(err < 1e-4) > 0.97
    # the FP32 value follows the FP64 one to FP32 rounding
    p32 = O.csg_psi32(src, x.astype(np.float32)).astype(np.float64)
    assert np.all(np.abs(p32 - psi) <= 1e-5 * np.maximum(1.0, np.abs(psi)))


def test_surface_distance_on_a_sphere_mesh():
    # unit-radius sphere primitive g = |x|^2 - 1: |g| / |grad g| = |1 - |x|^2| / (2 |x|)
    # lies within the chord sag of an inscribed icosphere: (1 - r_in) (1 + r_in) / (2 r_in)
    src = I.single_prim(I.PRIM_SPHERE, (0.0, 0.0, 0.0), params=(1.0,))
    v, t = _icosphere(1.0, 3)
    vv = v.astype(np.float64)
    n = np.cross(vv[t[:, 1]] - vv[t[:, 0]], vv[t[:, 2]] - vv[t[:, 0]])
    r_in = float(np.min(np.abs(np.einsum("ij,ij->i", n / np.linalg.norm(n, axis=1)[:, None], vv[t[:, 0]]))))
    mean, mx = Q.surface_distance(src, v, t, 20000, seed=2)
    bound = (1 - r_in) * (1 + r_in) / (2 * r_in)
    assert 0 < mean < mx <= bound * (1 + 1e-6) + 1e-6


def test_linear_1d_is_exact_on_box_faces_and_gradient_normals_recover_box_corners():
    """Eq. 1 on an axis-aligned box: psi = max_a(|x_a - c_a| - h_a) is linear
    along an edge crossing a face wherever the edge's own axis attains the
    max at both ends, so there the FP32 linear 1D point sits within 2^-(k+2)
    of an edge (quantisation) plus FP32 rounding from the face.  With
    bisected 1D points and gradient normals (exact face normals) the QEF of a
    corner cell returns the corner; linearly placed points near a corner are
    off (there psi switches branch along the edge), so MDC misses it."""
    c, hs = (0.013, -0.021, 0.008), (0.43, 0.37, 0.41)
    src = I.single_prim(I.PRIM_AABB, c, params=hs)
    g = I.cube_grid(24)
    k = 12
    r = oracle.extract(src, g, steps_1d=k, linear_1d=True, gradient_normals=True)
    h = 2.0 / 24
    e = r.edges
    a = e % 3
    v = e // 3
    nv = 25
    ijk = np.stack([v % nv, (v // nv) % nv, v // (nv * nv)], axis=1)
    X = -1.0 + ijk * h
    pos = X[np.arange(len(e)), a] + h * r.T / 2.0 ** (k + 1)
    faces = np.array(c)[a] + np.where(X[np.arange(len(e)), a] + 0.5 * h > np.array(c)[a], 1, -1) * np.array(hs)[a]
    lin = np.ones(len(e), bool)
    for end in (0.0, 1.0):
        P = X + end * h * np.eye(3)[a]
        terms = np.abs(P - np.array(c)) - np.array(hs)
        lin &= np.argmax(terms, axis=1) == a
    assert lin.sum() > len(e) // 3
    assert np.max(np.abs(pos - faces)[lin]) <= h * 2.0 ** -(k + 2) + 1e-6
    corners = np.array([[c[0] + sx * hs[0], c[1] + sy * hs[1], c[2] + sz * hs[2]]
                        for sx in (-1, 1) for sy in (-1, 1) for sz in (-1, 1)])
    assert meshcheck.check_closed_manifold(r.triangles)["ok"]
    d_lin = np.min(np.linalg.norm(r.vertices[:, None, :] - corners[None], axis=2), axis=0)
    r1 = oracle.extract(src, g, steps_1d=k, gradient_normals=True)
    d = np.min(np.linalg.norm(r1.vertices[:, None, :] - corners[None], axis=2), axis=0)
    assert np.all(d <= h * 2.0 ** -(k + 1) * math.sqrt(3) + 1e-6)
    assert np.max(d_lin) > 10 * np.max(d)
    assert meshcheck.check_closed_manifold(r1.triangles)["ok"]
