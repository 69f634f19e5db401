"""Mesh quality measures of the paper's evaluation (Sec. 6.1 "Evaluation
Metrics"), written plainly in FP64 (test infrastructure only).

* |phi - 0.5|: the occupancy of the shape's own function at points sampled
  uniformly (by area) on the output mesh, averaged; Sec. 6.1 samples 2M
  points per shape.  Here phi is the continuous occupancy sigmoid(z) of an
  MLP source and the deviation is |phi - iso|.  The samples come from a
  counter-based SplitMix64 stream (Steele, Lea and Flood, "Fast splittable
  pseudorandom number generators", OOPSLA 2014): value i is
  mix(seed + (i + 1) * 0x9E3779B97F4A7C15) with mix the published finaliser;
  sample j uses values 3j, 3j + 1, 3j + 2 as u0 (triangle, by the area CDF),
  u1, u2 (barycentric coordinates (1 - sqrt u1, sqrt u1 (1 - u2), sqrt u1 u2)).
* Self-intersection (SI): whether a mesh has intersecting triangle pairs.  A
  pair counts when the triangles share no vertex and their closed point sets
  meet, or share exactly one vertex and the edge of either triangle opposite
  that vertex meets the other triangle.  Triangles sharing an edge are
  never counted.  (The paper reports the share of meshes with any
  self-intersection; this module counts the pairs.)
* Manifoldness: oracle.meshcheck.check_closed_manifold.
"""
from __future__ import annotations

import numpy as np

from . import occupancy

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, idx: np.ndarray) -> np.ndarray:
    """Counter-based SplitMix64: value idx of the stream started at ``seed``."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (np.asarray(idx, np.uint64) + np.uint64(1)) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniforms(seed: int, n: int) -> np.ndarray:
    """(n, 3) doubles in [0, 1): (value >> 11) * 2^-53 of values 3j .. 3j + 2."""
    r = splitmix64(seed, np.arange(3 * n, dtype=np.uint64))
    return ((r >> np.uint64(11)).astype(np.float64) * 2.0 ** -53).reshape(n, 3)


def triangle_areas(verts: np.ndarray, tris: np.ndarray) -> np.ndarray:
    v = np.asarray(verts, np.float64)
    t = np.asarray(tris, np.int64).reshape(-1, 3)
    e1 = v[t[:, 1]] - v[t[:, 0]]
    e2 = v[t[:, 2]] - v[t[:, 0]]
    c = np.cross(e1, e2)
    return 0.5 * np.sqrt(np.einsum("ij,ij->i", c, c))


def surface_samples(verts: np.ndarray, tris: np.ndarray, n: int, seed: int) -> np.ndarray:
    """n points uniform by area on the mesh, rounded to float32."""
    v = np.asarray(verts, np.float64)
    t = np.asarray(tris, np.int64).reshape(-1, 3)
    cdf = np.cumsum(triangle_areas(v, t))
    u = uniforms(seed, n)
    k = np.minimum(np.searchsorted(cdf, u[:, 0] * cdf[-1], side="right"), t.shape[0] - 1)
    s = np.sqrt(u[:, 1])
    b0, b1, b2 = 1.0 - s, s * (1.0 - u[:, 2]), s * u[:, 2]
    p = (b0[:, None] * v[t[k, 0]] + b1[:, None] * v[t[k, 1]]) + b2[:, None] * v[t[k, 2]]
    return p.astype(np.float32)


def occupancy_deviation(mlp, verts, tris, n: int, seed: int, iso: float = 0.5) -> tuple[float, float]:
    """(mean, max) of |sigmoid(z(p)) - iso| over n area-uniform mesh samples (FP64 network)."""
    p = surface_samples(verts, tris, n, seed)
    z = occupancy.mlp_logit(mlp, p.astype(np.float64))
    d = np.abs(1.0 / (1.0 + np.exp(-z)) - iso)
    return float(d.mean()), float(d.max())


def voxel_deviation(src, verts, tris, n: int, seed: int, iso: float = 0.5) -> tuple[float, float]:
    """(mean, max) of |phi(p) - iso| for a voxel source (trilinear, FP64) at n
    area-uniform mesh samples."""
    p = surface_samples(verts, tris, n, seed)
    d = np.abs(occupancy.voxel_value(src, p) - iso)
    return float(d.mean()), float(d.max())


def implicit_psi(src, points: np.ndarray) -> np.ndarray:
    """psi of a CSG source in FP64 (the min/max fold of the primitives' g) at
    FP32-rounded points."""
    x = occupancy.to_query(points)
    psi, _ = occupancy.prim_g(src, 0, x)
    for i in range(1, src.n_prims):
        g, _ = occupancy.prim_g(src, i, x)
        psi = np.minimum(psi, g) if int(src.ops[i]) == 0 else np.maximum(psi, -g)
    return psi


def surface_distance(src, verts, tris, n: int, seed: int) -> tuple[float, float]:
    """(mean, max) of the first-order distance |psi| / |grad psi| of a CSG
    source's surface at n area-uniform mesh samples (the binary occupancy of a
    CSG source has no |phi - 0.5| to measure, so its fidelity is measured as
    a distance)."""
    p = surface_samples(verts, tris, n, seed)
    psi = implicit_psi(src, p)
    gn = np.linalg.norm(occupancy.csg_grad(src, p), axis=1)
    with np.errstate(divide="ignore", invalid="ignore"):
        d = np.where(gn > 0, np.abs(psi) / gn, np.abs(psi))
    return float(d.mean()), float(d.max())


# ---------------------------------------------------------------- SI
def _orient(a, b, c, d):
    """det[b - a, c - a, d - a] (signed six-fold tetrahedron volume), rows of points."""
    u, v, w = b - a, c - a, d - a
    return (u[:, 0] * (v[:, 1] * w[:, 2] - v[:, 2] * w[:, 1])
            + u[:, 1] * (v[:, 2] * w[:, 0] - v[:, 0] * w[:, 2])
            + u[:, 2] * (v[:, 0] * w[:, 1] - v[:, 1] * w[:, 0]))


def _orient2(a, b, c):
    return (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0])


def _seg_seg2(p, q, a, b):
    """Closed 2D segments pq and ab meet (orientation tests with collinear overlap)."""
    d1, d2 = _orient2(a, b, p), _orient2(a, b, q)
    d3, d4 = _orient2(p, q, a), _orient2(p, q, b)
    proper = (((d1 > 0) & (d2 < 0)) | ((d1 < 0) & (d2 > 0))) & (((d3 > 0) & (d4 < 0)) | ((d3 < 0) & (d4 > 0)))

    def on(s0, s1, r, d):
        return (d == 0) & (np.minimum(s0[:, 0], s1[:, 0]) <= r[:, 0]) & (r[:, 0] <= np.maximum(s0[:, 0], s1[:, 0])) \
            & (np.minimum(s0[:, 1], s1[:, 1]) <= r[:, 1]) & (r[:, 1] <= np.maximum(s0[:, 1], s1[:, 1]))
    return proper | on(a, b, p, d1) | on(a, b, q, d2) | on(p, q, a, d3) | on(p, q, b, d4)


def _in_tri2(p, a, b, c):
    s1, s2, s3 = _orient2(a, b, p), _orient2(b, c, p), _orient2(c, a, p)
    return ((s1 >= 0) & (s2 >= 0) & (s3 >= 0)) | ((s1 <= 0) & (s2 <= 0) & (s3 <= 0))


def segment_meets_triangle(p, q, a, b, c) -> np.ndarray:
    """Closed segment pq meets closed triangle abc (rows of points, FP64)."""
    d0, d1 = _orient(a, b, c, p), _orient(a, b, c, q)
    out = np.zeros(p.shape[0], bool)
    cop = (d0 == 0) & (d1 == 0)
    cross = ~cop & ~(((d0 > 0) & (d1 > 0)) | ((d0 < 0) & (d1 < 0)))
    if np.any(cross):
        i = np.nonzero(cross)[0]
        s1 = _orient(p[i], q[i], a[i], b[i])
        s2 = _orient(p[i], q[i], b[i], c[i])
        s3 = _orient(p[i], q[i], c[i], a[i])
        out[i] = ((s1 >= 0) & (s2 >= 0) & (s3 >= 0)) | ((s1 <= 0) & (s2 <= 0) & (s3 <= 0))
    if np.any(cop):
        i = np.nonzero(cop)[0]
        nrm = np.abs(np.cross(b[i] - a[i], c[i] - a[i]))
        ax = np.argmax(nrm, axis=1)             # drop the dominant axis
        keep = np.array([[1, 2], [0, 2], [0, 1]])[ax]
        r = np.arange(i.shape[0])[:, None]

        def pr(x):
            return x[i][r, keep]
        P, Q, A, B, Cc = pr(p), pr(q), pr(a), pr(b), pr(c)
        hit = _in_tri2(P, A, B, Cc) | _in_tri2(Q, A, B, Cc) | _seg_seg2(P, Q, A, B) | _seg_seg2(P, Q, B, Cc) \
            | _seg_seg2(P, Q, Cc, A)
        out[i] = hit
    return out


def self_intersections(verts: np.ndarray, tris: np.ndarray) -> tuple[int, np.ndarray]:
    """Intersecting triangle pairs under the module's definition: (count,
    per-triangle flag).  All pairs with overlapping bounding boxes are tested."""
    v = np.asarray(verts, np.float64)
    t = np.asarray(tris, np.int64).reshape(-1, 3)
    T = t.shape[0]
    P = v[t]                                   # (T, 3, 3)
    lo, hi = P.min(axis=1), P.max(axis=1)
    I, J = [], []
    for i in range(T - 1):
        j = np.arange(i + 1, T)
        ok = np.all(lo[j] <= hi[i], axis=1) & np.all(lo[i] <= hi[j], axis=1)
        j = j[ok]
        I.append(np.full(j.shape[0], i))
        J.append(j)
    if not I:
        return 0, np.zeros(T, bool)
    I, J = np.concatenate(I), np.concatenate(J)
    ti, tj = t[I], t[J]
    shared = (ti[:, :, None] == tj[:, None, :])          # (n, 3, 3)
    ns = shared.sum(axis=(1, 2))
    hit = np.zeros(I.shape[0], bool)
    # no shared vertex: any of the six edge-vs-triangle tests
    k = np.nonzero(ns == 0)[0]
    if k.size:
        Ai, Aj = P[I[k]], P[J[k]]
        h = np.zeros(k.size, bool)
        for e in range(3):
            h |= segment_meets_triangle(Ai[:, e], Ai[:, (e + 1) % 3], Aj[:, 0], Aj[:, 1], Aj[:, 2])
            h |= segment_meets_triangle(Aj[:, e], Aj[:, (e + 1) % 3], Ai[:, 0], Ai[:, 1], Ai[:, 2])
        hit[k] = h
    # one shared vertex: the edge opposite it, of either triangle, against the other
    k = np.nonzero(ns == 1)[0]
    if k.size:
        si = np.argmax(shared[k].any(axis=2), axis=1)     # position of the shared vertex in ti
        sj = np.argmax(shared[k].any(axis=1), axis=1)     # ... and in tj
        Ai, Aj = P[I[k]], P[J[k]]
        r = np.arange(k.size)
        oi0, oi1 = Ai[r, (si + 1) % 3], Ai[r, (si + 2) % 3]
        oj0, oj1 = Aj[r, (sj + 1) % 3], Aj[r, (sj + 2) % 3]
        h = segment_meets_triangle(oi0, oi1, Aj[:, 0], Aj[:, 1], Aj[:, 2])
        h |= segment_meets_triangle(oj0, oj1, Ai[:, 0], Ai[:, 1], Ai[:, 2])
        hit[k] = h
    flag = np.zeros(T, bool)
    flag[I[hit]] = True
    flag[J[hit]] = True
    return int(hit.sum()), flag
