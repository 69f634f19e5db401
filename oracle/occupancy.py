"""Occupancy phi(p) in FP64 for the oracle (test infrastructure only).

Paper: an occupancy function phi: R^3 -> {0 (out), 1 (in)} (Sec. 3); neural
occupancies are thresholded at the iso level to give binary labels (A.2.2).

Readings (the paper is silent on these):
  * The query point is rounded to FP32 before phi is evaluated, as every GPU
    occupancy network consumes FP32 coordinates.  Both the oracle and the CUDA
    path evaluate phi at the same FP32 point.
  * Ties are "out": a point is inside only if occ > iso strictly.
  * CSG: inside(prim) iff g_prim < 0.  Union is min, difference A \\ B is
    max(g_A, -g_B); folded left to right in primitive order.  As booleans this
    is ``in = in or in_p`` (union) and ``in = in and (g_p > 0)`` (difference).
  * MLP: the decision is taken on the pre-sigmoid logit, z > logit(iso).

Each evaluation also returns a *margin*: a distance-like measure of how far
the decision is from flipping (world units for CSG, |occ - iso| for MLP).  The
parity tests use it to flag decisions that finite precision could flip.
"""
from __future__ import annotations

import math

import numpy as np

from paper_2409_13418_gb300.inputs import (CSGSource, MLPSource, OP_UNION, PRIM_AABB,
                                           PRIM_CYLINDER, PRIM_OBOX, PRIM_SPHERE, PRIM_TORUS, VoxelSource)


def to_query(points: np.ndarray) -> np.ndarray:
    """Round query points to FP32 and widen back to FP64."""
    return np.asarray(points, np.float64).astype(np.float32).astype(np.float64)


def prim_g(src: CSGSource, i: int, x: np.ndarray):
    """Sign function g and margin of primitive ``i`` at FP64 points ``x`` (n, 3).

    g < 0 inside, g > 0 outside.  Every operand is an FP32 value widened to
    FP64; the operation order below is the definition of g.
    """
    t = int(src.types[i])
    c = src.centers[i].astype(np.float64)
    M = src.rot[i].astype(np.float64)
    p = src.params[i].astype(np.float64)
    dx = x[:, 0] - c[0]
    dy = x[:, 1] - c[1]
    dz = x[:, 2] - c[2]
    if t == PRIM_SPHERE:
        r = p[0]
        g = ((dx * dx + dy * dy) + dz * dz) - r * r
        return g, np.abs(g) / (2.0 * r)
    if t == PRIM_AABB:
        g = np.maximum(np.maximum(np.abs(dx) - p[0], np.abs(dy) - p[1]), np.abs(dz) - p[2])
        # every operation above is exact for float32 operands, so a tie g == 0
        # is decided identically ("out") in any precision: not a fragile decision
        return g, np.where(g == 0.0, np.inf, np.abs(g))
    if t == PRIM_OBOX:
        ls = [((M[k, 0] * dx + M[k, 1] * dy) + M[k, 2] * dz) for k in range(3)]
        g = np.maximum(np.maximum(np.abs(ls[0]) - p[0], np.abs(ls[1]) - p[1]), np.abs(ls[2]) - p[2])
        return g, np.abs(g)
    ax = M[2]
    tt = (ax[0] * dx + ax[1] * dy) + ax[2] * dz
    d2 = (dx * dx + dy * dy) + dz * dz
    if t == PRIM_CYLINDER:
        r, hh = p[0], p[1]
        radial = (d2 - tt * tt) - r * r
        axial = np.abs(tt) - hh
        g_r = radial / (2.0 * r)
        g = np.maximum(g_r, axial)
        return g, np.abs(g)
    if t == PRIM_TORUS:
        R, r = p[0], p[1]
        q = (d2 + R * R) - r * r
        g = q * q - (4.0 * R * R) * (d2 - tt * tt)
        return g, np.abs(g) / (8.0 * R * R * r)
    raise ValueError(f"unknown primitive type {t}")


def csg_eval(src: CSGSource, points: np.ndarray):
    """Labels (bool) and margins of a CSG source at ``points`` (n, 3)."""
    x = to_query(points)
    n = x.shape[0]
    inside = np.zeros(n, bool)
    margin = np.full(n, np.inf)
    for i in range(src.n_prims):
        g, m = prim_g(src, i, x)
        if i == 0 or int(src.ops[i]) == OP_UNION:
            inside = inside | (g < 0)
        else:
            inside = inside & (g > 0)
        margin = np.minimum(margin, m)
    return inside, margin


# ---- ablation variants (Sec. 6.3, Tab. 3): MDC's implicit value and gradient
# The MDC baselines of the ablation need a continuous implicit psi with a
# gradient (Sec. 4, Eqs. 1 and 3).  For a CSG source psi is the min/max fold of
# the primitives' g (union: min(psi, g), difference: max(psi, -g)); its zero
# set is the CSG surface.  Eq. 1 places a 1D point by linear interpolation of
# psi; the value is taken in FP32 with the operation order written below, so
# that the interpolation parameter (an integer after quantisation) is the
# same in any implementation that follows it.

def _prim_g32(src: CSGSource, i: int, x: np.ndarray) -> np.ndarray:
    """g of primitive i in FP32 arithmetic at FP32 points x (n, 3)."""
    f = np.float32
    t = int(src.types[i])
    c = src.centers[i].astype(f)
    M = src.rot[i].astype(f)
    p = src.params[i].astype(f)
    dx, dy, dz = x[:, 0] - c[0], x[:, 1] - c[1], x[:, 2] - c[2]
    if t == PRIM_SPHERE:
        return ((dx * dx + dy * dy) + dz * dz) - p[0] * p[0]
    if t == PRIM_AABB:
        return np.maximum(np.maximum(np.abs(dx) - p[0], np.abs(dy) - p[1]), np.abs(dz) - p[2])
    if t == PRIM_OBOX:
        ls = [((M[k, 0] * dx + M[k, 1] * dy) + M[k, 2] * dz) for k in range(3)]
        return np.maximum(np.maximum(np.abs(ls[0]) - p[0], np.abs(ls[1]) - p[1]), np.abs(ls[2]) - p[2])
    ax = M[2]
    tt = (ax[0] * dx + ax[1] * dy) + ax[2] * dz
    d2 = (dx * dx + dy * dy) + dz * dz
    if t == PRIM_CYLINDER:
        radial = (d2 - tt * tt) - p[0] * p[0]
        return np.maximum(radial / (f(2.0) * p[0]), np.abs(tt) - p[1])
    if t == PRIM_TORUS:
        q = (d2 + p[0] * p[0]) - p[1] * p[1]
        return q * q - ((f(4.0) * p[0]) * p[0]) * (d2 - tt * tt)
    raise ValueError(f"unknown primitive type {t}")


def csg_psi32(src: CSGSource, points: np.ndarray) -> np.ndarray:
    """psi in FP32 at FP32 points (every primitive evaluated, no culling)."""
    x = np.asarray(points, np.float32)
    psi = _prim_g32(src, 0, x)
    for i in range(1, src.n_prims):
        g = _prim_g32(src, i, x)
        psi = np.minimum(psi, g) if int(src.ops[i]) == OP_UNION else np.maximum(psi, -g)
    return psi


def _prim_grad(src: CSGSource, i: int, x: np.ndarray) -> np.ndarray:
    """Gradient of g of primitive i in FP64 (the branch attaining a max; the
    first one on ties; the sign of 0 taken as +)."""
    t = int(src.types[i])
    c = src.centers[i].astype(np.float64)
    M = src.rot[i].astype(np.float64)
    p = src.params[i].astype(np.float64)
    d = x - c
    n = x.shape[0]

    def sgn(v):
        return np.where(v < 0, -1.0, 1.0)
    if t == PRIM_SPHERE:
        return 2.0 * d
    if t in (PRIM_AABB, PRIM_OBOX):
        L = d if t == PRIM_AABB else d @ M.T
        rows = np.eye(3) if t == PRIM_AABB else M
        val = np.abs(L) - p[:3]
        k = np.zeros(n, np.int64)
        k = np.where(val[:, 1] > val[np.arange(n), k], 1, k)
        k = np.where(val[:, 2] > val[np.arange(n), k], 2, k)
        return sgn(L[np.arange(n), k])[:, None] * rows[k]
    ax = M[2]
    tt = d @ ax
    radial_dir = d - tt[:, None] * ax
    if t == PRIM_CYLINDER:
        r, hh = p[0], p[1]
        d2 = np.einsum("ij,ij->i", d, d)
        g_r = ((d2 - tt * tt) - r * r) / (2.0 * r)
        axial = np.abs(tt) - hh
        return np.where((g_r >= axial)[:, None], radial_dir / r, sgn(tt)[:, None] * ax)
    if t == PRIM_TORUS:
        R, r = p[0], p[1]
        d2 = np.einsum("ij,ij->i", d, d)
        q = (d2 + R * R) - r * r
        return 4.0 * q[:, None] * d - 8.0 * R * R * radial_dir
    raise ValueError(f"unknown primitive type {t}")


def csg_grad(src: CSGSource, points: np.ndarray) -> np.ndarray:
    """Gradient of psi in FP64 at FP32-rounded points: the gradient of the
    primitive the min/max fold selects (strict comparisons: the earlier
    operand wins ties), negated for a selected difference operand."""
    x = to_query(points)
    psi, _ = prim_g(src, 0, x)
    grad = _prim_grad(src, 0, x)
    for i in range(1, src.n_prims):
        g, _ = prim_g(src, i, x)
        gr = _prim_grad(src, i, x)
        if int(src.ops[i]) == OP_UNION:
            take = g < psi
            psi = np.where(take, g, psi)
            grad = np.where(take[:, None], gr, grad)
        else:
            take = -g > psi
            psi = np.where(take, -g, psi)
            grad = np.where(take[:, None], -gr, grad)
    return grad


def fourier_features(src: MLPSource, x: np.ndarray) -> np.ndarray:
    """g(x) = [sin(2 pi B x), cos(2 pi B x)] in FP64."""
    B = src.B.astype(np.float64)
    u = x @ B.T
    ang = 2.0 * math.pi * u
    return np.concatenate([np.sin(ang), np.cos(ang)], axis=1)


def mlp_f(src: MLPSource, x: np.ndarray, chunk: int = 32768) -> np.ndarray:
    """The network output f(x) in FP64 (FP32 weights widened)."""
    Ws = [w.astype(np.float64) for w in src.weights]
    bs = [b.astype(np.float64) for b in src.biases]
    out = np.empty(x.shape[0])
    lat = None if src.latent is None else src.latent.astype(np.float64)
    for s in range(0, x.shape[0], chunk):
        xs = x[s:s + chunk]
        h = fourier_features(src, xs)
        if lat is not None:
            h = np.concatenate([np.broadcast_to(lat, (xs.shape[0], lat.shape[0])), h], axis=1)
        for li in range(len(Ws) - 1):
            h = np.maximum(h @ Ws[li].T + bs[li], 0.0)
        out[s:s + chunk] = (h @ Ws[-1].T + bs[-1])[:, 0]
    return out


def mlp_logit(src: MLPSource, points: np.ndarray) -> np.ndarray:
    """z = scale * (radius - |x| + amp * f(x)), the envelope's pre-sigmoid logit."""
    x = to_query(points)
    r = np.sqrt((x[:, 0] * x[:, 0] + x[:, 1] * x[:, 1]) + x[:, 2] * x[:, 2])
    return float(np.float32(src.env_scale)) * (
        (float(np.float32(src.env_radius)) - r) + float(np.float32(src.env_amp)) * mlp_f(src, x))


def mlp_eval(src: MLPSource, points: np.ndarray, iso: float = 0.5):
    """Labels and margins |occ - iso| of an MLP source."""
    z = mlp_logit(src, points)
    t = math.log(iso / (1.0 - iso))
    occ = 1.0 / (1.0 + np.exp(-z))
    return z > t, np.abs(occ - iso)


def voxel_value(src: VoxelSource, points: np.ndarray) -> np.ndarray:
    """Trilinear interpolation of the sample volume at FP32-rounded points
    (FP64): per axis u = (x - lo) / (hi - lo) * (dims - 1) clamped to
    [0, dims - 1], cell i = min(floor(u), dims - 2), fraction u - i; then
    lerps along x, y, z."""
    x = to_query(points)
    v = src.values.astype(np.float64)
    dims = src.dims
    idx, frac = [], []
    for a in range(3):
        lo, hi = float(np.float32(src.lo[a])), float(np.float32(src.hi[a]))
        u = (x[:, a] - lo) / (hi - lo) * (dims[a] - 1)
        u = np.clip(u, 0.0, dims[a] - 1)
        i = np.minimum(np.floor(u).astype(np.int64), dims[a] - 2)
        idx.append(i)
        frac.append(u - i)
    i, j, k = idx
    fx, fy, fz = frac

    def lerp(a, b, f):
        return a + (b - a) * f
    c00 = lerp(v[k, j, i], v[k, j, i + 1], fx)
    c10 = lerp(v[k, j + 1, i], v[k, j + 1, i + 1], fx)
    c01 = lerp(v[k + 1, j, i], v[k + 1, j, i + 1], fx)
    c11 = lerp(v[k + 1, j + 1, i], v[k + 1, j + 1, i + 1], fx)
    return lerp(lerp(c00, c10, fy), lerp(c01, c11, fy), fz)


def voxel_eval(src: VoxelSource, points: np.ndarray, iso: float = 0.5):
    """Labels (value > iso) and margins |value - iso| of a voxel source."""
    phi = voxel_value(src, points)
    return phi > iso, np.abs(phi - iso)


class Occupancy:
    """Callable phi with query accounting: ``labels, margins = phi(points)``."""

    def __init__(self, src, iso: float = 0.5):
        self.src = src
        self.iso = float(np.float32(iso))   # iso is an FP32 parameter of the instance, like every other
        self.queries = 0

    def __call__(self, points: np.ndarray):
        points = np.asarray(points, np.float64).reshape(-1, 3)
        self.queries += points.shape[0]
        if points.shape[0] == 0:
            return np.zeros(0, bool), np.zeros(0)
        if isinstance(self.src, CSGSource):
            return csg_eval(self.src, points)
        if isinstance(self.src, MLPSource):
            return mlp_eval(self.src, points, self.iso)
        if isinstance(self.src, VoxelSource):
            return voxel_eval(self.src, points, self.iso)
        if callable(self.src):
            return self.src(to_query(points))
        raise TypeError(type(self.src))
