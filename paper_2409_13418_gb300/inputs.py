"""Seeded synthetic inputs for occupancy-based dual contouring (ODC).

This module only *draws* problem instances; it holds none of the method's
arithmetic.  Both the CUDA path and the FP64 oracle consume exactly the
arrays produced here, so every value that defines an instance is rounded to
FP32 once, here, and both sides widen the same FP32 numbers.

Instances:

* ``config1_csg()``: union of a sphere (r = 0.55 at (0.1, 0, 0)) and an
  axis-aligned box (half size 0.35 at (-0.3, 0.2, 0)).
* ``random_csg(seed, n_prims=64)``: a left-deep union/difference chain of
  spheres, axis-aligned boxes, rotated boxes, capped cylinders and tori with
  bounding radius U[0.05, 0.3] and centres U[-0.7, 0.7]^3, drawn with
  SplitMix64.
* ``envelope_mlp(seed)``: occ(x) = sigmoid(20 (0.5 - |x| + 0.15 f(x))) with
  f a Kaiming-initialised 128 -> 4 x 256 ReLU -> 1 MLP over 64 random Fourier
  frequencies (sigma = 4).

* ``voxel_random(seed, dims)`` / ``voxel_blobs(seed, dims)``: dense sample
  volumes (vertex-centred samples over a box) whose trilinear interpolation
  is the occupancy; random values stress the topology, smoothed blobs model
  user-provided volumes.

The occupancy function phi of the paper (Sec. 3) is any map R^3 -> {0, 1};
CSG and MLP sources stand in for the paper's neural occupancies (Sec. 6,
A.2.2), which need trained weights that are not available.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Primitive type codes shared by the C ABI (include/odc.h) and the oracle.
PRIM_SPHERE = 0
PRIM_AABB = 1
PRIM_OBOX = 2
PRIM_CYLINDER = 3
PRIM_TORUS = 4
PRIM_NAMES = {PRIM_SPHERE: "sphere", PRIM_AABB: "aabb", PRIM_OBOX: "obox",
              PRIM_CYLINDER: "cylinder", PRIM_TORUS: "torus"}

OP_UNION = 0
OP_DIFFERENCE = 1

# Record layout of one primitive (``odc_csg_prim`` in include/odc.h): 20 float32
# words = [type, op, centre (3), rot (3x3 row-major, 9), params (4), pad (2)].
PRIM_WORDS = 20


@dataclass
class CSGSource:
    """A CSG occupancy instance; every array is float32 / int32."""
    types: np.ndarray          # (P,) int32
    ops: np.ndarray            # (P,) int32, ops[0] == OP_UNION
    centers: np.ndarray        # (P, 3) float32
    rot: np.ndarray            # (P, 3, 3) float32, rows = local axes (identity if unused)
    params: np.ndarray         # (P, 4) float32, meaning per type (see ``prim_params_doc``)
    name: str = "csg"

    @property
    def n_prims(self) -> int:
        return int(self.types.shape[0])

    def packed(self) -> np.ndarray:
        """Pack into the (P, 20) float32 record layout of ``odc_csg_prim``."""
        P = self.n_prims
        rec = np.zeros((P, PRIM_WORDS), np.float32)
        rec[:, 0] = self.types.astype(np.float32)
        rec[:, 1] = self.ops.astype(np.float32)
        rec[:, 2:5] = self.centers
        rec[:, 5:14] = self.rot.reshape(P, 9)
        rec[:, 14:18] = self.params
        return rec


prim_params_doc = """
params per type (all lengths in world units):
  sphere:   [r, 0, 0, 0]
  aabb:     [ex, ey, ez, 0]     half extents along x, y, z (rot = identity)
  obox:     [ex, ey, ez, 0]     half extents along the rows of rot
  cylinder: [r, hh, 0, 0]       radius, half height; axis = rot[2]
  torus:    [R, r, 0, 0]        major, minor radius; axis = rot[2]
"""


class SplitMix64:
    """SplitMix64 (Steele, Lea, Flood 2014) as a plain Python generator."""

    MASK = (1 << 64) - 1

    def __init__(self, seed: int):
        self.state = seed & self.MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & self.MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & self.MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & self.MASK
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / (1 << 53)))


def _quat_to_rows(q):
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
    ], dtype=np.float64)


def _uniform_quat(rng: SplitMix64):
    # Shoemake's uniform random rotation from three uniforms.
    u1, u2, u3 = rng.uniform(), rng.uniform(), rng.uniform()
    a, b = math.sqrt(1 - u1), math.sqrt(u1)
    return (b * math.cos(2 * math.pi * u3), a * math.sin(2 * math.pi * u2),
            a * math.cos(2 * math.pi * u2), b * math.sin(2 * math.pi * u3))


def _frame_from_axis(axis):
    """Rows (u, v, axis) of an orthonormal frame whose third row is ``axis``."""
    a = np.asarray(axis, np.float64)
    a = a / np.linalg.norm(a)
    t = np.array([1.0, 0.0, 0.0]) if abs(a[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    u = np.cross(a, t)
    u /= np.linalg.norm(u)
    v = np.cross(a, u)
    return np.stack([u, v, a])


def _unit_vector(rng: SplitMix64):
    z = rng.uniform(-1.0, 1.0)
    phi = rng.uniform(0.0, 2 * math.pi)
    s = math.sqrt(max(0.0, 1 - z * z))
    return (s * math.cos(phi), s * math.sin(phi), z)


def _make(types, ops, centers, rot, params, name):
    return CSGSource(types=np.asarray(types, np.int32),
                     ops=np.asarray(ops, np.int32),
                     centers=np.asarray(centers, np.float64).astype(np.float32),
                     rot=np.asarray(rot, np.float64).astype(np.float32),
                     params=np.asarray(params, np.float64).astype(np.float32),
                     name=name)


def config1_csg() -> CSGSource:
    """Union of sphere (r=0.55 at (0.1,0,0)) and box (half 0.35 at (-0.3,0.2,0))."""
    eye = np.eye(3)
    return _make([PRIM_SPHERE, PRIM_AABB], [OP_UNION, OP_UNION],
                 [[0.1, 0.0, 0.0], [-0.3, 0.2, 0.0]], [eye, eye],
                 [[0.55, 0, 0, 0], [0.35, 0.35, 0.35, 0]], "sphere_box")


def single_prim(ptype: int, center, rot=None, params=(0, 0, 0, 0), name=None) -> CSGSource:
    rot = np.eye(3) if rot is None else rot
    return _make([ptype], [OP_UNION], [center], [rot], [list(params) + [0] * (4 - len(params))],
                 name or PRIM_NAMES[ptype])


def csg_from_list(prims, name="csg") -> CSGSource:
    """``prims``: list of (type, op, center, rot or None, params)."""
    types, ops, centers, rots, params = [], [], [], [], []
    for (t, op, c, r, p) in prims:
        types.append(t)
        ops.append(op)
        centers.append(c)
        rots.append(np.eye(3) if r is None else r)
        params.append(list(p) + [0] * (4 - len(p)))
    ops[0] = OP_UNION
    return _make(types, ops, centers, rots, params, name)


def random_csg(seed: int, n_prims: int = 64, size_range=(0.05, 0.3),
               center_range=(-0.7, 0.7)) -> CSGSource:
    """Seeded CSG chain; ``size`` is each primitive's bounding radius."""
    rng = SplitMix64(seed)
    types, ops, centers, rots, params = [], [], [], [], []
    for i in range(n_prims):
        t = int(rng.next_u64() % 5)
        s = rng.uniform(*size_range)
        c = [rng.uniform(*center_range) for _ in range(3)]
        op = OP_UNION if i == 0 else (OP_UNION if (rng.next_u64() >> 63) == 0 else OP_DIFFERENCE)
        rot = np.eye(3)
        p = [0.0, 0.0, 0.0, 0.0]
        if t == PRIM_SPHERE:
            p[0] = s
        elif t in (PRIM_AABB, PRIM_OBOX):
            w = np.array([rng.uniform(0.4, 1.0) for _ in range(3)])
            e = s * w / np.linalg.norm(w)
            p[:3] = list(e)
            if t == PRIM_OBOX:
                rot = _quat_to_rows(_uniform_quat(rng))
        elif t == PRIM_CYLINDER:
            th = rng.uniform(0.35, 1.2)
            p[0], p[1] = s * math.cos(th), s * math.sin(th)
            rot = _frame_from_axis(_unit_vector(rng))
        else:
            r = s * rng.uniform(0.15, 0.45)
            p[0], p[1] = s - r, r
            rot = _frame_from_axis(_unit_vector(rng))
        types.append(t)
        ops.append(op)
        centers.append(c)
        rots.append(rot)
        params.append(p)
    return _make(types, ops, centers, rots, params, f"csg_seed{seed}")


@dataclass
class MLPSource:
    """Envelope MLP occupancy: occ(x) = sigmoid(scale (radius - |x| + amp f(x))).

    f(x) = W5 relu(W4 relu(W3 relu(W2 relu(W1 g(x) + b1) + b2) + b3) + b4) + b5
    with Fourier features g(x) = [sin(2 pi B x), cos(2 pi B x)].
    ``latent`` (optional) is concatenated in front of g(x).
    """
    B: np.ndarray               # (F, 3) float32
    weights: list               # [W1 (H, D_in), W2..W4 (H, H), W5 (1, H)] float32
    biases: list                # [b1..b4 (H,), b5 (1,)] float32
    env_scale: float = 20.0
    env_radius: float = 0.5
    env_amp: float = 0.15
    latent: np.ndarray | None = None   # (L,) float32
    name: str = "mlp"

    @property
    def n_freq(self) -> int:
        return int(self.B.shape[0])

    @property
    def hidden(self) -> int:
        return int(self.weights[0].shape[0])

    @property
    def in_dim(self) -> int:
        return int(self.weights[0].shape[1])

    def flops_per_query(self) -> int:
        """Multiply-add FLOPs of the dense layers (2 per MAC)."""
        return int(sum(2 * w.shape[0] * w.shape[1] for w in self.weights))


def envelope_mlp(seed: int = 0, n_freq: int = 64, sigma: float = 4.0, hidden: int = 256,
                 n_hidden_layers: int = 4, latent_dim: int = 0) -> MLPSource:
    """Kaiming-normal random MLP over Fourier features (biases zero)."""
    rng = np.random.default_rng(seed)
    B = (rng.standard_normal((n_freq, 3)) * sigma).astype(np.float32)
    d_in = 2 * n_freq + latent_dim
    dims = [d_in] + [hidden] * n_hidden_layers + [1]
    weights, biases = [], []
    for i in range(len(dims) - 1):
        fan_in = dims[i]
        W = rng.standard_normal((dims[i + 1], fan_in)) * math.sqrt(2.0 / fan_in)
        weights.append(W.astype(np.float32))
        biases.append(np.zeros(dims[i + 1], np.float32))
    latent = None
    if latent_dim:
        latent = rng.standard_normal(latent_dim).astype(np.float32)
    return MLPSource(B=B, weights=weights, biases=biases, latent=latent,
                     name=f"mlp_seed{seed}")


@dataclass
class VoxelSource:
    """Dense sample volume: values[k, j, i] (float32) sit at lo + (hi - lo) *
    (i, j, k) / (dims - 1); the occupancy is their trilinear interpolation
    (clamped to the box) against iso."""
    values: np.ndarray          # (nz, ny, nx) float32
    lo: tuple = (-1.0, -1.0, -1.0)
    hi: tuple = (1.0, 1.0, 1.0)
    name: str = "voxels"

    @property
    def dims(self):
        nz, ny, nx = self.values.shape
        return (nx, ny, nz)


def voxel_random(seed: int, dims=(17, 17, 17), lo=(-1.0, -1.0, -1.0), hi=(1.0, 1.0, 1.0),
                 shell_out: bool = True) -> VoxelSource:
    """Independent U[0, 1) samples (a random-sign stress volume); with
    ``shell_out`` the outer layer of samples is 0 so surfaces close inside."""
    rng = np.random.default_rng(seed)
    v = rng.random((dims[2], dims[1], dims[0])).astype(np.float32)
    if shell_out:
        v[0], v[-1], v[:, 0], v[:, -1], v[:, :, 0], v[:, :, -1] = 0, 0, 0, 0, 0, 0
    return VoxelSource(values=v, lo=tuple(float(np.float32(x)) for x in lo),
                       hi=tuple(float(np.float32(x)) for x in hi), name=f"voxel_random{seed}")


def voxel_blobs(seed: int, dims=(65, 65, 65), n_blobs: int = 12) -> VoxelSource:
    """Sum of Gaussian bumps sampled on the volume's vertices (a smooth
    user-style volume); iso 0.5 cuts a few merged blobs."""
    rng = np.random.default_rng(seed)
    x = [np.linspace(-1.0, 1.0, d) for d in dims]
    zz, yy, xx = np.meshgrid(x[2], x[1], x[0], indexing="ij")
    v = np.zeros(zz.shape)
    for _ in range(n_blobs):
        c = rng.uniform(-0.55, 0.55, 3)
        r = rng.uniform(0.15, 0.35)
        v += np.exp(-((xx - c[0]) ** 2 + (yy - c[1]) ** 2 + (zz - c[2]) ** 2) / (2 * r * r))
    return VoxelSource(values=(0.8 * v / v.max()).astype(np.float32), name=f"voxel_blobs{seed}")


def with_latent(src: MLPSource, seed: int) -> MLPSource:
    """The same network with a fresh latent ~ N(0, I) (latent-conditioned shapes)."""
    if src.latent is None:
        raise ValueError("the network takes no latent")
    lat = np.random.default_rng(seed).standard_normal(src.latent.shape[0]).astype(np.float32)
    return MLPSource(B=src.B, weights=src.weights, biases=src.biases, env_scale=src.env_scale,
                     env_radius=src.env_radius, env_amp=src.env_amp, latent=lat, name=f"{src.name}_lat{seed}")


def serving_trace(seed: int, rate: float, duration: float, res_choices=(64, 128, 256, 512),
                  res_weights=(0.4, 0.3, 0.2, 0.1)):
    """Poisson arrivals at ``rate`` per second over ``duration`` seconds; each
    request draws a cube resolution from ``res_choices`` with ``res_weights``
    and a latent seed.  Returns a list of (arrival time s, resolution, latent seed)."""
    rng = np.random.default_rng(seed)
    out, t = [], 0.0
    p = np.asarray(res_weights, np.float64)
    p = p / p.sum()
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            return out
        res = int(rng.choice(np.asarray(res_choices), p=p))
        out.append((t, res, int(rng.integers(1, 2 ** 31))))


@dataclass
class Grid:
    lo: tuple = (-1.0, -1.0, -1.0)
    hi: tuple = (1.0, 1.0, 1.0)
    res: tuple = (32, 32, 32)

    def cells(self) -> int:
        return int(self.res[0]) * int(self.res[1]) * int(self.res[2])


@dataclass
class Params:
    """Search parameters (paper Sec. 5.1, A.1.4); defaults are the paper's."""
    iso: float = 0.5
    steps_1d: int = 15
    s2d_lin1: int = 4
    s2d_bin1: int = 11
    s2d_range1: float = 0.8
    s2d_lin2: int = 3
    s2d_bin2: int = 12
    s2d_range2: float = float(np.float32(math.sqrt(2.0) / 2.0))
    ic_split: int = 1


def cube_grid(n: int, lo: float = -1.0, hi: float = 1.0) -> Grid:
    return Grid((lo, lo, lo), (hi, hi, hi), (n, n, n))


CONFIGS = {
    "config1": dict(desc="32^3 sphere+box union, k=10", res=32, steps_1d=10),
    "config2": dict(desc="128^3 64-prim CSG, k=12", res=128, steps_1d=12),
    "config3": dict(desc="256^3 envelope MLP, k=15", res=256, steps_1d=15),
}
