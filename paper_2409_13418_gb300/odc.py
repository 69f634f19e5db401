"""Thin ctypes binding of the ODC C ABI (include/odc.h).

Argument marshalling only: every step of the path runs in the CUDA library.
The library is loaded from this package directory; if it is missing this
module raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libodc.so")

ODC_OK = 0
STATUS = {0: "ok", 1: "invalid argument", 2: "out of memory", 3: "CUDA error", 4: "timeout",
          5: "unsupported", 6: "internal error"}
SRC_CSG, SRC_MLP, SRC_RESIDENT, SRC_VOXEL = 0, 1, 2, 3
PREC_FP32, PREC_BF16, PREC_SPLIT, PREC_F16, PREC_FP8, PREC_FP8_RAW = 0, 1, 2, 3, 4, 5
MLP_REUPLOAD, MLP_NO_F16_TIER = 1, 2
DBG = dict(labels=0, edges=1, T=2, faces=3, slots=4, face_pts=5, face_flags=6, cells=7, configs=8,
           cycles=9, vlocal=10, qcase=11, flips=12, search=13)
_DBG_DTYPE = dict(labels=np.uint32, edges=np.uint32, T=np.uint32, faces=np.uint32, slots=np.uint8,
                  face_pts=np.float32, face_flags=np.uint8, cells=np.uint32, configs=np.uint8,
                  cycles=np.uint64, vlocal=np.float32, qcase=np.uint8, flips=np.uint32, search=np.uint32)
_DBG_SHAPE = dict(face_pts=4, vlocal=3, search=4)


class Prim(C.Structure):
    _fields_ = [("type", C.c_int32), ("op", C.c_int32), ("center", C.c_float * 3), ("rot", C.c_float * 9),
                ("params", C.c_float * 4), ("pad", C.c_float * 2)]


class Mlp(C.Structure):
    _fields_ = [("n_freq", C.c_int32), ("hidden", C.c_int32), ("n_hidden", C.c_int32), ("latent_dim", C.c_int32),
                ("B", C.c_void_p), ("W", C.c_void_p * 8), ("b", C.c_void_p * 8), ("latent", C.c_void_p),
                ("env_scale", C.c_float), ("env_radius", C.c_float), ("env_amp", C.c_float),
                ("precision", C.c_int32), ("band", C.c_float), ("no_split", C.c_int32),
                ("split_zmargin", C.c_float), ("flags", C.c_int32), ("h16_zmargin", C.c_float),
                ("split_acc_comp", C.c_float)]


class Voxels(C.Structure):
    _fields_ = [("dims", C.c_int32 * 3), ("lo", C.c_float * 3), ("hi", C.c_float * 3), ("values", C.c_void_p)]


class Source(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n_prims", C.c_int32), ("prims", C.c_void_p), ("mlp", C.c_void_p),
                ("voxels", C.c_void_p)]


class Grid(C.Structure):
    _fields_ = [("lo", C.c_float * 3), ("hi", C.c_float * 3), ("res", C.c_int32 * 3)]


class Params(C.Structure):
    _fields_ = [("iso", C.c_float), ("steps_1d", C.c_int32), ("s2d_lin1", C.c_int32), ("s2d_bin1", C.c_int32),
                ("s2d_range1", C.c_float), ("s2d_lin2", C.c_int32), ("s2d_bin2", C.c_int32),
                ("s2d_range2", C.c_float), ("ic_split", C.c_int32), ("flags", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("n_edges", C.c_int64), ("n_face_segs", C.c_int64), ("n_cells", C.c_int64),
                ("n_verts3", C.c_int64), ("n_case3", C.c_int64), ("n_flips", C.c_int64),
                ("fix_rounds", C.c_int64), ("n_queries", C.c_int64), ("n_requeries", C.c_int64),
                ("stage_ms", C.c_float * 8), ("mlp_flops", C.c_double), ("mlp_ms", C.c_float),
                ("n_launches", C.c_int32), ("mlp_launches", C.c_int64), ("tc_flops", C.c_double),
                ("tc_ms", C.c_float), ("pad_", C.c_int32), ("tc_launches", C.c_int64),
                ("split_flops", C.c_double), ("split_ms", C.c_float), ("pad2_", C.c_int32),
                ("split_launches", C.c_int64), ("n_split", C.c_int64), ("fp32_tile", C.c_int64),
                ("h16_flops", C.c_double), ("h16_ms", C.c_float), ("pad3_", C.c_int32),
                ("h16_launches", C.c_int64), ("n_h16", C.c_int64), ("fp8_flops", C.c_double),
                ("fp8_ms", C.c_float), ("pad4_", C.c_int32), ("fp8_launches", C.c_int64),
                ("split_zmargin", C.c_float), ("split_acc_comp", C.c_float)]


class SlabC(C.Structure):
    _fields_ = [("z0", C.c_int32), ("z1", C.c_int32), ("halo", C.c_int32), ("flips", C.c_void_p)]


class SlabInfoC(C.Structure):
    _fields_ = [("verts3_local", C.c_int64), ("verts3_before", C.c_int64), ("verts3_owned", C.c_int64),
                ("case3_before", C.c_int64), ("case3_owned", C.c_int64), ("tris_before", C.c_int64),
                ("tris_owned", C.c_int64), ("fix_near_plane", C.c_int64)]


def slab_bounds(res_z: int, n_slabs: int) -> list:
    """Cell-layer ranges [z0, z1) of n_slabs slabs of near-equal depth (the
    split odc_extract_slabbed uses)."""
    return [(res_z * i // n_slabs, res_z * (i + 1) // n_slabs) for i in range(n_slabs)]


def label_words(grid) -> int:
    """Words of a grid's label bit set (odc_grid_labels); flip words are 3x."""
    return ((grid.res[0] + 32) // 32) * (grid.res[1] + 1) * (grid.res[2] + 1)


def slab_bases(counts: list, rank: int) -> dict:
    """Placement of slab ``rank`` in the merged mesh from every slab's owned
    counts (verts3_owned, case3_owned, tris_owned), slabs in z order: its 3D
    points follow the lower slabs' 3D points, its edge points follow all 3D
    points and the lower slabs' edge points, its triangles the lower slabs'
    triangles.  Also the merged totals."""
    v3 = [int(c[0]) for c in counts]
    c3 = [int(c[1]) for c in counts]
    tr = [int(c[2]) for c in counts]
    V = sum(v3)
    return dict(verts3_base=sum(v3[:rank]), case3_base=V + sum(c3[:rank]), tris_base=sum(tr[:rank]),
                n_verts=V + sum(c3), n_tris=sum(tr))


class MeshC(C.Structure):
    _fields_ = [("n_verts", C.c_int64), ("n_tris", C.c_int64), ("d_verts", C.c_void_p), ("d_tris", C.c_void_p),
                ("stats", Stats)]


class QualityC(C.Structure):
    _fields_ = [("n_samples", C.c_int64), ("occ_dev_mean", C.c_double), ("occ_dev_max", C.c_double),
                ("dist_mean", C.c_double), ("dist_max", C.c_double),
                ("n_tris", C.c_int64), ("n_verts", C.c_int64), ("n_edges", C.c_int64), ("euler", C.c_int64),
                ("n_degenerate", C.c_int64), ("n_bad_edges", C.c_int64), ("n_bad_verts", C.c_int64),
                ("manifold", C.c_int32), ("si_checked", C.c_int32), ("n_si_pairs", C.c_int64),
                ("n_si_tris", C.c_int64)]


Q_OCC, Q_MANIFOLD, Q_SI = 1, 2, 4


class ServerConfig(C.Structure):
    _fields_ = [("device", C.c_int32), ("slots", C.c_int32), ("mem_budget", C.c_size_t), ("host_copy", C.c_int32),
                ("share_network", C.c_int32)]


class ResultC(C.Structure):
    _fields_ = [("status", C.c_int32), ("slot", C.c_int32), ("mesh", MeshC), ("h_verts", C.c_void_p),
                ("h_tris", C.c_void_p), ("t_submit", C.c_double), ("t_start", C.c_double), ("t_end", C.c_double),
                ("est_bytes", C.c_uint64)]


def launch_total() -> int:
    """Kernel launches issued by the library so far (all contexts)."""
    return int(load().odc_launch_count())


EXPORTS = ["odc_ctx_create", "odc_ctx_destroy", "odc_extract", "odc_mesh_copy", "odc_mesh_release",
           "odc_debug_copy", "odc_eval_points", "odc_source_upload", "odc_launch_count", "odc_compact_edges_noalloc", "odc_status_str",
           "odc_last_error", "odc_server_create", "odc_server_destroy", "odc_submit", "odc_poll", "odc_result_release",
           "odc_server_clock", "odc_mesh_quality", "odc_extract_slab", "odc_slab_place", "odc_extract_slabbed",
           "odc_ctx_memory", "odc_grid_labels", "odc_manifold_flips", "odc_ctx_set_wait_limit", "odc_batch_create",
           "odc_batch_destroy", "odc_batch_stats", "odc_ctx_join_batch", "odc_extract_many"]

_lib = None


def load(path: str = LIB_PATH):
    """Load libodc.so (build it first with ``paper_2409_13418_gb300.build.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the CUDA library first (there is no fallback)")
    lib = C.CDLL(path)
    P = C.c_void_p
    lib.odc_ctx_create.argtypes = [C.c_int, C.c_size_t, C.POINTER(P)]
    lib.odc_ctx_destroy.argtypes = [P]
    lib.odc_extract.argtypes = [P, C.POINTER(Source), C.POINTER(Grid), C.POINTER(Params), P, C.POINTER(MeshC)]
    lib.odc_mesh_copy.argtypes = [P, C.POINTER(MeshC), P, P, C.c_int]
    lib.odc_ctx_memory.argtypes = [P, C.POINTER(C.c_size_t)]
    lib.odc_ctx_set_wait_limit.argtypes = [P, C.c_uint64, P]
    lib.odc_batch_create.argtypes = [C.c_int, C.POINTER(P)]
    lib.odc_batch_destroy.argtypes = [P]
    lib.odc_batch_stats.argtypes = [P, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
    lib.odc_ctx_join_batch.argtypes = [P, P]
    lib.odc_extract_many.argtypes = [P, C.c_int32, P, P, P, P, P, P]
    for f in ["odc_batch_create", "odc_batch_destroy", "odc_batch_stats", "odc_ctx_join_batch", "odc_extract_many"]:
        getattr(lib, f).restype = C.c_int
    lib.odc_ctx_set_wait_limit.restype = C.c_int
    lib.odc_grid_labels.argtypes = [P, C.POINTER(Source), C.POINTER(Grid), C.POINTER(Params), C.c_int32, C.c_int32, P,
                                    P]
    lib.odc_manifold_flips.argtypes = [P, C.POINTER(Grid), P, P, C.c_int32, P, C.POINTER(C.c_int64)]
    lib.odc_extract_slab.argtypes = [P, C.POINTER(Source), C.POINTER(Grid), C.POINTER(Params), C.POINTER(SlabC), P,
                                     C.POINTER(MeshC), C.POINTER(SlabInfoC)]
    lib.odc_slab_place.argtypes = [P, C.POINTER(MeshC), C.POINTER(SlabInfoC), C.c_int64, C.c_int64, C.c_int64, P, P,
                                   P]
    lib.odc_extract_slabbed.argtypes = [P, C.POINTER(Source), C.POINTER(Grid), C.POINTER(Params), C.c_int32,
                                        C.c_int32, P, C.POINTER(MeshC)]
    lib.odc_mesh_release.argtypes = [P, C.POINTER(MeshC)]
    lib.odc_debug_copy.argtypes = [P, C.c_int, P, C.c_size_t, C.POINTER(C.c_int64), C.POINTER(C.c_int32)]
    lib.odc_eval_points.argtypes = [P, C.POINTER(Source), P, C.c_int64, C.c_float, C.c_int, P, P]
    lib.odc_source_upload.argtypes = [P, C.POINTER(Source)]
    lib.odc_compact_edges_noalloc.argtypes = [P, C.POINTER(C.c_int32), P, C.c_uint32, P,
                                              C.POINTER(C.c_uint32), P]
    lib.odc_compact_edges_noalloc.restype = C.c_int
    lib.odc_mesh_quality.argtypes = [P, C.POINTER(MeshC), C.c_float, C.c_int64, C.c_uint64, C.c_int32,
                                     C.POINTER(QualityC)]
    lib.odc_mesh_quality.restype = C.c_int
    lib.odc_server_create.argtypes = [C.POINTER(ServerConfig), C.POINTER(P)]
    lib.odc_server_destroy.argtypes = [P]
    lib.odc_submit.argtypes = [P, C.POINTER(Source), C.POINTER(Grid), C.POINTER(Params), C.POINTER(C.c_uint64)]
    lib.odc_poll.argtypes = [P, C.c_uint64, C.c_int32, C.POINTER(ResultC)]
    lib.odc_result_release.argtypes = [P, C.c_uint64]
    lib.odc_server_clock.argtypes = [P]
    lib.odc_server_clock.restype = C.c_double
    lib.odc_launch_count.restype = C.c_int64
    lib.odc_launch_count.argtypes = []
    lib.odc_status_str.restype = C.c_char_p
    lib.odc_status_str.argtypes = [C.c_int]
    lib.odc_last_error.restype = C.c_char_p
    for f in ["odc_ctx_create", "odc_ctx_destroy", "odc_extract", "odc_mesh_copy", "odc_mesh_release",
              "odc_debug_copy", "odc_eval_points", "odc_source_upload", "odc_server_create", "odc_server_destroy",
              "odc_submit", "odc_poll", "odc_result_release"]:
        getattr(lib, f).restype = C.c_int
    _lib = lib
    return lib


class OdcError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _check(status):
    if status != ODC_OK:
        raise OdcError(status, _lib.odc_last_error().decode(errors="replace"))


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


class _SourceHolder:
    """Keeps the numpy buffers behind a Source structure alive."""

    def __init__(self, src, precision=None, band=None, split=True, split_zmargin=0.0, reupload=False,
                 fp32_tile=None, h16=True, h16_zmargin=0.0, split_acc_comp=0.0):
        self.keep = []
        self.src = Source()
        if src is None:
            self.src.kind = SRC_RESIDENT
        elif isinstance(src, I.CSGSource):
            rec = np.zeros(src.n_prims, dtype=np.dtype([("type", "<i4"), ("op", "<i4"), ("center", "<f4", 3),
                                                         ("rot", "<f4", 9), ("params", "<f4", 4),
                                                         ("pad", "<f4", 2)]))
            rec["type"] = src.types
            rec["op"] = src.ops
            rec["center"] = src.centers
            rec["rot"] = src.rot.reshape(-1, 9)
            rec["params"] = src.params
            self.keep.append(rec)
            self.src.kind = SRC_CSG
            self.src.n_prims = src.n_prims
            self.src.prims = _ptr(rec)
        elif isinstance(src, I.MLPSource):
            m = Mlp()
            m.n_freq = src.n_freq
            m.hidden = src.hidden
            m.n_hidden = len(src.weights) - 1
            m.latent_dim = 0 if src.latent is None else int(src.latent.shape[0])
            B = np.ascontiguousarray(src.B, np.float32)
            self.keep.append(B)
            m.B = _ptr(B)
            for i, (W, b) in enumerate(zip(src.weights, src.biases)):
                W = np.ascontiguousarray(W, np.float32)
                b = np.ascontiguousarray(b, np.float32)
                self.keep += [W, b]
                m.W[i] = _ptr(W)
                m.b[i] = _ptr(b)
            if src.latent is not None:
                lat = np.ascontiguousarray(src.latent, np.float32)
                self.keep.append(lat)
                m.latent = _ptr(lat)
            m.env_scale, m.env_radius, m.env_amp = src.env_scale, src.env_radius, src.env_amp
            m.precision = PREC_FP32 if precision is None else precision
            m.band = 0.03 if band is None else band
            m.no_split = 0 if split else 1
            m.split_zmargin = split_zmargin
            m.h16_zmargin = h16_zmargin
            m.split_acc_comp = split_acc_comp
            m.flags = (MLP_REUPLOAD if reupload else 0) | (((fp32_tile + 1) << 8) if fp32_tile is not None else 0) | \
                (0 if h16 else MLP_NO_F16_TIER)
            self.keep.append(m)
            self.src.kind = SRC_MLP
            self.src.mlp = C.addressof(m)
        elif isinstance(src, I.VoxelSource):
            vals = np.ascontiguousarray(src.values, np.float32)
            vx = Voxels()
            for a in range(3):
                vx.dims[a] = int(src.dims[a])
                vx.lo[a], vx.hi[a] = float(src.lo[a]), float(src.hi[a])
            vx.values = _ptr(vals)
            self.keep += [vals, vx]
            self.src.kind = SRC_VOXEL
            self.src.voxels = C.addressof(vx)
        else:
            raise TypeError(type(src))


def make_grid(grid: I.Grid) -> Grid:
    g = Grid()
    for a in range(3):
        g.lo[a], g.hi[a], g.res[a] = grid.lo[a], grid.hi[a], int(grid.res[a])
    return g


ABL_LINEAR_1D, ABL_GRADIENT_NORMALS, POLY_MC = 1, 2, 4


def make_params(steps_1d=15, iso=0.5, lin1=4, bin1=11, range1=0.8, lin2=3, bin2=12,
                range2=float(np.float32(np.sqrt(2.0) / 2.0)), ic_split=True, linear_1d=False,
                gradient_normals=False, mc=False) -> Params:
    p = Params()
    p.iso, p.steps_1d = iso, steps_1d
    p.s2d_lin1, p.s2d_bin1, p.s2d_range1 = lin1, bin1, range1
    p.s2d_lin2, p.s2d_bin2, p.s2d_range2 = lin2, bin2, range2
    p.ic_split = int(bool(ic_split))
    p.flags = (ABL_LINEAR_1D if linear_1d else 0) | (ABL_GRADIENT_NORMALS if gradient_normals else 0) | \
        (POLY_MC if mc else 0)
    return p


def compact_edges_noalloc(d_label_bits: int, res, d_edges: int, max_edges: int, d_count: int,
                          stream: int | None = None, read_count: bool = True) -> int | None:
    """Crossing edges of a device label bitmask with no allocation (odc_compact_edges_noalloc).

    All pointers are device addresses owned by the caller.  With
    ``read_count`` the call synchronises ``stream`` and returns the edge
    count; without it the count is only written to ``d_count`` (stream
    ordered, no host wait) and None is returned.
    """
    r = (C.c_int32 * 3)(*[int(x) for x in res])
    h = C.c_uint32()
    _check(load().odc_compact_edges_noalloc(d_label_bits, r, d_edges, max_edges, d_count,
                                            C.byref(h) if read_count else None, stream))
    return int(h.value) if read_count else None


class Mesh:
    def __init__(self, ctx, c: MeshC):
        self.ctx = ctx
        self.c = c
        self.n_verts = int(c.n_verts)
        self.n_tris = int(c.n_tris)
        s = c.stats
        self.stats = {f: getattr(s, f) for f, _ in Stats._fields_ if f != "stage_ms"}
        self.stats["stage_ms"] = list(s.stage_ms)

    def to_host(self):
        v = np.empty((self.n_verts, 3), np.float32)
        t = np.empty((self.n_tris, 3), np.int32)
        _check(_lib.odc_mesh_copy(self.ctx.h, C.byref(self.c), _ptr(v), _ptr(t), 0))
        return v, t

    def quality(self, iso: float = 0.5, n_samples: int = 2_000_000, seed: int = 1,
                what: int = Q_OCC | Q_MANIFOLD | Q_SI) -> dict:
        """Sec. 6.1 measures of this mesh (odc_mesh_quality): occupancy deviation on
        area-uniform samples, manifoldness and Euler characteristic, self-intersections."""
        q = QualityC()
        _check(_lib.odc_mesh_quality(self.ctx.h, C.byref(self.c), iso, n_samples, seed, what, C.byref(q)))
        return {f: getattr(q, f) for f, _ in QualityC._fields_}

    def copy_to(self, verts_ptr: int, tris_ptr: int, on_device: bool):
        _check(_lib.odc_mesh_copy(self.ctx.h, C.byref(self.c), verts_ptr, tris_ptr, int(on_device)))


class Context:
    """An ODC context on one CUDA device (``odc_ctx``)."""

    def __init__(self, device: int = 0, mem_budget: int = 0):
        load()
        h = C.c_void_p()
        _check(_lib.odc_ctx_create(device, mem_budget, C.byref(h)))
        self.h = h

    def close(self):
        if self.h:
            _lib.odc_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def upload(self, src, precision=None, band=None, split=True, split_zmargin=0.0, h16=True, fp32_tile=None,
               h16_zmargin=0.0, split_acc_comp=0.0):
        """Make ``src`` the context's resident source (``extract(None, ...)`` reuses it)."""
        holder = _SourceHolder(src, precision, band, split, split_zmargin, fp32_tile=fp32_tile, h16=h16,
                               h16_zmargin=h16_zmargin, split_acc_comp=split_acc_comp)
        _check(_lib.odc_source_upload(self.h, C.byref(holder.src)))

    def extract(self, src, grid: I.Grid, steps_1d=15, stream=None, precision=None, band=None, split=True,
                split_zmargin=0.0, reupload=False, h16=True, fp32_tile=None, h16_zmargin=0.0, split_acc_comp=0.0,
                **kw) -> Mesh:
        """Run ODC; ``src=None`` reuses the resident source.  ``reupload`` forces
        the network weights to be prepared and copied even if the context holds them;
        ``h16=False`` skips the FP16 tier of the BF16 path (same mesh, other cost);
        ``fp32_tile`` forces a tile shape of the FP32 network (same bits);
        ``split_acc_comp`` sets the split tier's accumulation compensation (0:
        calibrated per network at upload, negative: none) and ``split_zmargin``
        its margin (0: calibrated per network at upload); the margin in use is
        ``Mesh.stats["split_zmargin"]``."""
        holder = _SourceHolder(src, precision, band, split, split_zmargin, reupload, fp32_tile=fp32_tile, h16=h16,
                               h16_zmargin=h16_zmargin, split_acc_comp=split_acc_comp)
        g = make_grid(grid)
        p = make_params(steps_1d=steps_1d, **kw)
        m = MeshC()
        _check(_lib.odc_extract(self.h, C.byref(holder.src), C.byref(g), C.byref(p),
                                stream if stream else None, C.byref(m)))
        return Mesh(self, m)

    def join_batch(self, batch) -> None:
        """odc_ctx_join_batch: share search-stage network evaluations with the
        group's other members (None: leave)."""
        _check(_lib.odc_ctx_join_batch(self.h, batch.h if batch is not None else None))

    def set_wait_limit(self, ns: int, gate: int | None = None) -> None:
        """odc_ctx_set_wait_limit: limit of the tensor-core kernels' pipeline
        waits in ns (0: the default) and an optional device go flag (address
        of a device int32, None for none)."""
        _check(_lib.odc_ctx_set_wait_limit(self.h, int(ns), gate))

    def device_bytes(self) -> int:
        """odc_ctx_memory: device bytes the context holds."""
        b = C.c_size_t()
        _check(_lib.odc_ctx_memory(self.h, C.byref(b)))
        return int(b.value)

    def grid_labels(self, src, grid: I.Grid, z0: int, z1: int, d_bits: int, stream=None, precision=None, band=None,
                    split=True, split_zmargin=0.0, iso: float = 0.5):
        """odc_grid_labels: label words of vertex layers [z0, z1] into d_bits."""
        holder = _SourceHolder(src, precision, band, split, split_zmargin)
        g = make_grid(grid)
        p = make_params(iso=iso)
        _check(_lib.odc_grid_labels(self.h, C.byref(holder.src), C.byref(g), C.byref(p), z0, z1, d_bits,
                                    stream if stream else None))

    def manifold_flips(self, grid: I.Grid, d_bits: int, d_flips: int, n_chunks: int = 8, stream=None) -> int:
        """odc_manifold_flips: the whole grid's manifold fix; returns faces flipped."""
        g = make_grid(grid)
        n = C.c_int64()
        _check(_lib.odc_manifold_flips(self.h, C.byref(g), d_bits, d_flips, n_chunks, stream if stream else None,
                                       C.byref(n)))
        return int(n.value)

    def extract_slab(self, src, grid: I.Grid, z0: int, z1: int, halo: int = 2, steps_1d=15, stream=None,
                     precision=None, band=None, split=True, split_zmargin=0.0, flips: int = 0, **kw):
        """odc_extract_slab: the slab extraction's mesh and its owned ranges
        (``flips``: device pointer to the whole grid's flip words, or 0)."""
        holder = _SourceHolder(src, precision, band, split, split_zmargin)
        g = make_grid(grid)
        p = make_params(steps_1d=steps_1d, **kw)
        sl = SlabC(z0, z1, halo, flips if flips else None)
        m = MeshC()
        info = SlabInfoC()
        _check(_lib.odc_extract_slab(self.h, C.byref(holder.src), C.byref(g), C.byref(p), C.byref(sl),
                                     stream if stream else None, C.byref(m), C.byref(info)))
        return Mesh(self, m), info

    def slab_place(self, mesh, info, verts3_base: int, case3_base: int, tris_base: int, d_verts: int, d_tris: int,
                   stream=None):
        """odc_slab_place: the owned part of the latest slab extraction into a
        whole-grid mesh in device memory (caller-owned pointers)."""
        _check(_lib.odc_slab_place(self.h, C.byref(mesh.c), C.byref(info), verts3_base, case3_base, tris_base,
                                   d_verts, d_tris, stream if stream else None))

    def extract_slabbed(self, src, grid: I.Grid, n_slabs: int, halo: int = 2, steps_1d=15, stream=None,
                        precision=None, band=None, split=True, split_zmargin=0.0, **kw) -> Mesh:
        """odc_extract_slabbed: the grid in n_slabs z-slabs on this context, merged."""
        holder = _SourceHolder(src, precision, band, split, split_zmargin)
        g = make_grid(grid)
        p = make_params(steps_1d=steps_1d, **kw)
        m = MeshC()
        _check(_lib.odc_extract_slabbed(self.h, C.byref(holder.src), C.byref(g), C.byref(p), n_slabs, halo,
                                        stream if stream else None, C.byref(m)))
        return Mesh(self, m)

    def face_points(self) -> np.ndarray:
        """2D points of the last extract as float64 (u, v) (stored float-float)."""
        r = self.debug("face_pts").astype(np.float64)
        return np.stack([r[:, 0] + r[:, 1], r[:, 2] + r[:, 3]], axis=1)

    def search_decisions(self) -> dict:
        """2D search decisions of the last extract: Jq, J1, J2, lab_m, found."""
        raw = self.debug("search")
        b = raw[:, 3].copy().view(np.uint8).reshape(-1, 4)
        return dict(Jq=raw[:, 0].astype(np.int64), J1=raw[:, 1].astype(np.int64), J2=raw[:, 2].astype(np.int64),
                    lab_m=b[:, 0].astype(bool), found=b[:, 1].astype(np.int64))

    def debug(self, what: str) -> np.ndarray:
        n = C.c_int64()
        eb = C.c_int32()
        _check(_lib.odc_debug_copy(self.h, DBG[what], None, 0, C.byref(n), C.byref(eb)))
        dt = np.dtype(_DBG_DTYPE[what])
        k = _DBG_SHAPE.get(what, 1)
        out = np.empty(int(n.value) * k, dt)
        _check(_lib.odc_debug_copy(self.h, DBG[what], _ptr(out), out.nbytes, C.byref(n), C.byref(eb)))
        return out.reshape(-1, k) if k > 1 else out

    def quality_of(self, d_verts: int, n_verts: int, d_tris: int, n_tris: int, iso: float = 0.5,
                   n_samples: int = 2_000_000, seed: int = 1, what: int = Q_OCC | Q_MANIFOLD | Q_SI) -> dict:
        """odc_mesh_quality on any mesh in device memory (float32 [n][3] vertices,
        int32 [m][3] triangles); the occupancy is the context's resident source."""
        m = MeshC()
        m.n_verts, m.n_tris, m.d_verts, m.d_tris = n_verts, n_tris, d_verts, d_tris
        q = QualityC()
        _check(_lib.odc_mesh_quality(self.h, C.byref(m), iso, n_samples, seed, what, C.byref(q)))
        return {f: getattr(q, f) for f, _ in QualityC._fields_}

    def eval_points(self, src, pts: np.ndarray, iso: float = 0.5, precision: int = -1, band=None, split=True,
                    fp32_tile=None, split_acc_comp=0.0):
        # the source's precision: FP32, BF16 or FP8 tiers; the single-network
        # overrides (split, FP16, raw FP8) run on a BF16 source's state
        sp = None if precision < 0 else (precision if precision in (PREC_FP32, PREC_BF16, PREC_FP8) else PREC_BF16)
        holder = _SourceHolder(src, sp, band, split, fp32_tile=fp32_tile, split_acc_comp=split_acc_comp)
        pts = np.ascontiguousarray(pts, np.float32).reshape(-1, 3)
        lab = np.empty(pts.shape[0], np.uint8)
        z = np.empty(pts.shape[0], np.float32)
        _check(_lib.odc_eval_points(self.h, C.byref(holder.src), _ptr(pts), pts.shape[0], iso, precision,
                                    _ptr(lab), _ptr(z)))
        return lab.astype(bool), z


class Batch:
    """A batch group (``odc_batch``): contexts that join it share the network
    evaluations of their search stages."""

    def __init__(self, device: int = 0):
        load()
        h = C.c_void_p()
        _check(_lib.odc_batch_create(device, C.byref(h)))
        self.h = h

    def close(self):
        if self.h:
            _lib.odc_batch_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def stats(self) -> dict:
        r, c = C.c_int64(), C.c_int64()
        _check(_lib.odc_batch_stats(self.h, C.byref(r), C.byref(c)))
        return {"rounds": int(r.value), "calls": int(c.value)}


def extract_many(batch, ctxs, jobs) -> list:
    """odc_extract_many: jobs[i] = (src, grid, kwargs) on ctxs[i] (distinct
    contexts), one host thread per shape, all joined to ``batch`` (None: no
    sharing).  Returns the meshes (each valid until its context's next
    extract)."""
    n = len(jobs)
    holders = [_SourceHolder(src, kw.get("precision"), kw.get("band"), kw.get("split", True), kw.get("split_zmargin", 0.0),
                             kw.get("reupload", False), h16=kw.get("h16", True)) for src, _, kw in jobs]
    srcs = (Source * n)(*[h.src for h in holders])
    grids = (Grid * n)(*[make_grid(g) for _, g, _ in jobs])
    skip = {"precision", "band", "split", "split_zmargin", "reupload", "h16"}
    prms = (Params * n)(*[make_params(**{k: v for k, v in kw.items() if k not in skip}) for _, _, kw in jobs])
    outs = (MeshC * n)()
    sts = (C.c_int * n)()
    hs = (C.c_void_p * n)(*[c.h.value for c in ctxs])
    r = _lib.odc_extract_many(batch.h if batch is not None else None, n, hs, srcs, grids, prms, outs, sts)
    _check(r)
    return [Mesh(c, outs[i]) for i, c in enumerate(ctxs)]


class Server:
    """The library's request loop (``odc_server``): requests of any grid size
    are admitted as slots and memory free up and run concurrently on the GPU."""

    def __init__(self, device: int = 0, slots: int = 4, mem_budget: int = 0, host_copy: bool = True,
                 share_network: bool = False):
        load()
        cfg = ServerConfig()
        cfg.device, cfg.slots, cfg.mem_budget, cfg.host_copy = device, slots, mem_budget, int(bool(host_copy))
        cfg.share_network = int(bool(share_network))
        h = C.c_void_p()
        _check(_lib.odc_server_create(C.byref(cfg), C.byref(h)))
        self.h = h

    def close(self):
        if self.h:
            _lib.odc_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def clock(self) -> float:
        return float(_lib.odc_server_clock(self.h))

    def submit(self, src, grid: I.Grid, steps_1d=15, precision=None, band=None, split=True, split_zmargin=0.0,
               **kw) -> int:
        """Queue one request (inputs are copied by the library); returns its id."""
        holder = _SourceHolder(src, precision, band, split, split_zmargin)
        g = make_grid(grid)
        p = make_params(steps_1d=steps_1d, **kw)
        rid = C.c_uint64()
        _check(_lib.odc_submit(self.h, C.byref(holder.src), C.byref(g), C.byref(p), C.byref(rid)))
        return int(rid.value)

    def poll(self, rid: int, timeout_ms: int = -1):
        """None while the request runs (after timeout_ms); else a dict with the
        request's status, host mesh copies (when the server keeps them), times
        and slot."""
        r = ResultC()
        st = _lib.odc_poll(self.h, rid, timeout_ms, C.byref(r))
        if st == 4:
            return None
        _check(st)
        out = dict(status=int(r.status), slot=int(r.slot), t_submit=r.t_submit, t_start=r.t_start, t_end=r.t_end,
                   est_bytes=int(r.est_bytes), n_verts=int(r.mesh.n_verts), n_tris=int(r.mesh.n_tris))
        if r.status != ODC_OK:
            out["error"] = _lib.odc_last_error().decode(errors="replace")
        else:
            s = r.mesh.stats
            out["stats"] = {f: getattr(s, f) for f, _ in Stats._fields_ if f != "stage_ms"}
            if r.h_verts or not out["n_verts"]:
                nv, nt = out["n_verts"], out["n_tris"]
                out["verts"] = np.ctypeslib.as_array((C.c_float * (3 * nv)).from_address(r.h_verts)).reshape(nv, 3).copy() if nv else np.zeros((0, 3), np.float32)
                out["tris"] = np.ctypeslib.as_array((C.c_int32 * (3 * nt)).from_address(r.h_tris)).reshape(nt, 3).copy() if nt else np.zeros((0, 3), np.int32)
        return out

    def release(self, rid: int):
        _check(_lib.odc_result_release(self.h, rid))
