"""GPU-vs-oracle parity of the whole CSG path through the C ABI.

Sizes span several 32-vertex words per row and ragged tails; the 128^3
64-primitive chain is the config the paper-scale CSG workload runs.
"""
import math

import numpy as np
import pytest

from oracle import meshcheck, odc as oracle
from paper_2409_13418_gb300 import inputs as I
from tests.parity_util import compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2409_13418_gb300 import build, odc
    build.build()
    c = odc.Context(0)
    yield c
    c.close()


def _run(ctx, src, grid, k, **kw):
    ref = oracle.extract(src, grid, steps_1d=k, **kw)
    mesh = ctx.extract(src, grid, steps_1d=k, **kw)
    rep, verts, tris = compare(ctx, mesh, ref)
    h = np.array([(grid.hi[a] - grid.lo[a]) / grid.res[a] for a in range(3)])
    if verts.shape == ref.vertices.shape:
        err = np.max(np.abs(verts - ref.vertices) / h, axis=1)
        nv3 = ref.verts_local.shape[0]
        ok = np.ones(len(err), bool)
        ok[:nv3] = ~(ref.vert_flag | (ref.vert_margin < 1e-12))
        assert err[ok].max(initial=0) < 1e-4 + 1e-6 / h.min()
    return ref, mesh, rep, verts, tris


def test_config1_sphere_box(ctx):
    ref, mesh, rep, verts, tris = _run(ctx, I.config1_csg(), I.cube_grid(32), 10)
    assert rep["vert_flagged_max_err"] < 1e-4
    assert meshcheck.check_closed_manifold(tris)["ok"]
    assert meshcheck.euler_characteristic(tris) == 2
    assert mesh.stats["n_edges"] == ref.stats["E"]


@pytest.mark.parametrize("seed", [1, 2])
def test_config2_random_csg_128(ctx, seed):
    src = I.random_csg(seed)
    ref, mesh, rep, verts, tris = _run(ctx, src, I.cube_grid(128), 12)
    print(seed, rep, ref.stats)
    # required: grid margins >= 1e-6 on reported seeds
    assert ref.label_margin.min() > 0
    assert meshcheck.check_closed_manifold(tris)["ok"]


@pytest.mark.parametrize("res", [(33, 33, 33), (47, 20, 35), (1, 1, 1), (2, 3, 5)])
def test_ragged_and_tiny_grids(ctx, res):
    src = I.random_csg(7, n_prims=8)
    g = I.Grid((-0.8, -0.9, -0.85), (0.9, 0.8, 0.95), res)
    _run(ctx, src, g, 9)


def test_empty_and_full(ctx):
    # nothing inside the box
    src = I.single_prim(I.PRIM_SPHERE, (5.0, 5.0, 5.0), params=(0.2,))
    m = ctx.extract(src, I.cube_grid(40), steps_1d=8)
    assert m.n_tris == 0 and m.n_verts == 0 and m.stats["n_edges"] == 0
    # everything inside: no crossing either
    src = I.single_prim(I.PRIM_SPHERE, (0.0, 0.0, 0.0), params=(10.0,))
    m = ctx.extract(src, I.cube_grid(40), steps_1d=8)
    assert m.n_tris == 0 and m.stats["n_cells"] == 0


def test_open_surface_at_boundary(ctx):
    # a sphere cut by the grid box: boundary crossing edges emit no quads
    src = I.single_prim(I.PRIM_SPHERE, (0.9, 0.0, 0.0), params=(0.5,))
    _run(ctx, src, I.cube_grid(24), 10)


def test_manifold_fix_cases(ctx):
    # random voxel-like CSG of many small boxes: ambiguous faces and flips
    prims = []
    rng = np.random.default_rng(3)
    for i in range(60):
        c = rng.integers(1, 9, 3) / 10.0 * 2 - 1
        prims.append((I.PRIM_AABB, I.OP_UNION, tuple(c), None, (0.09, 0.09, 0.09)))
    src = I.csg_from_list(prims)
    ref, mesh, rep, verts, tris = _run(ctx, src, I.cube_grid(20), 8)
    assert meshcheck.check_closed_manifold(tris)["ok"]


def test_ic_off_and_steps(ctx):
    src = I.random_csg(11, n_prims=16)
    _run(ctx, src, I.cube_grid(48), 14, ic_split=False)
    _run(ctx, src, I.cube_grid(48), 1)


def test_deterministic_bytes(ctx):
    src = I.random_csg(4)
    g = I.cube_grid(64)
    v1, t1 = ctx.extract(src, g, steps_1d=12).to_host()
    v2, t2 = ctx.extract(src, g, steps_1d=12).to_host()
    assert v1.tobytes() == v2.tobytes() and t1.tobytes() == t2.tobytes()


def test_point_labels_match_oracle(ctx):
    from oracle.occupancy import csg_eval
    src = I.random_csg(9)
    rng = np.random.default_rng(0)
    pts = rng.uniform(-1, 1, (200000, 3)).astype(np.float32)
    # points very close to primitive surfaces exercise the float-float path
    c = src.centers[0].astype(np.float64)
    dirs = rng.standard_normal((20000, 3))
    dirs /= np.linalg.norm(dirs, axis=1)[:, None]
    near = (c + dirs * float(src.params[0, 0]) * (1 + rng.uniform(-1e-6, 1e-6, (20000, 1)))).astype(np.float32)
    pts = np.concatenate([pts, near])
    lab, _ = ctx.eval_points(src, pts)
    ref, _ = csg_eval(src, pts.astype(np.float64))
    assert np.array_equal(lab, ref)


def test_invalid_arguments(ctx):
    from paper_2409_13418_gb300.odc import OdcError
    src = I.config1_csg()
    with pytest.raises(OdcError):
        ctx.extract(src, I.Grid((0, 0, 0), (1, 1, 1), (0, 4, 4)), steps_1d=5)
    with pytest.raises(OdcError):
        ctx.extract(src, I.Grid((1, 0, 0), (0, 1, 1), (4, 4, 4)), steps_1d=5)
    with pytest.raises(OdcError):
        ctx.extract(src, I.cube_grid(8), steps_1d=0)
    with pytest.raises(OdcError):
        ctx.extract(src, I.cube_grid(2000), steps_1d=5)
