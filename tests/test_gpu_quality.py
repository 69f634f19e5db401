"""odc_mesh_quality (Sec. 6.1 metrics) on the GPU against the oracle's
measures on the same mesh: the occupancy deviation on the same SplitMix64
samples, manifoldness and Euler characteristic, and the self-intersecting
triangle pairs."""
import math

import numpy as np
import pytest

from oracle import meshcheck, quality as Q
from paper_2409_13418_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2409_13418_gb300 import build, odc
    build.build()
    c = odc.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("n,precision", [(24, 0), (40, 1)])
def test_mlp_mesh_quality_matches_oracle(ctx, n, precision):
    mlp = I.envelope_mlp(0)
    mesh = ctx.extract(mlp, I.cube_grid(n), steps_1d=12, precision=precision)
    v, t = mesh.to_host()
    q = mesh.quality(n_samples=200000, seed=3)
    mean, mx = Q.occupancy_deviation(mlp, v, t, 200000, seed=3)
    print(q, mean, mx)
    assert q["n_samples"] == 200000
    assert abs(q["occ_dev_mean"] - mean) < 1e-5 and abs(q["occ_dev_max"] - mx) < 1e-4
    assert q["manifold"] == 1 and meshcheck.check_closed_manifold(t)["ok"]
    assert q["euler"] == meshcheck.euler_characteristic(t)
    assert q["n_bad_edges"] == 0 and q["n_bad_verts"] == 0 and q["n_degenerate"] == 0
    if n <= 24:
        c, flag = Q.self_intersections(v, t)
        assert q["n_si_pairs"] == c and q["n_si_tris"] == int(flag.sum())


def test_csg_mesh_quality_matches_oracle(ctx):
    src = I.random_csg(4, n_prims=12)
    mesh = ctx.extract(src, I.cube_grid(20), steps_1d=10)
    v, t = mesh.to_host()
    q = mesh.quality(n_samples=100000, seed=4)
    assert math.isnan(q["occ_dev_mean"]) and q["n_samples"] == 100000   # binary occupancy: distance instead
    dm, dx = Q.surface_distance(src, v, t, 100000, seed=4)
    print(q["dist_mean"], dm, q["dist_max"], dx)
    assert abs(q["dist_mean"] - dm) <= 1e-6 * max(dm, 1e-3) + 1e-9 and abs(q["dist_max"] - dx) <= 1e-5 * dx
    c, flag = Q.self_intersections(v, t)
    assert q["n_si_pairs"] == c > 0 and q["n_si_tris"] == int(flag.sum())
    assert q["manifold"] == 1 and q["euler"] == meshcheck.euler_characteristic(t)


def test_broken_meshes_are_flagged(ctx):
    import torch
    mesh = ctx.extract(I.config1_csg(), I.cube_grid(32), steps_1d=10)
    v, t = mesh.to_host()
    dv = torch.from_numpy(v).cuda()
    what = 2   # manifoldness only
    for tt, expect_bad in ((t, False), (t[1:], True), (np.concatenate([t, t[:1]]), True),
                           (np.concatenate([t, [[0, 0, 1]]]), True)):
        dt = torch.from_numpy(np.ascontiguousarray(tt, np.int32)).cuda()
        q = ctx.quality_of(dv.data_ptr(), v.shape[0], dt.data_ptr(), tt.shape[0], what=what)
        assert q["manifold"] == (0 if expect_bad else 1)
        assert (not meshcheck.check_closed_manifold(tt)["ok"]) == expect_bad
    from paper_2409_13418_gb300 import odc
    bad = torch.from_numpy(np.array([[0, 1, v.shape[0]]], np.int32)).cuda()
    with pytest.raises(odc.OdcError):
        ctx.quality_of(dv.data_ptr(), v.shape[0], bad.data_ptr(), 1, what=7)
