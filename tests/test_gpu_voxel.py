"""Dense voxel-grid occupancy source on the GPU against the oracle: labels,
1D and 2D decisions and topology exact (float-float trilinear against the
FP64 oracle; near-ties flagged), 3D points within 1e-4 cell; the random-sign
volumes stress the topology; served requests and MC meshes too."""
import numpy as np
import pytest

from oracle import meshcheck, odc as oracle, quality as Q
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


@pytest.mark.parametrize("case", ["random9-16", "random17-40", "blobs-48", "blobs-ragged", "random-iso"])
def test_voxel_extract_matches_oracle(ctx, case):
    iso = 0.5
    if case == "random9-16":
        src, g = I.voxel_random(1, (9, 9, 9)), I.cube_grid(16)
    elif case == "random17-40":
        src, g = I.voxel_random(2, (17, 13, 15)), I.cube_grid(40)
    elif case == "blobs-48":
        src, g = I.voxel_blobs(3), I.cube_grid(48)
    elif case == "blobs-ragged":
        src, g = I.voxel_blobs(4), I.Grid((-0.9, -0.85, -0.95), (0.87, 0.93, 0.8), (41, 37, 45))
    else:
        src, g, iso = I.voxel_random(5, (11, 11, 11)), I.cube_grid(24), 0.37
    mesh = ctx.extract(src, g, steps_1d=12, iso=iso)
    ref = oracle.extract(src, g, steps_1d=12, iso=iso)
    rep, v, t = compare(ctx, mesh, ref)
    print(case, rep)
    assert meshcheck.check_closed_manifold(t)["ok"]


def test_voxel_mc_quality_points_and_serving(ctx):
    from paper_2409_13418_gb300 import odc
    src, g = I.voxel_blobs(6), I.cube_grid(40)
    mesh = ctx.extract(src, g, steps_1d=12, mc=True)
    ref = oracle.extract(src, g, steps_1d=12, mc=True)
    v, t = mesh.to_host()
    assert np.array_equal(t.astype(np.int64), ref.triangles) and np.array_equal(v.astype(np.float64), ref.vertices)
    q = mesh.quality(n_samples=100000, seed=2)
    mean, mx = Q.voxel_deviation(src, v, t, 100000, seed=2)
    assert abs(q["occ_dev_mean"] - mean) < 1e-9 and abs(q["occ_dev_max"] - mx) < 1e-7
    rng = np.random.default_rng(0)
    pts = rng.uniform(-1.1, 1.1, (50000, 3)).astype(np.float32)
    lab, _ = ctx.eval_points(src, pts, iso=0.5)
    from oracle.occupancy import voxel_eval
    lr, mr = voxel_eval(src, pts.astype(np.float64), 0.5)
    sure = mr > 1e-12
    assert np.array_equal(lab[sure], lr[sure])
    alone = ctx.extract(src, g, steps_1d=12).to_host()
    with odc.Server(0, slots=2) as srv:
        rid = srv.submit(src, g, steps_1d=12)
        r = srv.poll(rid)
        assert np.array_equal(r["verts"], alone[0]) and np.array_equal(r["tris"], alone[1])
