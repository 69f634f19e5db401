"""GPU-vs-oracle parity of the MLP occupancy path (FP32 network).

The FP32 network differs from the FP64 oracle by rounding only; every
decision whose oracle margin |occ - 0.5| is below MARGIN (2e-5, i.e. |z| <
8e-5, an order of magnitude above the measured FP32 logit error) is flagged,
and elements fed by a flagged decision are excluded from the strict checks.
"""
import numpy as np
import pytest

from oracle import meshcheck, odc as oracle
from oracle.occupancy import mlp_logit
from paper_2409_13418_gb300 import inputs as I
from tests.parity_util import compare

pytestmark = pytest.mark.gpu

MARGIN = 2e-5


@pytest.fixture(scope="module")
def ctx():
    from paper_2409_13418_gb300 import build, odc
    build.build()
    c = odc.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def mlp():
    return I.envelope_mlp(0)


def test_fp32_logits_match_fp64(ctx, mlp):
    rng = np.random.default_rng(1)
    pts = rng.uniform(-1, 1, (60000, 3)).astype(np.float32)
    lab, z = ctx.eval_points(mlp, pts, precision=0)
    zr = mlp_logit(mlp, pts.astype(np.float64))
    err = np.abs(z.astype(np.float64) - zr)
    print("max |z_fp32 - z_fp64|", err.max(), "median", np.median(err))
    assert err.max() < 8e-5
    sure = np.abs(zr) > 8e-5
    assert np.array_equal(lab[sure], (zr > 0)[sure])


@pytest.mark.parametrize("n", [24, 40])
def test_fp32_extract_parity(ctx, mlp, n):
    g = I.cube_grid(n)
    ref = oracle.extract(mlp, g, steps_1d=15)
    mesh = ctx.extract(mlp, g, steps_1d=15)
    rep, verts, tris = compare(ctx, mesh, ref, margin_eps=MARGIN)
    print(n, rep, ref.stats, mesh.stats)
    assert meshcheck.check_closed_manifold(tris)["ok"]


def test_resident_source_gives_same_mesh(ctx, mlp):
    g = I.cube_grid(32)
    v1, t1 = ctx.extract(mlp, g, steps_1d=12).to_host()
    ctx.upload(mlp)
    v2, t2 = ctx.extract(None, g, steps_1d=12).to_host()
    assert np.array_equal(t1, t2) and np.array_equal(v1, v2)
