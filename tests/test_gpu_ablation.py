"""The ablation's Manifold Dual Contouring variants (Sec. 6.3, Tab. 3) on the
GPU against the oracle: linear 1D points (Eq. 1, FP32, quantised: bit-exact
integers), gradient normals (Eq. 3), the fixed quad diagonal; topology and
triangles exact, 3D points within 1e-4 cell."""
import numpy as np
import pytest

from oracle import meshcheck, odc as oracle
from paper_2409_13418_gb300 import inputs as I
from tests.parity_util import compare

pytestmark = pytest.mark.gpu

VARIANTS = {
    "mdc": dict(linear_1d=True, gradient_normals=True, ic_split=False),
    "mdc+1d": dict(gradient_normals=True, ic_split=False),
    "mdc+1d+2d": dict(ic_split=False),
    "linear+2d+ic": dict(linear_1d=True),
}


@pytest.fixture(scope="module")
def ctx():
    from paper_2409_13418_gb300 import build, odc
    build.build()
    c = odc.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("shape", ["config1", "csg2", "csg5"])
@pytest.mark.parametrize("variant", list(VARIANTS))
def test_ablation_variant_matches_oracle(ctx, shape, variant):
    src, n, k = {"config1": (I.config1_csg(), 32, 10), "csg2": (I.random_csg(2, n_prims=64), 64, 12),
                 "csg5": (I.random_csg(5, n_prims=24), 40, 12)}[shape]
    kw = VARIANTS[variant]
    g = I.cube_grid(n)
    mesh = ctx.extract(src, g, steps_1d=k, **kw)
    ref = oracle.extract(src, g, steps_1d=k, **kw)
    rep, verts, tris = compare(ctx, mesh, ref)
    print(shape, variant, rep)
    assert meshcheck.check_closed_manifold(tris)["ok"]


def test_ablation_flags_need_an_implicit(ctx):
    from paper_2409_13418_gb300 import odc
    with pytest.raises(odc.OdcError) as e:
        ctx.extract(I.envelope_mlp(0), I.cube_grid(16), steps_1d=8, gradient_normals=True)
    assert e.value.status == 5     # ODC_ERR_UNSUPPORTED
