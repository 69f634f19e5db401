"""Marching-cubes polygonization through the 1D points (Tab. A8's MC rows)
on the GPU against the oracle: the same vertices (1D points, edge order) and
the same triangles, for CSG (bisected and linear 1D points) and MLP sources."""
import numpy as np
import pytest

from oracle import meshcheck, odc as oracle
from paper_2409_13418_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2409_13418_gb300 import build, odc
    build.build()
    c = odc.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("case", ["config1", "csg2", "csg2-linear", "torus-ragged", "mlp", "mlp-bf16"])
def test_mc_mesh_matches_oracle(ctx, case):
    kw = dict(mc=True)
    if case == "config1":
        src, g, k = I.config1_csg(), I.cube_grid(32), 10
    elif case.startswith("csg2"):
        src, g, k = I.random_csg(2, n_prims=64), I.cube_grid(64), 12
        kw["linear_1d"] = case.endswith("linear")
    elif case == "torus-ragged":
        src = I.single_prim(I.PRIM_TORUS, (0.02, -0.03, 0.01), params=(0.5, 0.2))
        g, k = I.Grid((-0.83, -0.9, -0.4), (0.88, 0.79, 0.42), (45, 37, 29)), 12
    else:
        src, g, k = I.envelope_mlp(0), I.cube_grid(40), 15
    prec = dict(precision=1) if case == "mlp-bf16" else (dict(precision=0) if case == "mlp" else {})
    mesh = ctx.extract(src, g, steps_1d=k, **kw, **prec)
    v, t = mesh.to_host()
    if case.startswith("mlp"):
        # decisions near the surface may legitimately differ between FP32 and FP64;
        # replay the GPU's 1D results through the oracle
        T = ctx.debug("T").astype(np.int64)
        ref = oracle.extract(src, g, steps_1d=k, replay=dict(T=T, Jq=None, J1=None, J2=None, lab_m=None,
                                                             found=None), replay_margin=2e-5, **kw)
        assert ref.stats["edge_violations"] == 0
    else:
        ref = oracle.extract(src, g, steps_1d=k, **kw)
        assert np.array_equal(ctx.debug("T").astype(np.int64), ref.T)
    assert np.array_equal(t.astype(np.int64), ref.triangles)
    assert np.array_equal(v.astype(np.float64), ref.vertices)
    assert meshcheck.check_closed_manifold(t)["ok"] and meshcheck.signed_volume(v, t) > 0
    assert mesh.stats["n_verts3"] == 0 and mesh.n_verts == mesh.stats["n_edges"]
