"""Shared network evaluations (batch groups): shapes extracted together,
their search-stage queries merged into common network launches, give the
same meshes byte for byte as each shape extracted alone -- latent-conditioned
shapes of one network (each query carrying its shape's folded first-layer
bias), shapes at another iso level (evaluated apart, same group), a shape of
another network and a CSG shape (evaluated on their own), on cubic and
ragged grids, with the BF16 and the FP8 first pass; and the same through
the request loop with shared evaluations."""
import numpy as np
import pytest

from paper_2409_13418_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _alone(jobs):
    from paper_2409_13418_gb300 import odc
    out = []
    with odc.Context(0) as ctx:
        for src, g, kw in jobs:
            out.append(ctx.extract(src, g, **kw).to_host())
    return out


def _jobs(prec):
    net = I.envelope_mlp(12, latent_dim=128)
    other = I.envelope_mlp(3)
    return [
        (I.with_latent(net, 2001), I.cube_grid(48), dict(steps_1d=15, precision=prec)),
        (I.with_latent(net, 2002), I.cube_grid(64), dict(steps_1d=15, precision=prec)),
        (I.with_latent(net, 2003), I.Grid((-0.93, -0.88, -0.97), (0.91, 0.95, 0.9), (41, 33, 47)),
         dict(steps_1d=12, precision=prec)),
        (I.with_latent(net, 2004), I.cube_grid(40), dict(steps_1d=15, precision=prec, iso=0.4)),
        (I.with_latent(net, 2005), I.cube_grid(56), dict(steps_1d=15, precision=prec, lin1=2, bin1=9)),
        (other, I.cube_grid(44), dict(steps_1d=15, precision=prec)),
        (I.random_csg(5, 24), I.cube_grid(40), dict(steps_1d=12)),
    ]


@pytest.mark.parametrize("prec_name", ["bf16", "fp8"])
def test_extract_many_equals_alone(prec_name):
    from paper_2409_13418_gb300 import build, odc
    build.build()
    prec = odc.PREC_BF16 if prec_name == "bf16" else odc.PREC_FP8
    jobs = _jobs(prec)
    ref = _alone(jobs)
    ctxs = [odc.Context(0) for _ in jobs]
    try:
        with odc.Batch(0) as b:
            for rep in range(2):   # the second pass reuses bound contexts with new latents' rows
                meshes = odc.extract_many(b, ctxs, jobs)
                got = [m.to_host() for m in meshes]
                for i, ((v, t), (vr, tr)) in enumerate(zip(got, ref)):
                    assert v.tobytes() == vr.tobytes() and np.array_equal(t, tr), (rep, i)
            st = b.stats()
            print(prec_name, st)
            # the five shapes of the shared network met in common rounds
            assert st["rounds"] > 0 and st["calls"] > 1.5 * st["rounds"]
            for c in ctxs:
                c.join_batch(None)
    finally:
        for c in ctxs:
            c.close()


def test_server_shared_network_equals_alone():
    from paper_2409_13418_gb300 import build, odc
    build.build()
    jobs = _jobs(odc.PREC_BF16)
    ref = _alone(jobs)
    with odc.Server(0, slots=4, host_copy=True, share_network=True) as srv:
        for rep in range(2):
            ids = [srv.submit(src, g, **kw) for src, g, kw in jobs]
            for i, rid in enumerate(ids):
                r = srv.poll(rid)
                assert r["status"] == 0
                v, t = r["verts"], r["tris"]
                assert v.tobytes() == ref[i][0].tobytes() and np.array_equal(t, ref[i][1]), (rep, i)
                srv.release(rid)
