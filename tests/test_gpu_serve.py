"""The request loop (odc_submit / odc_poll): every request's mesh equals the
one odc_extract produces alone, byte for byte, whatever runs beside it; the
memory budget admits requests in arrival order."""
import numpy as np
import pytest

from paper_2409_13418_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2409_13418_gb300 import build, odc
    build.build()
    return odc


def _mix():
    lat_net = I.envelope_mlp(7, latent_dim=128)
    return [
        (I.config1_csg(), I.cube_grid(32), dict(steps_1d=10)),
        (I.random_csg(2, n_prims=64), I.cube_grid(64), dict(steps_1d=12)),
        (I.envelope_mlp(0), I.cube_grid(48), dict(steps_1d=15, precision=1)),
        (I.with_latent(lat_net, 1), I.cube_grid(40), dict(steps_1d=15, precision=1)),
        (I.with_latent(lat_net, 2), I.cube_grid(40), dict(steps_1d=15, precision=1)),
        (I.envelope_mlp(3), I.Grid((-0.8, -0.9, -0.7), (0.7, 0.8, 0.75), (29, 37, 31)), dict(steps_1d=12, precision=0)),
        (I.with_latent(lat_net, 1), I.cube_grid(40), dict(steps_1d=15, precision=1)),
    ]


def _alone(lib, jobs):
    out = []
    with lib.Context(0) as ctx:
        for src, g, kw in jobs:
            out.append(ctx.extract(src, g, **kw).to_host())
    return out


@pytest.mark.parametrize("slots", [1, 3])
def test_each_result_equals_the_request_alone(lib, slots):
    jobs = _mix()
    ref = _alone(lib, jobs)
    with lib.Server(0, slots=slots) as srv:
        ids = [srv.submit(src, g, **kw) for src, g, kw in jobs]
        res = [srv.poll(i) for i in ids]
        for r in res:
            assert r["status"] == 0, r.get("error")
        for (v, t), r in zip(ref, res):
            assert np.array_equal(r["verts"], v) and np.array_equal(r["tris"], t)
        if slots > 1:
            assert len({r["slot"] for r in res}) > 1
        for i in ids:
            srv.release(i)


def test_budget_admits_in_arrival_order_one_at_a_time(lib):
    jobs = _mix()[:4]
    with lib.Server(0, slots=3) as probe:
        est = []
        for src, g, kw in jobs:
            i = probe.submit(src, g, **kw)
            est.append(probe.poll(i)["est_bytes"])
            probe.release(i)
    budget = int(max(est) * 1.5)           # never two requests at once
    with lib.Server(0, slots=3, mem_budget=budget, host_copy=False) as srv:
        ids = [srv.submit(src, g, **kw) for src, g, kw in jobs]
        res = [srv.poll(i) for i in ids]
        for i in ids:
            srv.release(i)
    for r in res:
        assert r["status"] == 0
    spans = sorted((r["t_start"], r["t_end"]) for r in res)
    starts = [r["t_start"] for r in res]
    assert starts == sorted(starts)        # arrival order
    for (a0, a1), (b0, b1) in zip(spans, spans[1:]):
        assert b0 >= a1                    # no overlap under the budget


def test_poll_timeout_errors_and_release(lib):
    with lib.Server(0, slots=1) as srv:
        big = srv.submit(I.envelope_mlp(0), I.cube_grid(160), precision=0)
        small = srv.submit(I.config1_csg(), I.cube_grid(32), steps_1d=10)
        assert srv.poll(small, timeout_ms=0) is None          # queued behind the big one
        with pytest.raises(lib.OdcError):
            srv.release(small)                                 # not finished
        with pytest.raises(lib.OdcError):
            srv.poll(123456)                                   # unknown id
        with pytest.raises(lib.OdcError):
            srv.submit(None, I.cube_grid(8))                   # resident sources are per context
        with pytest.raises(lib.OdcError):
            srv.submit(I.config1_csg(), I.Grid((1, 1, 1), (0, 0, 0), (8, 8, 8)))
        r = srv.poll(small)
        assert r["status"] == 0 and r["t_start"] >= srv.poll(big)["t_end"]
        srv.release(small)
        srv.release(big)
        with pytest.raises(lib.OdcError):
            srv.poll(small)
