"""GPU-vs-oracle parity of the MLP occupancy path, by decision replay.

Every ODC search ends next to the iso-surface, so its last decisions sit
where the FP32 network (GPU) and the FP64 network (oracle) can legitimately
disagree: the measured FP32 logit error is below 7e-6 (test below), while the
logits at the final bisection steps are ~1e-4.  The comparison therefore
splits what is unique from what is a valid choice:

  * grid labels, crossing lists, configurations, flips, cycles: bit-exact;
  * every search decision the GPU took (1D results T, 2D line-binary
    results, labels of m) is replayed through the oracle and checked against
    its FP64 label wherever the FP64 margin |occ - 0.5| >= MARGIN (2e-5, i.e.
    |z| >= 8e-5, an order of magnitude above the FP32 error): no violation;
  * given those decisions, everything downstream (2D points, normals, QEF 3D
    points, quad splits, triangles) is unique: 2D points within 1e-5, 3D
    points within 1e-4 cell, split cases and triangles bit-exact.
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
    assert err.max() < 2e-5
    sure = np.abs(zr) > 2e-5
    assert np.array_equal(lab[sure], (zr > 0)[sure])


def replay_parity(ctx, src, grid, k, precision=0, band=None, **search):
    mesh = ctx.extract(src, grid, steps_1d=k, precision=precision, band=band, **search)
    T = ctx.debug("T").astype(np.int64)
    dec = ctx.search_decisions()
    ref = oracle.extract(src, grid, steps_1d=k, replay=dict(T=T, **dec), replay_margin=MARGIN, **search)
    assert ref.stats["edge_violations"] == 0, ref.stats
    assert ref.stats["face_violations"] == 0, ref.stats
    rep, verts, tris = compare(ctx, mesh, ref, margin_eps=0.0)
    own = oracle.extract(src, grid, steps_1d=k, **search)
    # Decisions the GPU took differently from the FP64 network's own choice:
    # each one sits inside the replay band (the replay above found no
    # violation), and they must stay a small minority of the searches.
    assert own.T.shape == T.shape and own.faces.shape == ref.faces.shape
    rep["T_choices_differing_from_fp64"] = int(np.sum(own.T != T))
    face_diff = np.zeros(len(own.faces), bool)
    for key in ("Jq", "J1", "J2", "lab_m"):
        face_diff |= np.asarray(own.search[key]).astype(np.int64) != np.asarray(dec[key]).astype(np.int64)
    rep["face_choices_differing_from_fp64"] = int(face_diff.sum())
    print("decisions differing from the FP64 network's own:", rep["T_choices_differing_from_fp64"], "of", len(T),
          "edges;", rep["face_choices_differing_from_fp64"], "of", len(face_diff), "faces;",
          own.stats["queries"], "decisions")
    # a search that differs differs in at least one decision: at most 1% of all
    # decisions (measured <= 0.1%), and per search at most 2% of the 1D
    # searches (measured <= 0.9%) and 8% of the 2D ones (measured <= 4.1%)
    n_diff = rep["T_choices_differing_from_fp64"] + rep["face_choices_differing_from_fp64"]
    assert n_diff <= max(2, 0.01 * own.stats["queries"]), rep
    assert rep["T_choices_differing_from_fp64"] <= max(2, 0.02 * len(T)), rep
    assert rep["face_choices_differing_from_fp64"] <= max(2, 0.08 * len(face_diff)), rep
    return mesh, ref, rep, verts, tris


@pytest.mark.parametrize("n", [24, 40])
def test_fp32_extract_replay_parity(ctx, mlp, n):
    mesh, ref, rep, verts, tris = replay_parity(ctx, mlp, I.cube_grid(n), 15)
    print(n, rep, ref.stats, mesh.stats)
    assert rep["vert_max_err"] < 1e-4
    assert meshcheck.check_closed_manifold(tris)["ok"]


def test_ragged_grid_replay_parity(ctx, mlp):
    g = I.Grid((-0.71, -0.8, -0.66), (0.69, 0.75, 0.7), (37, 29, 33))
    mesh, ref, rep, verts, tris = replay_parity(ctx, mlp, g, 12)
    assert rep["vert_max_err"] < 1e-4


def test_resident_source_gives_same_mesh(ctx, mlp):
    g = I.cube_grid(32)
    v1, t1 = ctx.extract(mlp, g, steps_1d=12).to_host()
    ctx.upload(mlp)
    v2, t2 = ctx.extract(None, g, steps_1d=12).to_host()
    assert np.array_equal(t1, t2) and np.array_equal(v1, v2)


def test_csg_replay_parity_agrees_with_direct(ctx):
    # the replay check also holds on the exact CSG path (no decision differs)
    src = I.random_csg(3, n_prims=24)
    mesh, ref, rep, verts, tris = replay_parity(ctx, src, I.cube_grid(48), 12)
    assert rep["T_choices_differing_from_fp64"] == 0


BF16_BAND = 0.03   # |occ - 0.5| (|z| < 0.12): twice the largest BF16 logit error seen (0.063)


def test_bf16_logits_within_band_of_fp32(ctx, mlp):
    rng = np.random.default_rng(2)
    pts = rng.uniform(-1, 1, (300000, 3)).astype(np.float32)
    _, z32 = ctx.eval_points(mlp, pts, precision=0)
    _, z16 = ctx.eval_points(mlp, pts, precision=1, band=0.0)    # raw tensor-core logits
    d = np.abs(z16.astype(np.float64) - z32)
    zb = 2 * np.arctanh(2 * BF16_BAND)
    print("bf16 |dz| max", d.max(), "median", np.median(d), "band |z|", zb)
    assert np.isfinite(z16).all()
    assert d.max() < 0.6 * zb
    # with the band, every label equals the FP32 plain path's
    l16, _ = ctx.eval_points(mlp, pts, precision=1, band=BF16_BAND)
    l32, _ = ctx.eval_points(mlp, pts, precision=0)
    assert np.array_equal(l16, l32)


F16_ZMARGIN = 0.025   # logit margin of the FP16 tier (library constant; measured max error 0.0091)


def test_f16_tier_logits_within_half_its_margin_of_fp32(ctx, mlp):
    """The single-product FP16 tier (FP16 activations, FP16 weights w 2^s,
    FP32 accumulation) stays within half its logit margin (0.025) of the
    FP32 network, uniformly over the box and on the surface shell where the
    searches query it."""
    from paper_2409_13418_gb300 import odc
    rng = np.random.default_rng(6)
    u = rng.normal(size=(500000, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    shell = u * rng.uniform(0.3, 0.7, (500000, 1))
    pts = np.concatenate([rng.uniform(-1, 1, (500000, 3)), shell]).astype(np.float32)
    _, z32 = ctx.eval_points(mlp, pts, precision=0)
    _, zh = ctx.eval_points(mlp, pts, precision=odc.PREC_F16)
    d = np.abs(zh.astype(np.float64) - z32)
    print("fp16 tier |dz| max", d.max(), "median", np.median(d))
    assert np.isfinite(zh).all()
    assert d.max() < 0.5 * F16_ZMARGIN


def test_split_bf16_logits_within_margin_of_fp32(ctx, mlp):
    """The split tier (FP16 hi + lo operands, three products per layer,
    corrections in their own accumulator, its round-toward-zero accumulation
    compensated by the calibrated factor) stays within 0.65 of the network's
    calibrated re-decision margin (1.9e-5 here) of the FP32 network,
    uniformly over the box (measured largest error 9.5e-6 on 2 M points,
    mean within 1e-7 of zero; without the compensation 1.29e-5 with a mean
    of -9.6e-7)."""
    margin = _split_margin(ctx, mlp)
    rng = np.random.default_rng(4)
    pts = rng.uniform(-1, 1, (1000000, 3)).astype(np.float32)
    _, z32 = ctx.eval_points(mlp, pts, precision=0)
    _, zs = ctx.eval_points(mlp, pts, precision=2)
    d = np.abs(zs.astype(np.float64) - z32)
    print("split |dz| max", d.max(), "median", np.median(d), "margin", margin)
    assert np.isfinite(zs).all()
    assert 1.2e-5 <= margin <= 3e-5
    assert d.max() < 0.65 * margin
    # the compensation removes the accumulation's bias
    assert abs(float(np.mean(zs.astype(np.float64) - z32))) < 2e-7


def _split_margin(ctx, src):
    """The split tier's margin the library calibrated for ``src``."""
    from paper_2409_13418_gb300 import odc
    m = ctx.extract(src, I.cube_grid(12), steps_1d=8, precision=odc.PREC_BF16)
    return float(m.stats["split_zmargin"])


@pytest.mark.parametrize("seed,latent", [(1, 0), (2, 0), (7, 128), (11, 128)])
def test_split_margin_holds_on_other_networks(ctx, seed, latent):
    """The split tier's margin holds on other networks of the same
    architecture, with and without a latent code folded into the first
    layer, each with its own calibrated accumulation compensation and
    margin: largest error within 0.7 of that margin (over eight networks the
    largest error on 3 M points was 9.5e-6 to 1.34e-5, and 1.14e-5 to
    1.72e-5 uncompensated) and a mean within 6e-7 of zero (measured within
    2.2e-7 on six of them, -5.5e-7 and -7.2e-7 on two latent codes of one
    network; uncompensated up to 4.2e-6), uniformly over the box and on the
    surface shell."""
    src = I.envelope_mlp(seed, latent_dim=latent)
    margin = _split_margin(ctx, src)
    rng = np.random.default_rng(100 + seed)
    u = rng.normal(size=(300000, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    pts = np.concatenate([rng.uniform(-1, 1, (300000, 3)), u * rng.uniform(0.3, 0.7, (300000, 1))]).astype(np.float32)
    _, z32 = ctx.eval_points(src, pts, precision=0)
    _, zs = ctx.eval_points(src, pts, precision=2)
    d = zs.astype(np.float64) - z32
    print("seed", seed, "latent", latent, "split |dz| max", np.abs(d).max(), "mean", d.mean(), "margin", margin)
    assert np.isfinite(zs).all()
    assert np.abs(d).max() < 0.7 * margin
    assert abs(float(d.mean())) < 6e-7


def test_split_acc_comp_sets_the_bias(ctx, mlp):
    """Without the compensation the split tier's logits sit below the FP32
    network's on average for this network (its accumulation rounds toward
    zero and its output is mostly positive here); the calibrated default
    centres them; an excess compensation moves them above; a value of 1e-3
    or more is refused."""
    from paper_2409_13418_gb300 import odc
    rng = np.random.default_rng(9)
    pts = rng.uniform(-1, 1, (300000, 3)).astype(np.float32)
    _, z32 = ctx.eval_points(mlp, pts, precision=0)
    mean = {}
    for c in (-1.0, 0.0, 6e-7):
        _, zs = ctx.eval_points(mlp, pts, precision=2, split_acc_comp=c)
        mean[c] = float(np.mean(zs.astype(np.float64) - z32))
    print("split mean error by compensation", mean)
    assert mean[-1.0] < -5e-7 and abs(mean[0.0]) < 2e-7 and mean[6e-7] > 5e-7
    with pytest.raises(odc.OdcError):
        ctx.eval_points(mlp, pts[:10], precision=2, split_acc_comp=1e-3)


@pytest.mark.parametrize("n,split,h16", [(48, True, True), (97, True, True), (64, False, True), (131, True, True),
                                         (131, False, True), (64, True, False), (97, False, False)])
def test_bf16_extract_equals_fp32_plain_path(ctx, mlp, n, split, h16):
    """BF16 tensor cores + tiered re-evaluation in the band (FP16 tier,
    split-FP16 tier, then FP32; with either middle tier switched off):
    every decision, and hence the whole mesh, equals the FP32 plain path's,
    byte for byte."""
    g = I.cube_grid(n)
    m32 = ctx.extract(mlp, g, steps_1d=15, precision=0)
    v32, t32 = m32.to_host()
    T32, d32 = ctx.debug("T"), ctx.search_decisions()
    m16 = ctx.extract(mlp, g, steps_1d=15, precision=1, band=BF16_BAND, split=split, h16=h16)
    v16, t16 = m16.to_host()
    assert np.array_equal(ctx.debug("T"), T32)
    d16 = ctx.search_decisions()
    for k in d32:
        assert np.array_equal(d16[k], d32[k]), k
    assert np.array_equal(t16, t32) and np.array_equal(v16, v32)
    assert m16.stats["n_requeries"] > 0
    assert (m16.stats["n_h16"] > 0) == h16 and (m16.stats["n_split"] > 0) == split


@pytest.mark.parametrize("iso", [0.3, 0.7])
def test_bf16_extract_equals_fp32_plain_path_off_half_iso(ctx, mlp, iso):
    """The band and the split margin are measured from logit(iso), not from 0."""
    g = I.cube_grid(56)
    v32, t32 = ctx.extract(mlp, g, steps_1d=15, precision=0, iso=iso).to_host()
    T32, d32 = ctx.debug("T"), ctx.search_decisions()
    m16 = ctx.extract(mlp, g, steps_1d=15, precision=1, band=BF16_BAND, iso=iso)
    v16, t16 = m16.to_host()
    assert np.array_equal(ctx.debug("T"), T32)
    d16 = ctx.search_decisions()
    for k in d32:
        assert np.array_equal(d16[k], d32[k]), k
    assert np.array_equal(t16, t32) and np.array_equal(v16, v32)
    rng = np.random.default_rng(5)
    pts = rng.uniform(-1, 1, (200000, 3)).astype(np.float32)
    l16, _ = ctx.eval_points(mlp, pts, iso=iso, precision=1, band=BF16_BAND)
    l32, _ = ctx.eval_points(mlp, pts, iso=iso, precision=0)
    assert np.array_equal(l16, l32)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("search", [dict(lin1=1, bin1=6, lin2=1, bin2=7),
                                    dict(lin1=7, bin1=8, lin2=6, bin2=9, range1=1.5, range2=1.2)])
def test_line_search_settings_replay_parity(ctx, mlp, precision, search):
    """Non-default line-binary searches (one line sample, or many samples
    over a longer range, where the line phase runs several early-exit rounds
    and can end without a crossing) match the oracle's by decision replay."""
    band = BF16_BAND if precision == 1 else None
    mesh, ref, rep, verts, tris = replay_parity(ctx, mlp, I.cube_grid(24), 12, precision=precision, band=band,
                                                **search)
    print(search, rep)
    assert rep["n_tris"] > 0


def test_bf16_extract_replay_parity(ctx, mlp):
    mesh, ref, rep, verts, tris = replay_parity(ctx, mlp, I.cube_grid(32), 15, precision=1, band=BF16_BAND)
    assert rep["vert_max_err"] < 1e-4


def test_fp32_tile_shapes_give_identical_bits(ctx, mlp):
    """The autotuner may pick any of the FP32 network's tile shapes: all give
    the same logits bit for bit (same FMA order per output), and the pick is
    one of them."""
    rng = np.random.default_rng(7)
    for npts in (3000, 50000):   # 3000: the 16-warp shapes take their small-list path (32-query tiles)
        pts = rng.uniform(-1, 1, (npts, 3)).astype(np.float32)
        ref = None
        for v in range(4):
            _, z = ctx.eval_points(mlp, pts, precision=0, fp32_tile=v)
            if ref is None:
                ref = z
            assert z.tobytes() == ref.tobytes(), (npts, v)
    _, z = ctx.eval_points(mlp, pts, precision=0)
    assert z.tobytes() == ref.tobytes()
    m = ctx.extract(mlp, I.cube_grid(24), steps_1d=10, precision=0)
    assert m.stats["fp32_tile"] in range(4)
    print("autotuned FP32 tile shape", m.stats["fp32_tile"])


FP8_ZBAND = 2.5   # logit band of the FP8 pass (library constant; largest measured error 1.19)


def test_fp8_logits_within_band_of_fp32(ctx, mlp):
    """The FP8 pass (E4M3 activations and weights, FP32 accumulation) stays
    within 0.6 of its logit band (2.0) of the FP32 network, uniformly over
    the box and on the surface shell."""
    from paper_2409_13418_gb300 import odc
    rng = np.random.default_rng(8)
    u = rng.normal(size=(300000, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    pts = np.concatenate([rng.uniform(-1, 1, (300000, 3)), u * rng.uniform(0.3, 0.7, (300000, 1))]).astype(np.float32)
    _, z32 = ctx.eval_points(mlp, pts, precision=0)
    _, z8 = ctx.eval_points(mlp, pts, precision=odc.PREC_FP8_RAW)
    d = np.abs(z8.astype(np.float64) - z32)
    print("fp8 |dz| max", d.max(), "median", np.median(d), "p99.9", np.quantile(d, 0.999))
    assert np.isfinite(z8).all()
    assert d.max() < 0.6 * FP8_ZBAND


@pytest.mark.parametrize("n", [48, 97])
def test_fp8_extract_equals_fp32_plain_path(ctx, mlp, n):
    """FP8 pass + BF16 pass + FP16, split and FP32 tiers: every decision and
    the whole mesh equal the FP32 plain path's, byte for byte."""
    from paper_2409_13418_gb300 import odc
    g = I.cube_grid(n)
    v32, t32 = ctx.extract(mlp, g, steps_1d=15, precision=0).to_host()
    T32, d32 = ctx.debug("T"), ctx.search_decisions()
    m8 = ctx.extract(mlp, g, steps_1d=15, precision=odc.PREC_FP8, band=BF16_BAND)
    v8, t8 = m8.to_host()
    assert np.array_equal(ctx.debug("T"), T32)
    d8 = ctx.search_decisions()
    for k in d32:
        assert np.array_equal(d8[k], d32[k]), k
    assert np.array_equal(t8, t32) and np.array_equal(v8, v32)
    assert m8.stats["fp8_launches"] > 0 and m8.stats["fp8_flops"] > 0


def test_fp8_latent_mlp_equals_fp32_plain_path(ctx):
    from paper_2409_13418_gb300 import odc
    src = I.with_latent(I.envelope_mlp(12, latent_dim=128), 2003)
    g = I.cube_grid(72)
    v32, t32 = ctx.extract(src, g, steps_1d=15, precision=0).to_host()
    v8, t8 = ctx.extract(src, g, steps_1d=15, precision=odc.PREC_FP8, band=BF16_BAND).to_host()
    assert np.array_equal(t8, t32) and np.array_equal(v8, v32)


def test_fp8_saturated_rows_are_handed_on(ctx):
    """A network whose hidden activations exceed the FP8 range (first
    hidden layer scaled up 40x): the FP8 pass marks those rows (their raw
    logit is the threshold itself, so the next tier must take them), and the
    tiered result still equals the FP32 plain path's."""
    from paper_2409_13418_gb300 import odc
    base = I.envelope_mlp(0)
    W = [w.copy() for w in base.weights]
    W[1] = (W[1] * 40.0).astype(np.float32)
    W[2] = (W[2] / 40.0).astype(np.float32)
    src = I.MLPSource(B=base.B, weights=W, biases=base.biases, env_scale=base.env_scale,
                      env_radius=base.env_radius, env_amp=base.env_amp, name="fp8-saturating")
    rng = np.random.default_rng(9)
    pts = rng.uniform(-1, 1, (100000, 3)).astype(np.float32)
    _, z8 = ctx.eval_points(src, pts, precision=odc.PREC_FP8_RAW)
    marked = z8 == 0.0
    print("rows handed on", int(marked.sum()))
    assert marked.sum() > 100
    l32, _ = ctx.eval_points(src, pts, precision=0)
    l8, _ = ctx.eval_points(src, pts, precision=odc.PREC_FP8, band=BF16_BAND)
    assert np.array_equal(l8, l32)
    g = I.cube_grid(40)
    v32, t32 = ctx.extract(src, g, steps_1d=12, precision=0).to_host()
    v8, t8 = ctx.extract(src, g, steps_1d=12, precision=odc.PREC_FP8, band=BF16_BAND).to_host()
    assert np.array_equal(t8, t32) and np.array_equal(v8, v32)


def test_split_calibration_is_deterministic(mlp):
    """The calibrated compensation is a function of the weights alone: two
    contexts, and a forced re-upload of the same weights, give the split
    tier the same logits bit for bit, and so the same tiered mesh."""
    from paper_2409_13418_gb300 import odc
    rng = np.random.default_rng(12)
    pts = rng.uniform(-1, 1, (200000, 3)).astype(np.float32)
    g = I.cube_grid(40)
    out = []
    for reupload in (False, True):
        with odc.Context(0) as c:
            _, zs = c.eval_points(mlp, pts, precision=2)
            v, t = c.extract(mlp, g, steps_1d=15, precision=odc.PREC_BF16, reupload=reupload).to_host()
            _, zs2 = c.eval_points(mlp, pts, precision=2)
            out.append((zs, zs2, v, t))
    (a, a2, va, ta), (b, b2, vb, tb) = out
    assert a.tobytes() == a2.tobytes() == b.tobytes() == b2.tobytes()
    assert va.tobytes() == vb.tobytes() and np.array_equal(ta, tb)
