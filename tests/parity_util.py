"""Helpers comparing the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: masks, configurations, cycles, flips, quads and
triangles bit-exact; 1D results T bit-exact (both sides query the same float32
points and decide the exact predicate); 2D points and 3D points within 1e-4
cell.  Elements whose oracle decision margin is below ``margin_eps`` or whose
oracle geometry sits at a threshold (parallel lines, degenerate normals,
eigenvalue truncation, zero concavity determinant) are *flagged*: they are
counted and must stay rare, and they are excluded from the strict checks.
"""
from __future__ import annotations

import numpy as np

VERT_TOL = 1e-4   # cell units (h)


def unpack_labels(words: np.ndarray, res) -> np.ndarray:
    nv = [r + 1 for r in res]
    W = (nv[0] + 31) // 32
    w = words.reshape(nv[2], nv[1], W)
    bits = np.unpackbits(w.view(np.uint8).reshape(nv[2], nv[1], W * 4), axis=2, bitorder="little")
    return bits[:, :, :nv[0]].astype(bool)


def unpack_cycles(c: np.ndarray) -> np.ndarray:
    out = np.zeros((c.shape[0], 12), np.int8)
    for le in range(12):
        v = ((c >> np.uint64(4 * le)) & np.uint64(0xF)).astype(np.int8)
        out[:, le] = np.where(v == 15, -1, v)
    return out


def compare(ctx, mesh, ref, margin_eps=1e-12):
    """Compare the last extract on ``ctx`` with oracle result ``ref``; returns a report."""
    rep = {}
    res = ref.res
    lab = unpack_labels(ctx.debug("labels"), res)
    assert np.array_equal(lab, ref.labels), "grid labels differ"
    edges = ctx.debug("edges").astype(np.int64)
    assert np.array_equal(edges, ref.edges), "crossing edge lists differ"
    faces = ctx.debug("faces").astype(np.int64)
    slots = ctx.debug("slots").astype(np.int64)
    assert np.array_equal(faces, ref.faces[:, 0]) and np.array_equal(slots, ref.faces[:, 1]), "face lists differ"
    cells = ctx.debug("cells").astype(np.int64)
    assert np.array_equal(cells, ref.cells), "crossing cell lists differ"
    assert np.array_equal(ctx.debug("configs"), ref.configs), "cell configurations differ"
    flips = ctx.debug("flips").astype(np.int64)
    assert np.array_equal(flips, ref.flips), "manifold-fix flips differ"
    cyc = unpack_cycles(ctx.debug("cycles"))
    assert np.array_equal(cyc, ref.cell_cyc), "cell cycles differ"

    # 1D points: exact integers unless the oracle flags a near-tie decision
    T = ctx.debug("T").astype(np.int64)
    eflag = ref.edge_margin < margin_eps
    rep["edge_flagged"] = int(eflag.sum())
    bad = (T != ref.T) & ~eflag
    assert not bad.any(), f"{int(bad.sum())} unflagged 1D results differ"

    # 2D points
    pf = ctx.face_points()
    fflag = (ref.face_margin < margin_eps) | ((ref.face_flags & 4) != 0)
    rep["face_flagged"] = int(fflag.sum())
    gflags = ctx.debug("face_flags").astype(np.int64)
    assert np.array_equal(gflags[~fflag] & 3, ref.face_flags[~fflag] & 3), "2D search branch (q == m / parallel) differs"
    d = np.linalg.norm(pf - ref.face_pts, axis=1) / np.maximum(1.0, np.linalg.norm(ref.face_pts, axis=1))
    rep["face_max_err"] = float(d[~fflag].max()) if (~fflag).any() else 0.0
    assert rep["face_max_err"] < 1e-5, f"2D points differ by {rep['face_max_err']}"

    # 3D points
    vl = ctx.debug("vlocal").astype(np.float64)
    assert vl.shape == ref.verts_local.shape
    vflag = (ref.vert_margin < margin_eps) | ref.vert_flag
    rep["vert_flagged"] = int(vflag.sum())
    dv = np.abs(vl - ref.verts_local).max(axis=1)
    rep["vert_max_err"] = float(dv[~vflag].max()) if (~vflag).any() else 0.0
    assert rep["vert_max_err"] < VERT_TOL, f"3D points differ by {rep['vert_max_err']} cell"
    rep["vert_flagged_max_err"] = float(dv[vflag].max()) if vflag.any() else 0.0
    # flagged vertices: rare and still close (their inputs sit at a decision tie)
    assert rep["vert_flagged"] <= max(2, 0.01 * len(vflag)), f"{rep['vert_flagged']} flagged vertices"
    assert rep["vert_flagged_max_err"] < 1e-2, f"flagged 3D points differ by {rep['vert_flagged_max_err']} cell"

    # quads and triangles
    qcase = ctx.debug("qcase").astype(np.int64)
    ref_case = np.zeros(len(ref.edges), np.int64)
    ref_case[ref.quad_edges] = ref.quad_case
    qflag = np.zeros(len(ref.edges), bool)
    qflag[ref.quad_edges] = ref.quad_flag | (ref.quad_margin < margin_eps)
    rep["quad_flagged"] = int(qflag.sum())
    assert np.array_equal(qcase[~qflag], ref_case[~qflag]), "quad split cases differ"
    rep["quad_flagged_differ"] = int(np.sum(qcase[qflag] != ref_case[qflag]))
    verts, tris = mesh.to_host()
    if np.array_equal(qcase, ref_case):
        # every split case agrees, so the triangle lists must agree bit for bit
        assert np.array_equal(tris.astype(np.int64), ref.triangles), "triangles differ"
        assert verts.shape == ref.vertices.shape
    rep["n_verts"] = int(verts.shape[0])
    rep["n_tris"] = int(tris.shape[0])
    return rep, verts, tris
