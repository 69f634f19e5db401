"""Windowed oracle parity: the oracle on a block of a large grid, compared on its core.

ODC is local.  A grid label is one occupancy query; a 1D point depends on
its edge, a 2D point on its face segment (the face's labels, the segment's
two 1D points and the queries of its line-binary searches), a 3D point on
its cell's cycles, 1D and 2D points (Eq. 2), and a crossing edge's
triangles on its four cells (A.1.5).  The one non-local step is the manifold
fix, which iterates over ambiguous faces until nothing changes, so a flip
can in principle chain from cell to cell.

So the oracle, too slow for a whole 256^3 grid, runs on a block of n^3 cells
starting at cell w: the sub-grid [x_w, x_{w+n}] with n cells per axis.  On
the dyadic cube grids used here its FP32 coordinates equal the full grid's
(checked).  The search decisions of the full-size result are replayed through
the oracle (each one checked against the FP64 label wherever the FP64 margin
is at least ``margin``), and the block's core -- cells at least ``core`` cells
inside the block, faces and edges all of whose cells are core cells -- is
compared element by element: labels, crossing lists and configurations
exactly, flips, cycles, 2D branch flags, quad cases and triangles exactly,
2D points within 1e-5 and 3D points within 1e-4 cell.

The full-size result is a plain dict of arrays (``full_from_oracle`` builds
it from a whole-grid oracle run, which pins the windowing itself on the CPU;
the GPU tests build it from the library's debug copies).
"""
from __future__ import annotations

import numpy as np

from oracle import odc as oracle
from oracle.occupancy import Occupancy
from paper_2409_13418_gb300 import inputs as I

VERT_TOL = 1e-4      # 3D points, cell units
FACE_TOL = 1e-5      # 2D points, relative to max(1, |p_f|)


def full_from_oracle(r) -> dict:
    """The full-size result dict of a whole-grid oracle run."""
    qcase = np.zeros(len(r.edges), np.int64)
    qcase[r.quad_edges] = r.quad_case
    return dict(res=tuple(int(x) for x in r.res), labels=r.labels, edges=r.edges.astype(np.int64),
                T=r.T.astype(np.int64), faces=r.faces[:, 0].astype(np.int64), slots=r.faces[:, 1].astype(np.int64),
                dec={k: np.asarray(v) for k, v in r.search.items()}, face_pts=r.face_pts,
                face_flags=r.face_flags.astype(np.int64), flips=r.flips.astype(np.int64),
                cells=r.cells.astype(np.int64), configs=r.configs.astype(np.int64),
                cyc=r.cell_cyc.astype(np.int64), vlocal=r.verts_local,
                qcase=qcase, tris=r.triangles.astype(np.int64))


def _vijk(v, nv):
    i = v % nv[0]
    t = v // nv[0]
    return np.stack([i, t % nv[1], t // nv[1]], axis=1)


def _vid(ijk, nv):
    return ijk[:, 0] + nv[0] * (ijk[:, 1] + nv[1] * ijk[:, 2])


def _vertex_keys(cells_g, cyc, case3_edges_g):
    """Key per output vertex: 16 * global cell id + cycle for 3D points,
    -(global edge id + 1) for the 1D points that case-3 splits add."""
    ncyc = (cyc.max(axis=1) + 1).astype(np.int64) if len(cells_g) else np.zeros(0, np.int64)
    first = np.repeat(np.cumsum(ncyc) - ncyc, ncyc)
    within = np.arange(int(ncyc.sum())) - first
    return np.concatenate([np.repeat(cells_g, ncyc) * 16 + within, -(case3_edges_g + 1)]), ncyc


def _tri_offsets(case):
    cnt = np.where(case == 0, 0, np.where(case == 3, 4, 2))
    return np.cumsum(cnt) - cnt, cnt


def window_parity(src, full: dict, grid, w, n: int, steps_1d: int, margin: float, core: int = 2):
    """Compare the full-size result with the oracle on the block of n^3 cells at ``w``.

    Returns a report dict, or None when a grid label in the block sits at a
    decision tie (FP64 margin below ``margin``) and differs: both labels are
    then valid and the block's crossing lists legitimately differ.
    """
    N = full["res"]
    NV = tuple(x + 1 for x in N)
    w = np.asarray(w, np.int64)
    assert all(0 <= w[a] and w[a] + n <= N[a] for a in range(3))
    X = oracle.grid_coords(grid)
    wg = I.Grid(tuple(float(X[a][w[a]]) for a in range(3)), tuple(float(X[a][w[a] + n]) for a in range(3)), (n, n, n))
    Xw = oracle.grid_coords(wg)
    for a in range(3):
        assert np.array_equal(Xw[a], X[a][w[a]:w[a] + n + 1]), "block coordinates differ from the grid's"
    nvw = (n + 1,) * 3
    rep = dict(origin=tuple(int(x) for x in w), n=n)

    # grid labels of the block
    zz, yy, xx = np.meshgrid(Xw[2], Xw[1], Xw[0], indexing="ij")
    lab, mar = Occupancy(src, 0.5)(np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1))
    lab = lab.reshape(n + 1, n + 1, n + 1)
    mar = mar.reshape(n + 1, n + 1, n + 1)
    flab = full["labels"][w[2]:w[2] + n + 1, w[1]:w[1] + n + 1, w[0]:w[0] + n + 1]
    diff = lab != flab
    assert not np.any(diff & (mar >= margin)), "grid labels differ where the FP64 margin is clear"
    if diff.any():
        return None

    # crossing edges inside the block, in block ids (same (k, j, i, axis) order)
    ev, ea = full["edges"] // 3, full["edges"] % 3
    eijk = _vijk(ev, NV) - w
    hi = n - np.eye(3, dtype=np.int64)[ea]
    ein = np.all((eijk >= 0) & (eijk <= hi), axis=1)
    e_idx = np.nonzero(ein)[0]
    e_w = 3 * _vid(eijk[ein], nvw) + ea[ein]
    o = np.argsort(e_w, kind="stable")
    e_idx, e_w = e_idx[o], e_w[o]

    # crossing face segments inside the block
    fv, fa = full["faces"] // 3, full["faces"] % 3
    fijk = _vijk(fv, NV) - w
    fhi = n - 1 + np.eye(3, dtype=np.int64)[fa]
    fin = np.all((fijk >= 0) & (fijk <= fhi), axis=1)
    f_idx = np.nonzero(fin)[0]
    f_w = 3 * _vid(fijk[fin], nvw) + fa[fin]
    fkey = 2 * f_w + full["slots"][fin]
    o = np.argsort(fkey, kind="stable")
    f_idx, f_w, fkey = f_idx[o], f_w[o], fkey[o]

    replay = dict(T=full["T"][e_idx], **{k: v[f_idx] for k, v in full["dec"].items()})
    r = oracle.extract(src, wg, steps_1d=steps_1d, replay=replay, replay_margin=margin)
    assert np.array_equal(r.edges, e_w), "crossing edge lists differ"
    assert np.array_equal(2 * r.faces[:, 0] + r.faces[:, 1], fkey), "crossing face lists differ"
    assert not r.violations["edges"].any(), f"{int(r.violations['edges'].sum())} 1D decisions contradict FP64"
    rep["E"], rep["F"] = int(len(e_w)), int(len(f_w))

    # cells: the block's crossing cells are exactly the full list's cells inside it
    ncell = np.asarray(N)
    cijk_full = np.stack([full["cells"] % ncell[0], (full["cells"] // ncell[0]) % ncell[1],
                          full["cells"] // (ncell[0] * ncell[1])], axis=1) - w
    cin = np.all((cijk_full >= 0) & (cijk_full < n), axis=1)
    c_idx = np.nonzero(cin)[0]
    c_w = cijk_full[cin, 0] + n * (cijk_full[cin, 1] + n * cijk_full[cin, 2])
    assert np.array_equal(r.cells, c_w), "crossing cell lists differ"
    rc = np.stack([r.cells % n, (r.cells // n) % n, r.cells // (n * n)], axis=1)
    assert np.array_equal(r.configs.astype(np.int64), full["configs"][c_idx].astype(np.int64)), "cell configurations differ"

    def is_core_cell(ijk):
        return np.all((ijk >= core) & (ijk < n - core), axis=1)

    ccore = is_core_cell(rc)
    rep["core_cells"] = int(ccore.sum())

    # flips and face segments on core faces (both cells of the face are core cells)
    EYE = np.eye(3, dtype=np.int64)

    def core_face(fid_w):
        v, a = fid_w // 3, fid_w % 3
        b = _vijk(v, nvw)
        return is_core_cell(b) & is_core_cell(b - EYE[a])

    fl_full = full["flips"]
    flv = _vijk(fl_full // 3, NV) - w
    fl_in = np.all((flv >= 0) & (flv <= n - 1 + EYE[fl_full % 3]), axis=1)
    fl_full_w = 3 * _vid(flv[fl_in], nvw) + (fl_full % 3)[fl_in]
    fl_full_w = fl_full_w[core_face(fl_full_w)]
    fl_ref = r.flips[core_face(r.flips)] if len(r.flips) else r.flips
    assert np.array_equal(np.sort(fl_full_w), np.sort(fl_ref)), "manifold-fix flips differ on the core"
    rep["core_flips"] = int(len(fl_ref))

    fcore = core_face(r.faces[:, 0])
    fviol = r.violations["faces"] & fcore
    assert not fviol.any(), f"{int(fviol.sum())} 2D decisions on core faces contradict FP64"
    fflag = (r.face_flags & 4) != 0
    sel = fcore & ~fflag
    gf = full["face_flags"][f_idx]
    assert np.array_equal(gf[sel] & 3, r.face_flags[sel] & 3), "2D branch flags differ"
    pf = full["face_pts"][f_idx]
    d = np.linalg.norm(pf - r.face_pts, axis=1) / np.maximum(1.0, np.linalg.norm(r.face_pts, axis=1))
    rep["core_faces"] = int(fcore.sum())
    rep["face_max_err"] = float(d[sel].max()) if sel.any() else 0.0
    assert rep["face_max_err"] < FACE_TOL, f"2D points differ by {rep['face_max_err']}"

    # cycles and 3D points of core cells
    fcyc = full["cyc"][c_idx]
    assert np.array_equal(fcyc[ccore], r.cell_cyc[ccore].astype(np.int64)), "cell cycles differ on the core"
    full_ncyc = (full["cyc"].max(axis=1) + 1).astype(np.int64)
    full_vbase = np.cumsum(full_ncyc) - full_ncyc
    rows_f, rows_r = [], []
    for ci in np.nonzero(ccore)[0]:
        m = int(r.cell_ncyc[ci])
        rows_f.extend(range(full_vbase[c_idx[ci]], full_vbase[c_idx[ci]] + m))
        rows_r.extend(range(r.vbase[ci], r.vbase[ci] + m))
    rows_f, rows_r = np.asarray(rows_f, np.int64), np.asarray(rows_r, np.int64)
    vflag = r.vert_flag[rows_r]
    dv = np.abs(full["vlocal"][rows_f] - r.verts_local[rows_r]).max(axis=1) if len(rows_r) else np.zeros(0)
    rep["core_verts"] = int(len(rows_r))
    rep["vert_flagged"] = int(vflag.sum())
    rep["vert_max_err"] = float(dv[~vflag].max()) if (~vflag).any() else 0.0
    assert rep["vert_max_err"] < VERT_TOL, f"3D points differ by {rep['vert_max_err']} cell"

    # quads and triangles of core edges (all four cells core)
    ra = r.edges % 3
    rijk = _vijk(r.edges // 3, nvw)
    ecore = np.ones(len(r.edges), bool)
    for db in (0, 1):
        for dc in (0, 1):
            cc = rijk - db * EYE[(ra + 1) % 3] - dc * EYE[(ra + 2) % 3]
            ecore &= is_core_cell(cc)
    rcase = np.zeros(len(r.edges), np.int64)
    rcase[r.quad_edges] = r.quad_case
    rflag = np.zeros(len(r.edges), bool)
    rflag[r.quad_edges] = r.quad_flag
    fcase = full["qcase"][e_idx]
    sel = ecore & ~rflag
    assert np.array_equal(fcase[sel], rcase[sel]), "quad split cases differ on the core"
    rep["core_edges"] = int(ecore.sum())
    rep["quad_flagged"] = int((ecore & rflag).sum())

    c3_full = full["edges"][full["qcase"] == 3]
    keys_f, _ = _vertex_keys(full["cells"], full["cyc"], c3_full)
    off_f, cnt_f = _tri_offsets(full["qcase"])
    gcell = lambda cw: (cw % n + w[0]) + N[0] * ((cw // n) % n + w[1] + N[1] * (cw // (n * n) + w[2]))
    r3 = r.edges[r.quad_edges[r.quad_case == 3]]
    r3v = _vijk(r3 // 3, nvw) + w
    r3_g = 3 * _vid(r3v, NV) + r3 % 3
    keys_r, _ = _vertex_keys(gcell(r.cells), r.cell_cyc.astype(np.int64), r3_g)
    off_r, cnt_r = _tri_offsets(rcase)
    same = sel & (fcase == rcase)
    ntri = 0
    for ei in np.nonzero(same)[0]:
        tf = full["tris"][off_f[e_idx[ei]]:off_f[e_idx[ei]] + cnt_f[e_idx[ei]]]
        tr = r.triangles[off_r[ei]:off_r[ei] + cnt_r[ei]]
        assert np.array_equal(keys_f[tf], keys_r[tr]), "triangles differ on the core"
        ntri += len(tr)
    rep["core_tris"] = ntri
    return rep


def block_at(point, grid, n: int, res: int) -> np.ndarray:
    """Cell origin of the n^3 block centred (as nearly as the grid allows) at a world point."""
    lo = np.asarray(grid.lo, np.float64)
    h = (np.asarray(grid.hi, np.float64) - lo) / res
    c = np.floor((np.asarray(point, np.float64) - lo) / h).astype(np.int64) - n // 2
    return np.clip(c, 0, res - n)
