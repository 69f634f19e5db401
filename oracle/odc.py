"""Occupancy-based dual contouring, written out plainly in FP64 (test infrastructure only).

Follows the paper step by step:
  Sec. 3            grid, labels, crossing edges E^S and crossing cells C^S
  A.1.1, Fig. A1    partition of a cell's crossing edges into cycles, manifold fix
  Sec. 5.1          1D points by binary search on each crossing edge
  Sec. 5.2, A.1.3-4 2D points by three line-binary searches per face segment
  Sec. 5.3          normal at a 1D point from its two adjacent 2D points
  Eq. 2             one QEF 3D point per cycle, with the 2D-point normals
  Sec. 4, 5.4, A.1.5 one quad per interior crossing edge, split into 2 or 4
                    triangles by the convex/concave analysis (Eqs. A1, A2)

Readings where the paper is silent (each is listed in the design doc):
  * 1D output: the midpoint of the final interval, T/2^(k+1) with T odd.
  * 2D ray r: towards the side of l whose segment corners carry the label
    opposite to m's; "q coincides with m" means the line-binary search never
    moved off its start point.
  * Line-binary search: samples p_i = p + (R i / N) d, the first i whose label
    differs from p's (else N), then b bisections keeping the near end's label;
    the output is the near end.  Sample parameters are R J / (N 2^b) for an
    integer J.
  * Parallel lines in step 3 (|det| <= 1e-9 |r1||r2|) give p_f = m.
  * Normal n = (p_f1 - p_e) x (p_f2 - p_e); dropped when |n| < 1e-12.
  * QEF: mass point = mean of the cycle's 1D points; eigenvalues below 0.01
    of the largest are truncated; no clamping.
  * Quads only for edges with four incident cells; case 1 when both splits
    are valid; concavity for c1, c3, c4 by cyclic relabelling of Eqs. A1/A2.
All geometry is in cell-local units (a cell is the unit cube).

Parity unpinned: none of the above readings is printed in the paper; each is
pinned instead by the closed forms and invariants in tests/test_oracle_pins.py.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import topology as topo
from .occupancy import Occupancy

FACE_UV = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])   # face corners (u, v)

PAR_EPS = 1e-9       # relative parallel-line threshold of 2D step 3
NORMAL_EPS = 1e-12   # degenerate-normal threshold (cell units^2)
QEF_TRUNC = 0.01     # relative eigenvalue truncation


@dataclass
class Result:
    res: tuple
    steps: int
    labels: np.ndarray            # (Nz+1, Ny+1, Nx+1) bool, [k, j, i]
    label_margin: np.ndarray
    edges: np.ndarray             # sorted crossing edge ids 3 v + a
    T: np.ndarray                 # odd integers, 1D point = T / 2^(k+1) along the edge
    edge_margin: np.ndarray
    faces: np.ndarray             # (F, 2) [face id 3 v + a, slot], sorted
    face_pts: np.ndarray          # (F, 2) face-local (u, v) of the 2D point
    face_flags: np.ndarray        # (F,) bit0: q == m, bit1: parallel lines
    face_margin: np.ndarray
    flips: np.ndarray             # sorted face ids flipped by the manifold fix
    cells: np.ndarray             # sorted crossing cell ids
    configs: np.ndarray           # (C,) uint8
    cell_cyc: np.ndarray          # (C, 12) int8 cycle per local edge, -1 if none
    cell_ncyc: np.ndarray         # (C,)
    vbase: np.ndarray             # (C,) first vertex id of each cell
    verts_local: np.ndarray       # (V3, 3) cell-local 3D points
    vert_margin: np.ndarray       # (V3,) min decision margin feeding each 3D point
    vert_flag: np.ndarray         # (V3,) geometric near-threshold flag
    vertices: np.ndarray          # (V, 3) world positions (3D points, then case-3 points)
    triangles: np.ndarray         # (T, 3) int64
    quad_edges: np.ndarray        # edge list indices that emitted a quad
    quad_case: np.ndarray         # 1, 2 or 3 per quad
    quad_flag: np.ndarray         # near-zero concavity determinant or flagged vertex
    quad_margin: np.ndarray
    queries: int = 0
    stats: dict = field(default_factory=dict)


def grid_coords(grid):
    """Per-axis FP32 grid coordinates x_i = fl32(lo + (hi - lo) i / N), widened."""
    out = []
    for a in range(3):
        n = int(grid.res[a])
        i = np.arange(n + 1, dtype=np.float64)
        out.append((grid.lo[a] + (grid.hi[a] - grid.lo[a]) * i / n).astype(np.float32).astype(np.float64))
    return out


class _Geo:
    """Index helpers: vertex (i, j, k) <-> id, edge/face id = 3 v + a."""

    def __init__(self, res):
        self.N = tuple(int(r) for r in res)
        self.NV = tuple(n + 1 for n in self.N)

    def vid(self, i, j, k):
        return i + self.NV[0] * (j + self.NV[1] * k)

    def vijk(self, v):
        i = v % self.NV[0]
        t = v // self.NV[0]
        return i, t % self.NV[1], t // self.NV[1]

    def cid(self, i, j, k):
        return i + self.N[0] * (j + self.N[1] * k)

    def cijk(self, c):
        i = c % self.N[0]
        t = c // self.N[0]
        return i, t % self.N[1], t // self.N[1]


def _lab(labels, ijk):
    i, j, k = ijk
    return labels[k, j, i]


def _unit(a):
    return np.eye(3, dtype=np.int64)[a]


def _face_ambiguous(labels, geo, a):
    """Ids of faces perpendicular to axis ``a`` with four crossing edges."""
    NV = geo.NV
    b, c = (a + 1) % 3, (a + 2) % 3
    shp = [NV[0], NV[1], NV[2]]
    shp[b] -= 1
    shp[c] -= 1
    ii, jj, kk = np.meshgrid(np.arange(shp[0]), np.arange(shp[1]), np.arange(shp[2]), indexing="ij")
    ii, jj, kk = ii.ravel(), jj.ravel(), kk.ravel()
    base = np.stack([ii, jj, kk], axis=1)
    labs = []
    for (u, v) in ((0, 0), (1, 0), (1, 1), (0, 1)):
        q = base + u * _unit(b) + v * _unit(c)
        labs.append(labels[q[:, 2], q[:, 1], q[:, 0]])
    labs = np.stack(labs, axis=1)
    amb = (labs[:, 0] == labs[:, 2]) & (labs[:, 1] == labs[:, 3]) & (labs[:, 0] != labs[:, 1])
    return 3 * geo.vid(ii[amb], jj[amb], kk[amb]) + a


def dual_topology(labels):
    """Crossing cells, manifold fix and per-cell cycles for a label grid.

    ``labels`` is indexed [k, j, i].  Returns a dict with the cell configs,
    the set of flipped face ids, the cycle of every local edge and the first
    3D-point id of every crossing cell (A.1.1).
    """
    NVz, NVy, NVx = labels.shape
    geo = _Geo((NVx - 1, NVy - 1, NVz - 1))
    N = geo.N
    cfg = np.zeros((N[2], N[1], N[0]), np.int64)
    for corner in range(8):
        dx, dy, dz = topo.corner_offset(corner)
        cfg |= labels[dz:dz + N[2], dy:dy + N[1], dx:dx + N[0]].astype(np.int64) << corner
    cflat = cfg.ravel()
    cells = np.nonzero((cflat != 0) & (cflat != 255))[0].astype(np.int64)
    configs = cflat[cells].astype(np.uint8)
    C = cells.shape[0]

    flipped = set()

    def cell_flipmask(ci, cj, ck):
        m = 0
        for f in range(6):
            a, s = f // 2, f % 2
            q = [ci, cj, ck]
            q[a] += s
            if 3 * geo.vid(*q) + a in flipped:
                m |= 1 << f
        return m

    amb_cells = []
    for a in range(3):
        for fid in _face_ambiguous(labels, geo, a):
            v = int(fid // 3)
            q = [int(t) for t in geo.vijk(v)]
            if q[a] == 0 or q[a] == N[a]:
                continue   # boundary face: one cell only, never flipped
            below = list(q)
            below[a] -= 1
            amb_cells.append((int(fid), a, tuple(below), tuple(q)))
    amb_cells.sort()
    rounds = 0
    while True:
        marked = []
        for (fid, a, below, above) in amb_cells:
            cb = int(cfg[below[2], below[1], below[0]])
            ca = int(cfg[above[2], above[1], above[0]])
            if (topo.face_same_cycle(cb, cell_flipmask(*below), 2 * a + 1)
                    and topo.face_same_cycle(ca, cell_flipmask(*above), 2 * a)):
                marked.append(fid)
        if not marked:
            break
        for fid in marked:
            flipped ^= {fid}
        rounds += 1
        if rounds > 64:
            raise RuntimeError("manifold fix did not converge")

    ci, cj, ck = geo.cijk(cells)
    cell_cyc = np.full((C, 12), -1, np.int8)
    cell_ncyc = np.zeros(C, np.int64)
    cell_flipm = np.zeros(C, np.int64)
    for n in range(C):
        fm = cell_flipmask(int(ci[n]), int(cj[n]), int(ck[n])) if flipped else 0
        cell_flipm[n] = fm
        cyc, nc = topo.cell_cycles(int(configs[n]), fm)
        cell_cyc[n] = cyc
        cell_ncyc[n] = nc
    vbase = np.concatenate([[0], np.cumsum(cell_ncyc)[:-1]]).astype(np.int64) if C else np.zeros(0, np.int64)
    return dict(cfg=cfg, cells=cells, configs=configs, flipped=flipped, rounds=rounds,
                cell_cyc=cell_cyc, cell_ncyc=cell_ncyc, cell_flipm=cell_flipm,
                vbase=vbase, V3=int(cell_ncyc.sum()))


def quad_ring(a, lower_in):
    """Offsets (db, dc) of the four cells around an axis-``a`` edge, ordered so
    that the triangle of the first three cell centres faces from the inside
    end of the edge to the outside end (A.1.5)."""
    return [(0, 0), (1, 0), (1, 1), (0, 1)] if lower_in else [(0, 0), (0, 1), (1, 1), (1, 0)]


def topology_triangles(labels):
    """Triangles (two per quad, first diagonal) of the dual mesh of a label grid.

    Topology only: vertex ids are the 3D-point ids, no geometry is computed.
    """
    t = dual_topology(labels)
    NVz, NVy, NVx = labels.shape
    geo = _Geo((NVx - 1, NVy - 1, NVz - 1))
    N = geo.N
    cell_pos = {int(c): n for n, c in enumerate(t["cells"])}
    tris = []
    for a in range(3):
        ax = 2 - a
        sl0 = [slice(None)] * 3
        sl1 = [slice(None)] * 3
        sl0[ax] = slice(0, -1)
        sl1[ax] = slice(1, None)
        diff = labels[tuple(sl0)] != labels[tuple(sl1)]
        for (kk, jj, ii) in zip(*np.nonzero(diff)):
            v = np.array([ii, jj, kk])
            b, c = (a + 1) % 3, (a + 2) % 3
            if not (1 <= v[b] <= N[b] - 1 and 1 <= v[c] <= N[c] - 1):
                continue
            ids = []
            for (db, dc) in quad_ring(a, bool(labels[kk, jj, ii])):
                cc = v - db * _unit(b) - dc * _unit(c)
                n = cell_pos[int(geo.cid(*cc))]
                ids.append(int(t["vbase"][n]) + int(t["cell_cyc"][n, topo.edge_index(a, db, dc)]))
            tris += [(ids[0], ids[1], ids[2]), (ids[0], ids[2], ids[3])]
    return np.array(tris, np.int64).reshape(-1, 3), t



def extract(src, grid, steps_1d=15, lin1=4, bin1=11, range1=0.8, lin2=3, bin2=12,
            range2=float(np.float32(math.sqrt(2.0) / 2.0)), iso=0.5, ic_split=True) -> Result:
    """Run ODC on ``src`` (a CSG/MLP source or a callable) over ``grid``."""
    phi = Occupancy(src, iso)
    geo = _Geo(grid.res)
    N, NV = geo.N, geo.NV
    X = grid_coords(grid)
    range1 = float(np.float32(range1))
    range2 = float(np.float32(range2))
    k1 = int(steps_1d)

    # ---- grid labels (Sec. 3) ------------------------------------------------
    zz, yy, xx = np.meshgrid(X[2], X[1], X[0], indexing="ij")
    pts = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1)
    lab, lmar = phi(pts)
    labels = lab.reshape(NV[2], NV[1], NV[0])
    label_margin = lmar.reshape(NV[2], NV[1], NV[0])

    # ---- crossing edges E^S (Sec. 3) ------------------------------------------
    ids = []
    for a in range(3):
        ax = 2 - a
        sl0 = [slice(None)] * 3
        sl1 = [slice(None)] * 3
        sl0[ax] = slice(0, -1)
        sl1[ax] = slice(1, None)
        diff = labels[tuple(sl0)] != labels[tuple(sl1)]
        kk, jj, ii = np.nonzero(diff)
        ids.append(3 * geo.vid(ii, jj, kk) + a)
    edges = np.sort(np.concatenate(ids)).astype(np.int64)
    E = edges.shape[0]
    ev = edges // 3
    ea = edges % 3
    ei, ej, ek = geo.vijk(ev)
    eijk = np.stack([ei, ej, ek], axis=1)

    # ---- crossing faces and their corner labels --------------------------------
    fids = []
    for a in range(3):
        b, c = (a + 1) % 3, (a + 2) % 3
        shp = [NV[0], NV[1], NV[2]]
        shp[b] -= 1
        shp[c] -= 1
        ii, jj, kk = np.meshgrid(np.arange(shp[0]), np.arange(shp[1]), np.arange(shp[2]), indexing="ij")
        ii, jj, kk = ii.ravel(), jj.ravel(), kk.ravel()
        base = np.stack([ii, jj, kk], axis=1)
        labs = []
        for (u, v) in ((0, 0), (1, 0), (1, 1), (0, 1)):
            off = u * _unit(b) + v * _unit(c)
            q = base + off
            labs.append(labels[q[:, 2], q[:, 1], q[:, 0]])
        labs = np.stack(labs, axis=1)
        ncross = sum((labs[:, t] != labs[:, (t + 1) % 4]).astype(int) for t in range(4))
        sel = ncross > 0
        v = geo.vid(ii[sel], jj[sel], kk[sel])
        fid = 3 * v + a
        nseg = ncross[sel] // 2
        fids.append(np.stack([fid, nseg], axis=1))
    fall = np.concatenate(fids)
    fall = fall[np.argsort(fall[:, 0])]
    face_list = []
    for s in (0, 1):
        m = fall[:, 1] > s
        face_list.append(np.stack([fall[m, 0], np.full(int(m.sum()), s)], axis=1))
    faces = np.concatenate(face_list)
    faces = faces[np.lexsort((faces[:, 1], faces[:, 0]))]
    F = faces.shape[0]

    def face_labels(fid):
        v, a = fid // 3, fid % 3
        i, j, k = geo.vijk(v)
        b, c = (a + 1) % 3, (a + 2) % 3
        out = []
        for (u, w) in ((0, 0), (1, 0), (1, 1), (0, 1)):
            q = np.array([i, j, k]) + u * _unit(b) + w * _unit(c)
            out.append(bool(labels[q[2], q[1], q[0]]))
        return tuple(out)

    # ---- crossing cells, manifold fix and cycles (Sec. 3, A.1.1) ---------------
    topo_res = dual_topology(labels)
    cfg, cells, configs = topo_res["cfg"], topo_res["cells"], topo_res["configs"]
    flipped, rounds = topo_res["flipped"], topo_res["rounds"]
    cell_cyc, cell_ncyc, cell_flipm = topo_res["cell_cyc"], topo_res["cell_ncyc"], topo_res["cell_flipm"]
    vbase, V3 = topo_res["vbase"], topo_res["V3"]
    flips = np.array(sorted(flipped), np.int64)
    C = cells.shape[0]
    ci, cj, ck = geo.cijk(cells)

    # ---- 1D search (Sec. 5.1): k bisections on every crossing edge ---------------
    x_lo = np.stack([X[0][ei], X[1][ej], X[2][ek]], axis=1) if E else np.zeros((0, 3))
    span = np.zeros(E)
    for a in range(3):
        m = ea == a
        idx = eijk[m, a]
        span[m] = X[a][idx + 1] - X[a][idx]
    lab0 = labels[ek, ej, ei] if E else np.zeros(0, bool)
    edge_margin = np.minimum(label_margin[ek, ej, ei], np.zeros(E) + np.inf) if E else np.zeros(0)
    if E:
        up = eijk + np.eye(3, dtype=np.int64)[ea]
        edge_margin = np.minimum(edge_margin, label_margin[up[:, 2], up[:, 1], up[:, 0]])
    lo = np.zeros(E)
    width = 1.0
    for _ in range(k1):
        mid = lo + width / 2.0
        q = x_lo.copy()
        q[np.arange(E), ea] = x_lo[np.arange(E), ea] + span * mid
        lab, mar = phi(q)
        edge_margin = np.minimum(edge_margin, mar)
        lo = np.where(lab == lab0, mid, lo)
        width /= 2.0
    T = (2 * np.round(lo * (1 << k1)).astype(np.int64) + 1) if E else np.zeros(0, np.int64)
    tau = T / float(1 << (k1 + 1))

    def edge_pos(eid):
        return np.searchsorted(edges, eid)

    # ---- 2D search (Sec. 5.2, A.1.3, A.1.4) ------------------------------------------
    fv = faces[:, 0] // 3
    fa = faces[:, 0] % 3
    fslot = faces[:, 1]
    fi, fj, fk = geo.vijk(fv)
    fijk = np.stack([fi, fj, fk], axis=1)
    P1 = np.zeros((F, 2))
    P2 = np.zeros((F, 2))
    in_w = np.zeros((F, 2))       # out-corner -> in-corner along the first segment edge
    seg_margin = np.zeros(F)
    seg_edges = np.zeros((F, 2), np.int64)
    face_lab_cache = {}
    for n in range(F):
        fid = int(faces[n, 0])
        a = int(fa[n])
        labs4 = face_labels(fid)
        face_lab_cache[fid] = labs4
        segs = topo.face_segments(labs4, fid in flipped)
        (s0, s1) = segs[int(fslot[n])]
        v0 = fijk[n]
        b, c = (a + 1) % 3, (a + 2) % 3
        pts2 = []
        for t, fe in enumerate((s0, s1)):
            # global edge of face edge fe
            if fe == 0:
                g = 3 * geo.vid(*v0) + b
            elif fe == 1:
                g = 3 * geo.vid(*(v0 + _unit(b))) + c
            elif fe == 2:
                g = 3 * geo.vid(*(v0 + _unit(c))) + b
            else:
                g = 3 * geo.vid(*v0) + c
            pi = edge_pos(g)
            assert edges[pi] == g
            seg_edges[n, t] = pi
            tt = tau[pi]
            pts2.append({0: (tt, 0.0), 1: (1.0, tt), 2: (tt, 1.0), 3: (0.0, tt)}[fe])
        P1[n] = pts2[0]
        P2[n] = pts2[1]
        ca, cb = s0, (s0 + 1) % 4
        if labs4[ca]:
            in_w[n] = FACE_UV[ca] - FACE_UV[cb]
        else:
            in_w[n] = FACE_UV[cb] - FACE_UV[ca]
    if F:
        seg_margin = np.minimum(edge_margin[seg_edges[:, 0]], edge_margin[seg_edges[:, 1]])

    def face_world(uv, sel):
        """World point of face-local (u, v) on the faces ``sel`` (index array)."""
        out = np.zeros((uv.shape[0], 3))
        fa_s, fijk_s = fa[sel], fijk[sel]
        for a in range(3):
            m = fa_s == a
            if not m.any():
                continue
            b, c = (a + 1) % 3, (a + 2) % 3
            ia, ib, ic = fijk_s[m, a], fijk_s[m, b], fijk_s[m, c]
            out[m, a] = X[a][ia]
            out[m, b] = X[b][ib] + (X[b][ib + 1] - X[b][ib]) * uv[m, 0]
            out[m, c] = X[c][ic] + (X[c][ic + 1] - X[c][ic]) * uv[m, 1]
        return out

    face_margin = seg_margin.copy()

    def query(uv, active):
        lab = np.zeros(F, bool)
        if active.any():
            l, mar = phi(face_world(uv[active], np.nonzero(active)[0]))
            lab[active] = l
            face_margin[active] = np.minimum(face_margin[active], mar)
        return lab

    def lbs(p, d, R, n, b, lab0, active):
        """Line-binary search (A.1.3); returns the integer J of the near end."""
        denom = float(n * (1 << b))
        first = np.full(F, n, np.int64)
        found = np.zeros(F, bool)
        for i in range(1, n + 1):
            s = R * (i * (1 << b)) / denom
            act = active & ~found
            lab = query(p + s * d, act)
            hit = act & (lab != lab0)
            first[hit] = i
            found |= hit
        Ja = (first - 1) * (1 << b)
        Jc = first * (1 << b)
        for _ in range(b):
            Jm = (Ja + Jc) // 2
            s = R * Jm.astype(np.float64) / denom
            lab = query(p + s[:, None] * d, active)
            same = lab == lab0
            Ja = np.where(active & same, Jm, Ja)
            Jc = np.where(active & ~same, Jm, Jc)
        return Ja, denom

    flags = np.zeros(F, np.int64)
    pf = np.zeros((F, 2))
    if F:
        allf = np.ones(F, bool)
        m = (P1 + P2) / 2.0
        lab_m = query(m, allf)
        d0 = np.stack([-(P2[:, 1] - P1[:, 1]), P2[:, 0] - P1[:, 0]], axis=1)
        sig = np.sign(d0[:, 0] * in_w[:, 0] + d0[:, 1] * in_w[:, 1])
        d_in = sig[:, None] * d0 / np.linalg.norm(d0, axis=1)[:, None]
        d = np.where(lab_m[:, None], -d_in, d_in)
        Jq, den1 = lbs(m, d, range1, lin1, bin1, lab_m, allf)
        qm = Jq == 0
        flags[qm] |= 1
        q = m + (range1 * Jq.astype(np.float64) / den1)[:, None] * d
        act = ~qm
        u1 = (P1 - P2) / np.linalg.norm(P1 - P2, axis=1)[:, None]
        J1, den2 = lbs(q, u1, range2, lin2, bin2, lab_m, act)
        J2, _ = lbs(q, -u1, range2, lin2, bin2, lab_m, act)
        q1 = q + (range2 * J1.astype(np.float64) / den2)[:, None] * u1
        q2 = q - (range2 * J2.astype(np.float64) / den2)[:, None] * u1
        r1 = q1 - P1
        r2 = q2 - P2
        det = r1[:, 0] * r2[:, 1] - r1[:, 1] * r2[:, 0]
        par = act & (np.abs(det) <= PAR_EPS * np.linalg.norm(r1, axis=1) * np.linalg.norm(r2, axis=1))
        flags[par] |= 2
        dp = P2 - P1
        with np.errstate(divide="ignore", invalid="ignore"):
            alpha = (dp[:, 0] * r2[:, 1] - dp[:, 1] * r2[:, 0]) / det
        inter = P1 + alpha[:, None] * r1
        use_m = qm | par
        pf = np.where(use_m[:, None], m, inter)
        # near the parallel threshold finite precision could decide differently
        near_par = act & (np.abs(det) <= 1e3 * PAR_EPS * np.linalg.norm(r1, axis=1) * np.linalg.norm(r2, axis=1))
        flags[near_par & ~par] |= 4

    def face_pos(fid, slot):
        return np.searchsorted(faces[:, 0] * 2 + faces[:, 1], fid * 2 + slot)

    # ---- normals (Sec. 5.3) and QEF 3D points (Eq. 2) --------------------------------
    verts_local = np.zeros((V3, 3))
    vert_margin = np.full(V3, np.inf)
    vert_flag = np.zeros(V3, bool)
    for n in range(C):
        cfg_n = int(configs[n])
        fm = int(cell_flipm[n])
        cijk = np.array([ci[n], cj[n], ck[n]])
        cyc = cell_cyc[n]
        for cy in range(int(cell_ncyc[n])):
            A = np.zeros((3, 3))
            bvec = np.zeros(3)
            pes = []
            vid = int(vbase[n]) + cy
            mar = np.inf
            flag = False
            for le in range(12):
                if cyc[le] != cy:
                    continue
                a, o1, o2 = topo.edge_axis_offsets(le)
                d0 = np.array(topo.edge_start(le))
                gid = 3 * geo.vid(*(cijk + d0)) + a
                pi = edge_pos(gid)
                pe = d0.astype(np.float64)
                pe[a] = tau[pi]
                pes.append(pe)
                mar = min(mar, edge_margin[pi])
                pfs = []
                for f in topo.edge_faces(le):
                    fa_, s_ = f // 2, f % 2
                    fq = cijk.copy()
                    fq[fa_] += s_
                    gfid = 3 * geo.vid(*fq) + fa_
                    slot = topo.face_slot_of_edge(cfg_n, fm, f, le)
                    fpi = face_pos(gfid, slot)
                    assert faces[fpi, 0] == gfid and faces[fpi, 1] == slot
                    uv = pf[fpi]
                    p3 = np.zeros(3)
                    p3[fa_] = s_
                    p3[(fa_ + 1) % 3] = uv[0]
                    p3[(fa_ + 2) % 3] = uv[1]
                    pfs.append(p3)
                    mar = min(mar, face_margin[fpi])
                    if flags[fpi] & 4:
                        flag = True
                v1 = pfs[0] - pe
                v2 = pfs[1] - pe
                nrm = np.cross(v1, v2)
                nn = np.linalg.norm(nrm)
                if nn < 1e4 * NORMAL_EPS or nn < 1e-4 * np.linalg.norm(v1) * np.linalg.norm(v2):
                    flag = True
                if nn < NORMAL_EPS:
                    continue
                nh = nrm / nn
                A += np.outer(nh, nh)
                bvec += nh * np.dot(nh, pe)
            cbar = np.mean(pes, axis=0)
            lam, V = np.linalg.eigh(A)
            lmax = lam.max()
            x = cbar.copy()
            if lmax > 0:
                inv = np.zeros(3)
                keep = lam >= QEF_TRUNC * lmax
                inv[keep] = 1.0 / lam[keep]
                if np.any(np.abs(lam / lmax - QEF_TRUNC) < 1e-6):
                    flag = True
                x = cbar + V @ (inv * (V.T @ (bvec - A @ cbar)))
            verts_local[vid] = x
            vert_margin[vid] = mar
            vert_flag[vid] = flag

    cell_world0 = np.stack([X[0][ci], X[1][cj], X[2][ck]], axis=1) if C else np.zeros((0, 3))
    cell_span = np.stack([X[0][ci + 1] - X[0][ci], X[1][cj + 1] - X[1][cj], X[2][ck + 1] - X[2][ck]], axis=1) if C else np.zeros((0, 3))
    vcell = np.repeat(np.arange(C), cell_ncyc) if C else np.zeros(0, np.int64)
    verts3 = cell_world0[vcell] + cell_span[vcell] * verts_local if V3 else np.zeros((0, 3))

    # ---- quads with IC splitting (Sec. 4, Sec. 5.4, A.1.5) --------------------------------
    tris = []
    extra = []
    quad_edges, quad_case, quad_flag, quad_margin = [], [], [], []
    cell_pos = {int(c): n for n, c in enumerate(cells)}
    for n in range(E):
        a = int(ea[n])
        b, c = (a + 1) % 3, (a + 2) % 3
        v = eijk[n]
        if not (1 <= v[b] <= N[b] - 1 and 1 <= v[c] <= N[c] - 1):
            continue
        lower_in = bool(lab0[n])
        order = quad_ring(a, lower_in)
        vids, P = [], []
        mar = edge_margin[n]
        flag = False
        for (db, dc) in order:
            cc = v - db * _unit(b) - dc * _unit(c)
            cn = cell_pos[int(geo.cid(*cc))]
            le = topo.edge_index(a, db, dc)
            cy = int(cell_cyc[cn, le])
            vid = int(vbase[cn]) + cy
            vids.append(vid)
            P.append(verts_local[vid] - db * _unit(b) - dc * _unit(c))
            mar = min(mar, vert_margin[vid])
            flag |= bool(vert_flag[vid])
        P = np.array(P)
        p_in = np.zeros(3) if lower_in else _unit(a).astype(np.float64)
        p_out = _unit(a).astype(np.float64) if lower_in else np.zeros(3)
        case = 1
        if ic_split:
            conc = []
            dets = []
            for kq in range(4):
                pk, pp, pn = P[kq], P[(kq - 1) % 4], P[(kq + 1) % 4]
                d_out = np.dot(pk - p_out, np.cross(pp - p_out, pn - p_out))
                d_in = np.dot(pk - p_in, np.cross(pp - p_in, pn - p_in))
                dets += [d_out, d_in]
                conc.append(d_out < 0 or d_in > 0)
            ok1 = not (conc[1] or conc[3])
            ok2 = not (conc[0] or conc[2])
            case = 1 if ok1 else (2 if ok2 else 3)
            if min(abs(t) for t in dets) < 1e-5:
                flag = True
        c1, c2, c3, c4 = vids
        if case == 1:
            tris += [(c1, c2, c3), (c1, c3, c4)]
        elif case == 2:
            tris += [(c1, c2, c4), (c2, c3, c4)]
        else:
            pe_id = V3 + len(extra)
            pe = x_lo[n].copy()
            pe[a] = x_lo[n, a] + span[n] * tau[n]
            extra.append(pe)
            tris += [(pe_id, c1, c2), (pe_id, c2, c3), (pe_id, c3, c4), (pe_id, c4, c1)]
        quad_edges.append(n)
        quad_case.append(case)
        quad_flag.append(flag)
        quad_margin.append(mar)
    vertices = np.concatenate([verts3, np.array(extra).reshape(-1, 3)]) if (V3 or extra) else np.zeros((0, 3))
    triangles = np.array(tris, np.int64).reshape(-1, 3)

    return Result(res=N, steps=k1, labels=labels, label_margin=label_margin,
                  edges=edges, T=T, edge_margin=edge_margin, faces=faces, face_pts=pf,
                  face_flags=flags, face_margin=face_margin, flips=flips, cells=cells,
                  configs=configs, cell_cyc=cell_cyc, cell_ncyc=cell_ncyc, vbase=vbase,
                  verts_local=verts_local, vert_margin=vert_margin, vert_flag=vert_flag,
                  vertices=vertices, triangles=triangles,
                  quad_edges=np.array(quad_edges, np.int64), quad_case=np.array(quad_case, np.int64),
                  quad_flag=np.array(quad_flag, bool), quad_margin=np.array(quad_margin),
                  queries=phi.queries,
                  stats=dict(E=E, F=F, C=C, V3=V3, case3=len(extra), flips=len(flips),
                             fix_rounds=rounds, queries=phi.queries))
