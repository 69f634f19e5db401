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

Readings where the paper is silent:
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

Pins: the paper prints none of the above readings, so each is pinned by
the closed forms and invariants in tests/test_oracle_pins.py,
and the IC case rule (ic_cases) by the envelope-containment brute force and
the intersection-free guarantee of A.1.5 in tests/test_oracle_ic.py.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import occupancy
from . import topology as topo
from .occupancy import Occupancy

FACE_UV = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])   # face corners (u, v)

def _fe_point(fe, t):
    """Face-local (u, v) of the point at parameter t along face edge fe."""
    u = np.where(fe == 1, 1.0, np.where(fe == 3, 0.0, t))
    v = np.where(fe == 2, 1.0, np.where(fe == 0, 0.0, t))
    return np.stack([u, v], axis=-1)


FE_POINT = _fe_point


def _seg_table():
    """SEG[lab4, flip, slot] = (face edge 1, face edge 2) from topology.face_segments."""
    t = np.full((16, 2, 2, 2), -1, np.int64)
    for L in range(16):
        for fl in (0, 1):
            for s, (i, j) in enumerate(topo.face_segments([(L >> b) & 1 for b in range(4)], bool(fl))):
                t[L, fl, s] = (i, j)
    return t


def _slot_table():
    """SLOT[config, flip of face f, f, local edge] = segment slot holding the edge."""
    t = np.zeros((256, 2, 6, 12), np.int64)
    for cfg in range(256):
        for fl in (0, 1):
            for f in range(6):
                for le in topo.face_edges(f):
                    try:
                        t[cfg, fl, f, le] = topo.face_slot_of_edge(cfg, fl << f, f, le)
                    except ValueError:
                        pass
    return t


SEG_TABLE = _seg_table()
SLOT_TABLE = _slot_table()

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
    search: dict = field(default_factory=dict)   # 2D decisions: Jq, J1, J2, lab_m, found
    violations: dict = field(default_factory=dict)   # per-element replay violations: edges (E,), faces (F,)


def grid_coords(grid):
    """Per-axis FP32 grid coordinates x_i = fl32(lo + (hi - lo) i / N), widened.

    The box bounds are float32 values (they define the instance), widened to
    double before the formula is evaluated.
    """
    out = []
    for a in range(3):
        n = int(grid.res[a])
        lo = float(np.float32(grid.lo[a]))
        hi = float(np.float32(grid.hi[a]))
        i = np.arange(n + 1, dtype=np.float64)
        out.append((lo + (hi - lo) * i / n).astype(np.float32).astype(np.float64))
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



def ic_cases(P, p_in, p_out):
    """Split case of each quad by the convex/concave analysis (A.1.5).

    P [Q, 4, 3]: the 3D points of cells c1..c4 around a crossing edge, ordered
    so that the triangle of the cell centres c1, c2, c3 has its normal along
    v_in -> v_out; p_in, p_out [Q, 3]: the edge's inside and outside ends.
    Eq. A1: the edge (p_c2, v_out) is concave when p_c2 lies below the oriented
    triangle (p_c1, p_c3, v_out); Eq. A2: the edge (p_c2, v_in) is concave when
    p_c2 lies above (p_c1, p_c3, v_in); p_c2 is concave when either is.  The
    other three vertices take the same tests with their own ring neighbours
    (c_{k-1}, c_{k+1}) in place of (c1, c3).  Case 1 (diagonal c1 c3) is valid
    when neither c2 nor c4 is concave, case 2 (diagonal c2 c4) when neither
    c1 nor c3 is; case 1 when both are valid, case 3 (a fan around p_e) when
    neither is.  Returns (case [Q], smallest |determinant| over the tests).
    """
    Q = P.shape[0]
    conc = np.zeros((Q, 4), bool)
    mindet = np.full(Q, np.inf)
    for kq in range(4):
        pk, pp, pn = P[:, kq], P[:, (kq - 1) % 4], P[:, (kq + 1) % 4]
        d_out = np.einsum("ij,ij->i", pk - p_out, np.cross(pp - p_out, pn - p_out))
        d_in = np.einsum("ij,ij->i", pk - p_in, np.cross(pp - p_in, pn - p_in))
        conc[:, kq] = (d_out < 0) | (d_in > 0)
        mindet = np.minimum(mindet, np.minimum(np.abs(d_out), np.abs(d_in)))
    ok1 = ~(conc[:, 1] | conc[:, 3])
    ok2 = ~(conc[:, 0] | conc[:, 2])
    return np.where(ok1, 1, np.where(ok2, 2, 3)), mindet


def extract(src, grid, steps_1d=15, lin1=4, bin1=11, range1=0.8, lin2=3, bin2=12,
            range2=float(np.float32(math.sqrt(2.0) / 2.0)), iso=0.5, ic_split=True,
            replay=None, replay_margin=0.0, linear_1d=False, gradient_normals=False, mc=False) -> Result:
    """Run ODC on ``src`` (a CSG/MLP source or a callable) over ``grid``.

    Ablation variants (Sec. 6.3, Tab. 3; CSG sources only, which have an
    implicit psi and its gradient): ``linear_1d`` places each 1D point by
    Eq. 1 (linear interpolation of psi between the edge's ends, taken in FP32
    and quantised to the 1D lattice of 2^-(k+1) edge) instead of the binary
    search; ``gradient_normals`` uses grad psi at the 1D point as the plane
    normal of Eq. 3 instead of the 2D points (the 2D search is skipped).

    ``mc`` polygonizes as marching cubes with the same cycles (Tab. A8's "MC"
    rows): the mesh vertices are the 1D points (edge order) and every cycle
    of every crossing cell (cell order, cycle order) is fanned from its
    smallest local edge along topology.mc_successors; no 2D search, QEF or
    quads.

    ``replay`` (optional) supplies the search decisions of another
    implementation instead of taking them from phi: ``T`` (1D results) and
    the 2D decisions ``Jq, J1, J2, lab_m, found``.  Every replayed decision is
    still checked against phi here: a replayed label that disagrees with phi
    where phi's margin is at least ``replay_margin`` is a violation, counted
    per element in ``stats['edge_violations']`` / ``stats['face_violations']``
    (totals) and ``violations['edges']`` / ``violations['faces']`` (masks).
    All geometry downstream is then computed from the replayed decisions.
    """
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
    edge_viol = np.zeros(E, bool)
    if replay is not None:
        lo_rep = (np.asarray(replay["T"], np.int64) - 1) // 2      # k-bit low end of the final interval
    for step in range(0 if linear_1d else k1):
        mid = lo + width / 2.0
        q = x_lo.copy()
        q[np.arange(E), ea] = x_lo[np.arange(E), ea] + span * mid
        lab, mar = phi(q)
        edge_margin = np.minimum(edge_margin, mar)
        same = lab == lab0
        if replay is not None:
            rep_same = ((lo_rep >> (k1 - 1 - step)) & 1).astype(bool)
            edge_viol |= (rep_same != same) & (mar >= replay_margin)
            same = rep_same
        lo = np.where(same, mid, lo)
        width /= 2.0
    T = (2 * np.round(lo * (1 << k1)).astype(np.int64) + 1) if E else np.zeros(0, np.int64)
    if linear_1d and E:
        # Eq. 1 in FP32: t = psi(p0) / (psi(p0) - psi(p1)) along the edge from its
        # lower end, clamped to [0, 1], rounded to the nearest multiple of
        # 2^-(k+1) strictly inside the edge
        f32 = np.float32
        x_hi = x_lo.copy()
        up = eijk + np.eye(3, dtype=np.int64)[ea]
        for a in range(3):
            m = ea == a
            x_hi[m, a] = X[a][up[m, a]]
        psi0 = occupancy.csg_psi32(src, x_lo.astype(f32))
        psi1 = occupancy.csg_psi32(src, x_hi.astype(f32))
        den = psi0 - psi1
        with np.errstate(divide="ignore", invalid="ignore"):
            tl = np.where(den != 0, psi0 / np.where(den != 0, den, f32(1)), f32(0.5)).astype(f32)
        tl = np.minimum(np.maximum(tl, f32(0.0)), f32(1.0))
        full = 1 << (k1 + 1)
        T = np.clip(np.rint(tl * f32(full)).astype(np.int64), 1, full - 1)
    tau = T / float(1 << (k1 + 1))

    def edge_pos(eid):
        return np.searchsorted(edges, eid)

    # ---- 2D search (Sec. 5.2, A.1.3, A.1.4) ------------------------------------------
    fv = faces[:, 0] // 3
    fa = faces[:, 0] % 3
    fslot = faces[:, 1]
    fi, fj, fk = geo.vijk(fv)
    fijk = np.stack([fi, fj, fk], axis=1)
    fb = (fa + 1) % 3
    fc = (fa + 2) % 3
    EYE = np.eye(3, dtype=np.int64)
    # face-corner labels in face order (u, v) = (0,0), (1,0), (1,1), (0,1)
    lab4 = np.zeros((F, 4), bool)
    for t, (du, dv) in enumerate(((0, 0), (1, 0), (1, 1), (0, 1))):
        q = fijk + du * EYE[fb] + dv * EYE[fc]
        lab4[:, t] = labels[q[:, 2], q[:, 1], q[:, 0]]
    lab4i = lab4 @ np.array([1, 2, 4, 8])
    fflip = np.isin(faces[:, 0], flips)
    s0 = SEG_TABLE[lab4i, fflip.astype(np.int64), fslot, 0]
    s1 = SEG_TABLE[lab4i, fflip.astype(np.int64), fslot, 1]

    def face_edge_pos(fe):
        """Index in ``edges`` of the global edge under face edge ``fe``."""
        q = fijk + (fe == 1)[:, None] * EYE[fb] + (fe == 2)[:, None] * EYE[fc]
        axis = np.where((fe == 0) | (fe == 2), fb, fc)
        g = 3 * geo.vid(q[:, 0], q[:, 1], q[:, 2]) + axis
        pi = np.searchsorted(edges, g)
        assert np.all(edges[pi] == g)
        return pi

    seg_edges = np.stack([face_edge_pos(s0), face_edge_pos(s1)], axis=1) if F else np.zeros((0, 2), np.int64)
    P1 = FE_POINT(s0, tau[seg_edges[:, 0]]) if F else np.zeros((0, 2))
    P2 = FE_POINT(s1, tau[seg_edges[:, 1]]) if F else np.zeros((0, 2))
    # out-corner -> in-corner along the first segment edge (face corners s0, s0+1)
    ca, cb = s0, (s0 + 1) % 4
    inA = lab4[np.arange(F), ca] if F else np.zeros(0, bool)
    in_w = np.where(inA[:, None], FACE_UV[ca] - FACE_UV[cb], FACE_UV[cb] - FACE_UV[ca]) if F else np.zeros((0, 2))
    seg_margin = np.minimum(edge_margin[seg_edges[:, 0]], edge_margin[seg_edges[:, 1]]) if F else np.zeros(0)

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

    face_viol = np.zeros(F, bool)

    def query(uv, active):
        lab = np.zeros(F, bool)
        mar_out = np.full(F, np.inf)
        if active.any():
            l, mar = phi(face_world(uv[active], np.nonzero(active)[0]))
            lab[active] = l
            mar_out[active] = mar
            face_margin[active] = np.minimum(face_margin[active], mar)
        return lab, mar_out

    def lbs(p, d, R, n, b, lab0, active, rep=None):
        """Line-binary search (A.1.3); returns the integer J of the near end.

        ``rep = (J, found)`` replays another run's result: the first line
        sample with a label change is J // 2^b + 1 when ``found`` (else the
        last sample keeps p's label), and the bits of J below 2^b are the
        bisection decisions, most significant first (1: kept p's label).
        """
        nonlocal face_viol
        denom = float(n * (1 << b))
        first = np.full(F, n, np.int64)
        found = np.zeros(F, bool)
        if rep is not None:
            Jr, fr = np.asarray(rep[0], np.int64), np.asarray(rep[1], bool)
            first_r = np.where(fr, (Jr >> b) + 1, n)
        for i in range(1, n + 1):
            s = R * (i * (1 << b)) / denom
            if rep is None:
                act = active & ~found
                lab, _ = query(p + s * d, act)
                hit = act & (lab != lab0)
            else:
                act = active & (i <= first_r)
                lab, mar = query(p + s * d, act)
                hit = act & (i == first_r) & fr
                face_viol |= act & ((lab != lab0) != hit) & (mar >= replay_margin)
            first[hit] = i
            found |= hit
        if rep is not None:
            first = np.where(active, first_r, first)
        Ja = (first - 1) * (1 << b)
        Jc = first * (1 << b)
        for t in range(b):
            Jm = (Ja + Jc) // 2
            s = R * Jm.astype(np.float64) / denom
            lab, mar = query(p + s[:, None] * d, active)
            same = lab == lab0
            if rep is not None:
                rep_same = (((Jr - (first - 1) * (1 << b)) >> (b - 1 - t)) & 1).astype(bool)
                face_viol |= active & (rep_same != same) & (mar >= replay_margin)
                same = rep_same
            Ja = np.where(active & same, Jm, Ja)
            Jc = np.where(active & ~same, Jm, Jc)
        lbs.found = found
        return Ja, denom

    flags = np.zeros(F, np.int64)
    pf = np.zeros((F, 2))
    search = dict(Jq=np.zeros(0, np.int64), J1=np.zeros(0, np.int64), J2=np.zeros(0, np.int64),
                  lab_m=np.zeros(0, bool), found=np.zeros(0, np.int64))
    if F and not gradient_normals and not mc:
        allf = np.ones(F, bool)
        m = (P1 + P2) / 2.0
        lab_m, mar_m = query(m, allf)
        if replay is not None:
            rlab = np.asarray(replay["lab_m"], bool)
            face_viol |= (rlab != lab_m) & (mar_m >= replay_margin)
            lab_m = rlab
            rfound = np.asarray(replay["found"], np.int64)
        d0 = np.stack([-(P2[:, 1] - P1[:, 1]), P2[:, 0] - P1[:, 0]], axis=1)
        sig = np.sign(d0[:, 0] * in_w[:, 0] + d0[:, 1] * in_w[:, 1])
        d_in = sig[:, None] * d0 / np.linalg.norm(d0, axis=1)[:, None]
        d = np.where(lab_m[:, None], -d_in, d_in)
        Jq, den1 = lbs(m, d, range1, lin1, bin1, lab_m, allf,
                       None if replay is None else (replay["Jq"], rfound & 1))
        found_bits = lbs.found.astype(np.int64)
        qm = Jq == 0
        flags[qm] |= 1
        q = m + (range1 * Jq.astype(np.float64) / den1)[:, None] * d
        act = ~qm
        u1 = (P1 - P2) / np.linalg.norm(P1 - P2, axis=1)[:, None]
        J1, den2 = lbs(q, u1, range2, lin2, bin2, lab_m, act,
                       None if replay is None else (replay["J1"], (rfound >> 1) & 1))
        found_bits |= (lbs.found & act).astype(np.int64) << 1
        J2, _ = lbs(q, -u1, range2, lin2, bin2, lab_m, act,
                    None if replay is None else (replay["J2"], (rfound >> 2) & 1))
        found_bits |= (lbs.found & act).astype(np.int64) << 2
        search = dict(Jq=Jq, J1=np.where(act, J1, 0), J2=np.where(act, J2, 0), lab_m=lab_m, found=found_bits)
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

    fkey = faces[:, 0] * 2 + faces[:, 1]

    if mc:
        # ---- marching-cubes polygons through the 1D points (Tab. A8) ---------------
        pw = x_lo.copy()
        pw[np.arange(E), ea] = x_lo[np.arange(E), ea] + span * tau
        verts = pw.astype(np.float32).astype(np.float64)
        tris = []
        for c in range(C):
            cyc = cell_cyc[c]
            succ = topo.mc_successors(int(configs[c]), int(cell_flipm[c]))
            cell = np.array([ci[c], cj[c], ck[c]])
            gid = {}
            for le in range(12):
                if cyc[le] >= 0:
                    a, o1, o2 = topo.edge_axis_offsets(le)
                    q = cell.copy()
                    q[(a + 1) % 3] += o1
                    q[(a + 2) % 3] += o2
                    gid[le] = int(np.searchsorted(edges, 3 * geo.vid(q[0], q[1], q[2]) + a))
            for cy in range(int(cell_ncyc[c])):
                le0 = min(le for le in range(12) if cyc[le] == cy)
                ring = [le0]
                while succ[ring[-1]] != le0:
                    ring.append(succ[ring[-1]])
                for t in range(1, len(ring) - 1):
                    tris.append((gid[ring[0]], gid[ring[t]], gid[ring[t + 1]]))
        z3 = np.zeros((0, 3))
        return Result(res=N, steps=k1, labels=labels, label_margin=label_margin,
                      edges=edges, T=T, edge_margin=edge_margin, faces=faces, face_pts=pf, face_flags=flags,
                      face_margin=face_margin, flips=flips, cells=cells, configs=configs, cell_cyc=cell_cyc,
                      cell_ncyc=cell_ncyc, vbase=vbase, verts_local=z3, vert_margin=np.zeros(0), vert_flag=np.zeros(0, bool),
                      vertices=verts, triangles=np.array(tris, np.int64).reshape(-1, 3),
                      quad_edges=np.zeros(0, np.int64), quad_case=np.zeros(0, np.int64), quad_flag=np.zeros(0, bool),
                      quad_margin=np.zeros(0), queries=phi.queries, search=search,
                      violations=dict(edges=edge_viol, faces=np.zeros(F, bool)),
                      stats=dict(E=E, F=F, C=C, V3=0, case3=0, flips=len(flips), fix_rounds=rounds,
                                 queries=phi.queries, edge_violations=int(edge_viol.sum()), face_violations=0))

    # ---- normals (Sec. 5.3) and QEF 3D points (Eq. 2) --------------------------------
    # every (crossing cell, crossing local edge) pair contributes one plane to
    # the QEF of the cycle holding the edge
    pc, ple = np.nonzero(cell_cyc >= 0)
    K = pc.shape[0]
    pvid = vbase[pc] + cell_cyc[pc, ple]
    pa = ple // 4
    po1, po2 = ple & 1, (ple >> 1) & 1
    d0 = np.zeros((K, 3), np.int64)
    d0[np.arange(K), (pa + 1) % 3] = po1
    d0[np.arange(K), (pa + 2) % 3] = po2
    cijk_all = np.stack([ci, cj, ck], axis=1)
    pcell = cijk_all[pc]
    q = pcell + d0
    ppi = np.searchsorted(edges, 3 * geo.vid(q[:, 0], q[:, 1], q[:, 2]) + pa)
    pe = d0.astype(np.float64)
    pe[np.arange(K), pa] = tau[ppi]
    mar = edge_margin[ppi].copy()
    pflag = np.zeros(K, bool)
    pfs = []
    for f in (2 * ((pa + 1) % 3) + po1, 2 * ((pa + 2) % 3) + po2):   # the two faces holding the edge
        fa_, s_ = f // 2, f % 2
        fq = pcell + s_[:, None] * EYE[fa_]
        gfid = 3 * geo.vid(fq[:, 0], fq[:, 1], fq[:, 2]) + fa_
        slot = SLOT_TABLE[configs[pc], (cell_flipm[pc] >> f) & 1, f, ple]
        fpi = np.searchsorted(fkey, gfid * 2 + slot)
        assert np.all(fkey[fpi] == gfid * 2 + slot)
        uv = pf[fpi]
        p3 = np.zeros((K, 3))
        p3[np.arange(K), fa_] = s_
        p3[np.arange(K), (fa_ + 1) % 3] = uv[:, 0]
        p3[np.arange(K), (fa_ + 2) % 3] = uv[:, 1]
        pfs.append(p3)
        mar = np.minimum(mar, face_margin[fpi])
        pflag |= (flags[fpi] & 4) != 0
    v1 = pfs[0] - pe
    v2 = pfs[1] - pe
    nrm = np.cross(v1, v2)
    if gradient_normals and K:
        # Eq. 3: grad psi at the 1D point, as a normal in cell-local units
        span_c = np.stack([X[0][ci + 1] - X[0][ci], X[1][cj + 1] - X[1][cj], X[2][ck + 1] - X[2][ck]], axis=1)[pc]
        world0 = np.stack([X[0][ci], X[1][cj], X[2][ck]], axis=1)[pc]
        nrm = occupancy.csg_grad(src, world0 + span_c * pe) * span_c
    nn = np.linalg.norm(nrm, axis=1)
    pflag |= nn < 1e4 * NORMAL_EPS
    if not gradient_normals:   # a cross product of nearly parallel rays
        pflag |= nn < 1e-4 * np.linalg.norm(v1, axis=1) * np.linalg.norm(v2, axis=1)
    keep = nn >= NORMAL_EPS
    nh = np.zeros((K, 3))
    nh[keep] = nrm[keep] / nn[keep, None]
    A = np.zeros((V3, 3, 3))
    bvec = np.zeros((V3, 3))
    csum = np.zeros((V3, 3))
    np.add.at(A, pvid, nh[:, :, None] * nh[:, None, :])
    np.add.at(bvec, pvid, nh * np.einsum("ij,ij->i", nh, pe)[:, None])
    np.add.at(csum, pvid, pe)
    cnt = np.bincount(pvid, minlength=V3)
    vert_margin = np.full(V3, np.inf)
    np.minimum.at(vert_margin, pvid, mar)
    vert_flag = np.zeros(V3, bool)
    np.logical_or.at(vert_flag, pvid, pflag)
    cbar = csum / np.maximum(cnt, 1)[:, None]
    verts_local = cbar.copy()
    if V3:
        lam, V = np.linalg.eigh(A)
        lmax = lam.max(axis=1)
        pos = lmax > 0
        with np.errstate(divide="ignore", invalid="ignore"):
            ratio = lam / lmax[:, None]
            inv = np.where((ratio >= QEF_TRUNC) & pos[:, None], 1.0 / lam, 0.0)
            vert_flag |= pos & np.any(np.abs(ratio - QEF_TRUNC) < 1e-6, axis=1)
        rhs = bvec - np.einsum("vij,vj->vi", A, cbar)
        t = inv * np.einsum("vji,vj->vi", V, rhs)
        verts_local = cbar + np.einsum("vij,vj->vi", V, t)

    cell_world0 = np.stack([X[0][ci], X[1][cj], X[2][ck]], axis=1) if C else np.zeros((0, 3))
    cell_span = np.stack([X[0][ci + 1] - X[0][ci], X[1][cj + 1] - X[1][cj], X[2][ck + 1] - X[2][ck]], axis=1) if C else np.zeros((0, 3))
    vcell = np.repeat(np.arange(C), cell_ncyc) if C else np.zeros(0, np.int64)
    verts3 = cell_world0[vcell] + cell_span[vcell] * verts_local if V3 else np.zeros((0, 3))

    # ---- quads with IC splitting (Sec. 4, Sec. 5.4, A.1.5) --------------------------------
    eb, ec = (ea + 1) % 3, (ea + 2) % 3
    ar = np.arange(E)
    qsel = ((eijk[ar, eb] >= 1) & (eijk[ar, eb] <= np.array(N)[eb] - 1) &
            (eijk[ar, ec] >= 1) & (eijk[ar, ec] <= np.array(N)[ec] - 1)) if E else np.zeros(0, bool)
    qn = np.nonzero(qsel)[0]
    Q = qn.shape[0]
    qa, qb, qc = ea[qn], eb[qn], ec[qn]
    lower_in = lab0[qn].astype(bool)
    RING_IN = np.array([(0, 0), (1, 0), (1, 1), (0, 1)])
    RING_OUT = np.array([(0, 0), (0, 1), (1, 1), (1, 0)])
    vids = np.zeros((Q, 4), np.int64)
    P = np.zeros((Q, 4, 3))
    qmar = edge_margin[qn].copy()
    qflag = np.zeros(Q, bool)
    for kq in range(4):
        db = np.where(lower_in, RING_IN[kq, 0], RING_OUT[kq, 0])
        dc = np.where(lower_in, RING_IN[kq, 1], RING_OUT[kq, 1])
        off = db[:, None] * EYE[qb] + dc[:, None] * EYE[qc]
        cc = eijk[qn] - off
        cpos = np.searchsorted(cells, geo.cid(cc[:, 0], cc[:, 1], cc[:, 2]))
        le = 4 * qa + db + 2 * dc
        vids[:, kq] = vbase[cpos] + cell_cyc[cpos, le]
        P[:, kq] = verts_local[vids[:, kq]] - off
        qmar = np.minimum(qmar, vert_margin[vids[:, kq]])
        qflag |= vert_flag[vids[:, kq]]
    p_in = np.where(lower_in[:, None], 0.0, EYE[qa].astype(np.float64))
    p_out = np.where(lower_in[:, None], EYE[qa].astype(np.float64), 0.0)
    case = np.ones(Q, np.int64)
    if ic_split and Q:
        case, mindet = ic_cases(P, p_in, p_out)
        qflag |= mindet < 1e-5
    is3 = case == 3
    pe_id = V3 + np.cumsum(is3) - 1
    c1, c2, c3, c4 = vids[:, 0], vids[:, 1], vids[:, 2], vids[:, 3]
    tri4 = np.full((Q, 4, 3), -1, np.int64)
    m1, m2 = case == 1, case == 2
    tri4[m1, 0] = np.stack([c1, c2, c3], 1)[m1]
    tri4[m1, 1] = np.stack([c1, c3, c4], 1)[m1]
    tri4[m2, 0] = np.stack([c1, c2, c4], 1)[m2]
    tri4[m2, 1] = np.stack([c2, c3, c4], 1)[m2]
    tri4[is3, 0] = np.stack([pe_id, c1, c2], 1)[is3]
    tri4[is3, 1] = np.stack([pe_id, c2, c3], 1)[is3]
    tri4[is3, 2] = np.stack([pe_id, c3, c4], 1)[is3]
    tri4[is3, 3] = np.stack([pe_id, c4, c1], 1)[is3]
    triangles = tri4.reshape(-1, 3)
    triangles = triangles[triangles[:, 0] >= 0]
    extra = x_lo[qn[is3]].copy()
    extra[np.arange(extra.shape[0]), ea[qn[is3]]] = x_lo[qn[is3], ea[qn[is3]]] + span[qn[is3]] * tau[qn[is3]]
    vertices = np.concatenate([verts3, extra.reshape(-1, 3)])
    quad_edges, quad_case, quad_flag, quad_margin = qn, case, qflag, qmar

    return Result(res=N, steps=k1, labels=labels, label_margin=label_margin,
                  edges=edges, T=T, edge_margin=edge_margin, faces=faces, face_pts=pf,
                  face_flags=flags, face_margin=face_margin, flips=flips, cells=cells,
                  configs=configs, cell_cyc=cell_cyc, cell_ncyc=cell_ncyc, vbase=vbase,
                  verts_local=verts_local, vert_margin=vert_margin, vert_flag=vert_flag,
                  vertices=vertices, triangles=triangles,
                  quad_edges=quad_edges.astype(np.int64), quad_case=quad_case.astype(np.int64),
                  quad_flag=quad_flag.astype(bool), quad_margin=qmar,
                  queries=phi.queries, search=search,
                  violations=dict(edges=edge_viol, faces=face_viol),
                  stats=dict(E=E, F=F, C=C, V3=V3, case3=int(is3.sum()), flips=len(flips),
                             fix_rounds=rounds, queries=phi.queries,
                             edge_violations=int(edge_viol.sum()), face_violations=int(face_viol.sum())))
