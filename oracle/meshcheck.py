"""Plain mesh checks used to pin the oracle (test infrastructure only).

A closed oriented 2-manifold triangle mesh has every undirected edge in
exactly two triangles, traversed once in each direction, and the triangles
around every vertex form a single fan (its link is one cycle).  The Euler
characteristic is then chi = V - E + F = V - T/2 (each triangle has 3 edges,
each edge 2 triangles).  The enclosed volume is sum det[p0, p1, p2] / 6.
"""
from __future__ import annotations

from collections import defaultdict

import numpy as np


def check_closed_manifold(tris: np.ndarray, n_verts: int | None = None) -> dict:
    tris = np.asarray(tris, np.int64).reshape(-1, 3)
    out = dict(ok=True, n_tris=int(tris.shape[0]), problems=[])
    if tris.shape[0] == 0:
        return out
    if np.any(tris[:, 0] == tris[:, 1]) or np.any(tris[:, 1] == tris[:, 2]) or np.any(tris[:, 0] == tris[:, 2]):
        out["ok"] = False
        out["problems"].append("degenerate triangle (repeated vertex)")
    directed = np.concatenate([tris[:, [0, 1]], tris[:, [1, 2]], tris[:, [2, 0]]])
    # each directed edge exactly once, and its reverse exactly once
    key = directed[:, 0] * (1 << 32) + directed[:, 1]
    uniq, cnt = np.unique(key, return_counts=True)
    if np.any(cnt != 1):
        out["ok"] = False
        out["problems"].append(f"{int(np.sum(cnt != 1))} directed edges used more than once")
    rkey = directed[:, 1] * (1 << 32) + directed[:, 0]
    missing = ~np.isin(rkey, uniq)
    if np.any(missing):
        out["ok"] = False
        out["problems"].append(f"{int(missing.sum())} edges without opposite half-edge (boundary)")
    # vertex links: the fan around each vertex is a single cycle
    nxt = defaultdict(list)
    for t in tris:
        for r in range(3):
            v, a, b = t[r], t[(r + 1) % 3], t[(r + 2) % 3]
            nxt[int(v)].append((int(a), int(b)))
    bad = 0
    for v, pairs in nxt.items():
        succ = {}
        for (a, b) in pairs:
            if a in succ:
                bad += 1
                break
            succ[a] = b
        else:
            start = pairs[0][0]
            cur, steps = start, 0
            while True:
                cur = succ.get(cur)
                steps += 1
                if cur is None or steps > len(pairs):
                    break
                if cur == start:
                    break
            if cur != start or steps != len(pairs):
                bad += 1
    if bad:
        out["ok"] = False
        out["problems"].append(f"{bad} vertices whose link is not a single cycle")
    return out


def euler_characteristic(tris: np.ndarray) -> int:
    tris = np.asarray(tris).reshape(-1, 3)
    V = np.unique(tris).shape[0]
    return int(V - tris.shape[0] // 2)


def signed_volume(verts: np.ndarray, tris: np.ndarray) -> float:
    v = np.asarray(verts, np.float64)
    t = np.asarray(tris, np.int64).reshape(-1, 3)
    p0, p1, p2 = v[t[:, 0]], v[t[:, 1]], v[t[:, 2]]
    return float(np.sum(np.einsum("ij,ij->i", p0, np.cross(p1, p2))) / 6.0)


def components(tris: np.ndarray) -> int:
    """Number of connected components (by shared vertices)."""
    t = np.asarray(tris, np.int64).reshape(-1, 3)
    if t.shape[0] == 0:
        return 0
    verts = np.unique(t)
    parent = {int(v): int(v) for v in verts}

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x
    for a, b, c in t:
        ra, rb, rc = find(int(a)), find(int(b)), find(int(c))
        parent[rb] = ra
        parent[find(rc)] = ra
    return len({find(int(v)) for v in verts})
