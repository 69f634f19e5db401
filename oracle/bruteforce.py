"""Exhaustive topology brute force over small label grids (test infrastructure only).

Every sign pattern of the 3 x 3 x 2 inner vertices of a 5 x 5 x 4 vertex grid
whose outer shell is outside is meshed by the oracle's dual topology (A.1.1
cycles, manifold fix, one quad per interior crossing edge); the result must be
a closed oriented 2-manifold.  Worker functions live here so that a ``spawn``
process pool can import them.
"""
from __future__ import annotations

import numpy as np

from . import meshcheck, odc, topology

INNER = [(i, j, k) for k in range(1, 3) for j in range(1, 4) for i in range(1, 4)]


def pattern(bits: int) -> np.ndarray:
    lab = np.zeros((4, 5, 5), bool)
    for n, (i, j, k) in enumerate(INNER):
        lab[k, j, i] = (bits >> n) & 1
    return lab


def check_range(args):
    """Mesh patterns lo..hi-1; returns (bad patterns, patterns with flips, max rounds)."""
    lo, hi, disable_fix = args
    saved = topology.face_same_cycle
    if disable_fix:
        topology.face_same_cycle = lambda *a: False
    bad, nflip, rounds = [], 0, 0
    try:
        for b in range(lo, hi):
            tris, t = odc.topology_triangles(pattern(b))
            nflip += bool(t["flipped"])
            rounds = max(rounds, t["rounds"])
            if not meshcheck.check_closed_manifold(tris)["ok"]:
                bad.append(b)
    finally:
        topology.face_same_cycle = saved
    return bad, nflip, rounds
