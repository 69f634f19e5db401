"""Pins of the windowed comparison used for full-size parity (CPU only).

The oracle on a block of a grid must reproduce, on the block's core, what
the oracle on the whole grid computes there (ODC is local up to the manifold
fix, whose flips are compared too), and the comparison must catch a mistake
planted anywhere in the full-size result.
"""
import copy

import numpy as np
import pytest

from oracle import odc as oracle
from paper_2409_13418_gb300 import inputs as I
from tests.window_util import full_from_oracle, window_parity

RES, K, N_BLOCK = 32, 15, 10


@pytest.fixture(scope="module")
def whole():
    src = I.envelope_mlp(0)
    g = I.cube_grid(RES)
    r = oracle.extract(src, g, steps_1d=K)
    return src, g, r, full_from_oracle(r)


def _blocks(r, count, seed):
    rng = np.random.default_rng(seed)
    nv = RES + 1
    out = []
    for e in r.edges[rng.integers(0, len(r.edges), count)]:
        v = e // 3
        p = np.array([v % nv, (v // nv) % nv, v // (nv * nv)])
        out.append(np.clip(p - N_BLOCK // 2, 0, RES - N_BLOCK))
    return out


def test_blocks_reproduce_the_whole_grid_on_their_core(whole):
    src, g, r, full = whole
    tot = dict(core_cells=0, core_flips=0, core_faces=0, core_verts=0, core_tris=0)
    for w in _blocks(r, 5, 1):
        rep = window_parity(src, full, g, w, N_BLOCK, K, 2e-5)
        assert rep is not None
        assert rep["face_max_err"] == 0.0 and rep["vert_max_err"] == 0.0
        for k in tot:
            tot[k] += rep[k]
    assert all(v > 0 for v in tot.values()), tot


def _core_edge_block(r, full):
    """A block and the index (in the full edge list) of an edge deep inside it."""
    w = _blocks(r, 1, 2)[0]
    nv = RES + 1
    v = full["edges"] // 3
    p = np.stack([v % nv, (v // nv) % nv, v // (nv * nv)], axis=1) - w
    deep = np.all((p >= 4) & (p <= N_BLOCK - 4), axis=1) & (full["qcase"] > 0)
    return w, int(np.nonzero(deep)[0][0])


@pytest.mark.parametrize("plant", ["T", "triangle", "vertex", "flip", "config", "face_point", "cycle"])
def test_block_comparison_catches_planted_mistakes(whole, plant):
    src, g, r, full = whole
    w, e = _core_edge_block(r, full)
    bad = copy.deepcopy(full)
    nv, n = RES + 1, RES
    off = np.cumsum(np.where(full["qcase"] == 0, 0, np.where(full["qcase"] == 3, 4, 2)))
    t0 = off[e] - (4 if full["qcase"][e] == 3 else 2)
    if plant == "T":
        bad["T"][e] ^= 1 << K          # the first bisection decision, far from any tie
        msg = "1D decisions"
    elif plant == "triangle":
        bad["tris"][t0] = bad["tris"][t0][[0, 2, 1]]
        msg = "triangles differ"
    else:
        # a core cell of the block: the lower cell of the deep edge
        v = full["edges"][e] // 3
        ijk = np.array([v % nv, (v // nv) % nv, v // (nv * nv)])
        a = full["edges"][e] % 3
        ijk[(a + 1) % 3] -= 1
        ijk[(a + 2) % 3] -= 1
        cid = ijk[0] + n * (ijk[1] + n * ijk[2])
        ci = int(np.searchsorted(full["cells"], cid))
        assert full["cells"][ci] == cid
        ncyc = full["cyc"].max(axis=1) + 1
        vb = int(np.sum(ncyc[:ci]))
        if plant == "vertex":
            bad["vlocal"][vb, 0] += 1e-3
            msg = "3D points differ"
        elif plant == "config":
            bad["configs"][ci] ^= 1
            msg = "configurations differ"
        elif plant == "cycle":
            le = int(np.nonzero(full["cyc"][ci] >= 0)[0][0])
            bad["cyc"][ci, le] = 9
            msg = "cycles differ"
        elif plant == "flip":
            # flip a face of that cell that the manifold fix left alone
            fid = 3 * (ijk[0] + nv * (ijk[1] + nv * ijk[2])) + 0
            assert fid not in set(full["flips"].tolist())
            bad["flips"] = np.sort(np.append(full["flips"], fid))
            msg = "flips differ"
        else:
            fv = full["faces"] // 3
            fp = np.stack([fv % nv, (fv // nv) % nv, fv // (nv * nv)], axis=1) - w
            k = int(np.nonzero(np.all((fp >= 4) & (fp <= N_BLOCK - 4), axis=1))[0][0])
            bad["face_pts"][k] += 1e-3
            msg = "2D points differ"
    with pytest.raises(AssertionError, match=msg):
        window_parity(src, bad, g, w, N_BLOCK, K, 2e-5)
