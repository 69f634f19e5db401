"""Host logic of slab extraction (no GPU): the z split and the placement
bases; the bases agree across gloo ranks after one count all-gather."""
import os

import pytest
import torch.multiprocessing as mp

from paper_2409_13418_gb300.odc import slab_bases, slab_bounds


def test_bounds_cover_the_grid_once():
    for n, k in [(16, 1), (16, 3), (61, 7), (1024, 8), (5, 5)]:
        b = slab_bounds(n, k)
        assert b[0][0] == 0 and b[-1][1] == n
        assert all(z0 < z1 for z0, z1 in b)
        assert all(b[i][1] == b[i + 1][0] for i in range(k - 1))
        assert max(z1 - z0 for z0, z1 in b) - min(z1 - z0 for z0, z1 in b) <= 1


def test_bases_are_prefix_sums():
    counts = [(10, 2, 30), (0, 0, 0), (7, 1, 15), (5, 3, 9)]
    V = 22
    for r in range(4):
        b = slab_bases(counts, r)
        assert b["verts3_base"] == sum(c[0] for c in counts[:r])
        assert b["case3_base"] == V + sum(c[1] for c in counts[:r])
        assert b["tris_base"] == sum(c[2] for c in counts[:r])
        assert b["n_verts"] == V + 6 and b["n_tris"] == 54
    # consecutive slabs tile the merged arrays without gaps or overlaps
    ends = [slab_bases(counts, r) for r in range(4)]
    for r in range(3):
        assert ends[r]["verts3_base"] + counts[r][0] == ends[r + 1]["verts3_base"]
        assert ends[r]["case3_base"] + counts[r][1] == ends[r + 1]["case3_base"]
        assert ends[r]["tris_base"] + counts[r][2] == ends[r + 1]["tris_base"]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = (100 + 7 * rank, rank, 300 + rank)          # this rank's owned counts
    allc = [None] * world
    dist.all_gather_object(allc, mine)
    q.put((rank, slab_bases(allc, rank)))
    dist.destroy_process_group()


def test_bases_agree_across_gloo_ranks():
    world, port = 2, 29000 + os.getpid() % 2000
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    got = dict(q.get(timeout=120) for _ in range(world))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    counts = [(100 + 7 * r, r, 300 + r) for r in range(world)]
    for r in range(world):
        assert got[r] == slab_bases(counts, r)
    assert got[1]["verts3_base"] == 100 and got[1]["case3_base"] == 207 + 0 and got[1]["tris_base"] == 300
