"""The allocation-free edge compaction against the regular extraction.

odc_compact_edges_noalloc serves callers that cannot allocate device memory
(stream captures that must not gain allocation nodes, allocator-free hosts,
plug-ins whose host owns all device memory).  It keeps its scratch in a fixed
device array shared by all calls, so two calls in a row must each give the
same crossing-edge list as odc_extract's own compaction of the same labels.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_edges_match_extract_twice():
    import torch

    from paper_2409_13418_gb300 import build, inputs as I, odc
    build.build()
    ctx = odc.Context(0)
    try:
        for seed, n in ((3, 96), (5, 61)):      # second call: other grid, reused scratch
            src = I.random_csg(seed)
            grid = I.cube_grid(n)
            ctx.extract(src, grid, steps_1d=8)
            bits = ctx.debug("labels")
            ref = ctx.debug("edges")
            d_bits = torch.from_numpy(bits.view(np.int32).copy()).cuda()
            d_edges = torch.full((ref.size + 64,), -1, dtype=torch.int32, device="cuda")
            d_count = torch.zeros(1, dtype=torch.int32, device="cuda")
            stream = torch.cuda.current_stream().cuda_stream
            cnt = odc.compact_edges_noalloc(d_bits.data_ptr(), grid.res, d_edges.data_ptr(), d_edges.numel(),
                                            d_count.data_ptr(), stream)
            got = d_edges[:cnt].cpu().numpy().view(np.uint32)
            assert cnt == ref.size == int(d_count.item())
            assert np.array_equal(got, ref)
            assert np.all(d_edges[cnt:].cpu().numpy() == -1)   # nothing written past the count
    finally:
        ctx.close()


def test_noalloc_rejects_oversized_grid_and_small_buffer():
    import torch

    from paper_2409_13418_gb300 import build, odc
    build.build()
    d = torch.zeros(16, dtype=torch.int32, device="cuda")
    with pytest.raises(odc.OdcError) as e:
        odc.compact_edges_noalloc(d.data_ptr(), (512, 512, 512), d.data_ptr(), 4, d.data_ptr())
    assert e.value.status == 1
    # a grid with crossings and a one-edge buffer: the count is reported, OOM raised
    bits = np.zeros((5, 5, 1), np.uint32)
    bits[2, 2, 0] = 1 << 2                      # one inside vertex at (2, 2, 2): 6 crossing edges
    d_bits = torch.from_numpy(bits.reshape(-1).view(np.int32).copy()).cuda()
    with pytest.raises(odc.OdcError) as e:
        odc.compact_edges_noalloc(d_bits.data_ptr(), (4, 4, 4), d.data_ptr(), 1, d[8:].data_ptr())
    assert e.value.status == 2


def test_noalloc_count_stays_on_device_without_host_count():
    """Without a host count the call only queues its work: the count lands in
    the caller's device word, stream ordered, and matches odc_extract's."""
    import torch

    from paper_2409_13418_gb300 import build, inputs as I, odc
    build.build()
    ctx = odc.Context(0)
    try:
        src, grid = I.random_csg(8), I.cube_grid(72)
        ctx.extract(src, grid, steps_1d=8)
        bits, ref = ctx.debug("labels"), ctx.debug("edges")
        d_bits = torch.from_numpy(bits.view(np.int32).copy()).cuda()
        d_edges = torch.full((ref.size + 16,), -1, dtype=torch.int32, device="cuda")
        d_count = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        stream = torch.cuda.current_stream()
        for _ in range(2):
            assert odc.compact_edges_noalloc(d_bits.data_ptr(), grid.res, d_edges.data_ptr(), d_edges.numel(),
                                             d_count.data_ptr(), stream.cuda_stream, read_count=False) is None
            stream.synchronize()
            assert int(d_count.item()) == ref.size
            assert np.array_equal(d_edges[:ref.size].cpu().numpy().view(np.uint32), ref)
    finally:
        ctx.close()
