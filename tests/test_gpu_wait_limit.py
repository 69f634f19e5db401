"""Failure detection of the tensor-core pipelines: an expired device wait
comes back as ODC_ERR_TIMEOUT and leaves the context usable.

The wait is made to run out the way a real dependency would fail to arrive:
the kernels are held behind a device go flag that nothing sets, under a
short limit.  Nothing traps, faults or hangs: the kernel's own bounded wait
gives up, every role of the CTA stops, the loads and tensor-core operations
already started are waited for, and TMEM is released.  The next call with
the default limit and no gate gives the same mesh as before, byte for byte.
"""
import numpy as np
import pytest

from paper_2409_13418_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_expired_wait_returns_timeout_and_context_recovers():
    import torch

    from paper_2409_13418_gb300 import build, odc
    build.build()
    mlp, g = I.envelope_mlp(0), I.cube_grid(40)
    with odc.Context(0) as ctx:
        v0, t0 = ctx.extract(mlp, g, steps_1d=12, precision=odc.PREC_BF16, band=0.03).to_host()
        never = torch.zeros(1, dtype=torch.int32, device="cuda")    # a go flag nothing sets
        torch.cuda.synchronize()
        ctx.set_wait_limit(2_000_000, never.data_ptr())               # 2 ms
        with pytest.raises(odc.OdcError) as e:
            ctx.extract(mlp, g, steps_1d=12, precision=odc.PREC_BF16, band=0.03)
        assert e.value.status == 4, e.value       # ODC_ERR_TIMEOUT
        # the point evaluation path reports it too
        pts = np.random.default_rng(0).uniform(-1, 1, (4096, 3)).astype(np.float32)
        with pytest.raises(odc.OdcError) as e:
            ctx.eval_points(mlp, pts, precision=odc.PREC_BF16, band=0.0)
        assert e.value.status == 4
        ctx.set_wait_limit(0, None)
        v1, t1 = ctx.extract(mlp, g, steps_1d=12, precision=odc.PREC_BF16, band=0.03).to_host()
        assert v1.tobytes() == v0.tobytes() and np.array_equal(t1, t0)
        # a gate that is set lets the kernels through under the short limit
        go = torch.ones(1, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        ctx.set_wait_limit(50_000_000, go.data_ptr())
        v2, t2 = ctx.extract(mlp, g, steps_1d=12, precision=odc.PREC_BF16, band=0.03).to_host()
        ctx.set_wait_limit(0, None)
        assert v2.tobytes() == v0.tobytes() and np.array_equal(t2, t0)
