"""The allocation-free quality entry point (lfd_quality_mip_static).

Some callers cannot allocate device memory: a host application that owns all
device memory and hands a plug-in fixed buffers, or a real-time loop that must
not stall on an allocation. For them the library computes the DCT entropy of a
projection image with its intermediates in a static device array. These tests
call it through the C ABI and compare it with lfd_quality, which computes the
same quantity from the volume with context-owned buffers, on two calls in a
row (the static array keeps the previous call's contents). This file is
collected last on purpose.
"""
import numpy as np
import pytest

from paper_2208_11422_gb300 import synth

from gpu_util import Ctx, lib

pytestmark = pytest.mark.gpu

TOL = 1e-9   # relative, as for lfd_quality against the oracle


@pytest.mark.parametrize("l2_region", [1, 0])
def test_static_quality_matches_context_quality(l2_region):
    import torch
    lib()
    g = synth.CONFIGS[0]
    psf = synth.make_psf(0)
    vols = [synth.ground_truth(0).astype(np.float32),
            synth.random_volume(77, g.nz, g.H, g.W, 0.0, 3.0)]
    with Ctx(psf, g.nnum, g.H, g.W, l2_over_region=l2_region) as c:
        geo = c.lfd.lfd_get_geometry(c.ctx)
        out = torch.zeros(1, dtype=torch.float64, device=c.dev)
        for v in vols:                       # two calls in a row
            ref = c.lfd.lfd_quality(c.ctx, v)
            mip = torch.from_numpy(v).to(c.dev).amax(dim=0).contiguous()
            c.lfd.lfd_quality_mip_static(mip, g.H, g.W, geo["XS"], geo["YS"], l2_region, out)
            torch.cuda.synchronize()
            got = float(out.item())
            assert abs(got - ref) <= TOL * abs(ref), (got, ref)


def test_static_quality_rejects_sizes_beyond_its_scratch():
    import torch
    L = lib().load()
    mip = torch.ones((8, 8), device="cuda:0")
    out = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    ok = L.lfd_quality_mip_static(mip.data_ptr(), 8, 8, 4, 4, 1, out.data_ptr(), None)
    assert ok == 0
    assert L.lfd_quality_mip_static(mip.data_ptr(), 5000, 8, 4, 4, 1, out.data_ptr(), None) == 1
    assert L.lfd_quality_mip_static(mip.data_ptr(), 8, 8, 9, 4, 1, out.data_ptr(), None) == 1
    assert L.lfd_quality_mip_static(mip.data_ptr(), 4096, 4096, 129, 4, 1, out.data_ptr(), None) == 1
