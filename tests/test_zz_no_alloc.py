"""The allocation-free quality entry point (lfd_quality_mip_static).

Some callers cannot allocate device memory: a host application that owns all
device memory and hands a plug-in fixed buffers, or a real-time loop that must
not stall on an allocation. For them the library computes the DCT entropy of a
projection image with its intermediates in a static device array. These tests
call it through the C ABI and compare it with lfd_quality, which computes the
same quantity from the volume with context-owned buffers, on two calls in a
row (the static array keeps the previous call's contents), and with the FP64
oracle's metric at the sizes the array is made for. They also check that the
calls really allocate nothing and that host pointers are refused. This file is
collected last on purpose.
"""
import numpy as np
import pytest

from oracle import metric
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


def _image(seed, H, W):
    """Sparse bright spots on a dim background, like a volume's z-maximum."""
    rng = np.random.default_rng(seed)
    img = rng.uniform(0.0, 0.05, (H, W))
    n = max(8, H * W // 4000)
    img[rng.integers(0, H, n), rng.integers(0, W, n)] += rng.uniform(0.5, 1.0, n)
    return img.astype(np.float32)


# (H, W, XS, YS): the large frame's sensor and region (Eqs. 7, 9-11 give 50),
# the array's limits, and a non-square image at the limits
@pytest.mark.parametrize("H,W,XS,YS", [(2025, 2025, 50, 50), (4096, 4096, 128, 128),
                                       (1000, 4096, 128, 31)])
def test_static_quality_matches_oracle(H, W, XS, YS):
    import torch
    lfd = lib()
    img = _image(H + W + XS, H, W)
    mip = torch.from_numpy(img).to("cuda:0")
    out = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    for l2_region in (1, 0):
        lfd.lfd_quality_mip_static(mip, H, W, XS, YS, l2_region, out)
        torch.cuda.synchronize()
        got = float(out.item())
        ref = metric.dct_entropy(img, XS, YS, bool(l2_region))
        assert abs(got - ref) <= TOL * abs(ref), (l2_region, got, ref)


def test_static_quality_allocates_nothing():
    """After a first call (which may load the module), further calls leave the
    device's free memory and torch's allocator untouched."""
    import torch
    lfd = lib()
    H, W, XS, YS = 615, 615, 15, 15
    mip = torch.from_numpy(_image(3, H, W)).to("cuda:0")
    out = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    vals = []
    for _ in range(2):                       # warm-up
        lfd.lfd_quality_mip_static(mip, H, W, XS, YS, 1, out)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    reserved0 = torch.cuda.memory_reserved()
    allocated0 = torch.cuda.memory_allocated()
    for _ in range(2):
        lfd.lfd_quality_mip_static(mip, H, W, XS, YS, 1, out)
        torch.cuda.synchronize()
        vals.append(float(out.item()))
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_reserved() == reserved0
    assert torch.cuda.memory_allocated() == allocated0
    assert vals[0] == vals[1]


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


def test_static_quality_rejects_host_pointers():
    """The entry point stages nothing, so host buffers are refused before any
    launch (a kernel given a host address would fault or read wrong memory)."""
    import torch
    lfd = lib()
    L = lfd.load()
    host_img = np.ones((8, 8), np.float32)
    host_out = np.zeros(1, np.float64)
    dev_img = torch.ones((8, 8), device="cuda:0")
    dev_out = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    himg = host_img.__array_interface__["data"][0]
    hout = host_out.__array_interface__["data"][0]
    assert L.lfd_quality_mip_static(himg, 8, 8, 4, 4, 1, dev_out.data_ptr(), None) == 1
    assert L.lfd_quality_mip_static(dev_img.data_ptr(), 8, 8, 4, 4, 1, hout, None) == 1
    with pytest.raises(ValueError):
        lfd.lfd_quality_mip_static(host_img, 8, 8, 4, 4, 1, dev_out)
    with pytest.raises(ValueError):
        lfd.lfd_quality_mip_static(dev_img, 8, 8, 4, 4, 1, torch.zeros(1, dtype=torch.float64))
    assert host_out[0] == 0.0
