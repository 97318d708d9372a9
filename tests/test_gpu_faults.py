"""Failure detection without a GPU fault: a bounded device wait that can never
complete gives up, reports its error word and leaves the context usable;
host-side allocation-failure injection makes calls fail with LFD_ENOMEM and
leaves contexts and servers usable; lfd_poll's timeout expires on a request
that is still running."""
import numpy as np
import pytest

import oracle
from paper_2208_11422_gb300 import synth

from gpu_util import Ctx, lib, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    lib()


def tiny():
    g = synth.CONFIGS[0]
    psf = synth.make_psf(0)
    v = synth.ground_truth(0)
    y = synth.poisson_data(oracle.forward(psf, g.nnum, v), g.scale, g.background, 200)
    return g, psf, y


def test_bounded_wait_gives_up_and_the_context_stays_usable():
    from paper_2208_11422_gb300 import lfd
    st, code = lfd.lfd_selftest_bounded_wait(20_000_000)   # 20 ms
    assert st == lfd.LFD_ETIMEDOUT and code == 77
    g, psf, y = tiny()
    v = synth.random_volume(5, g.nz, g.H, g.W)
    with Ctx(psf, g.nnum, g.H, g.W, "bf16x3", variant="fft") as c:
        assert rel_l2(c.forward(v), oracle.forward(psf, g.nnum, v.astype(np.float64))) <= 1e-4


def test_injected_allocation_failure_in_create():
    import torch
    from paper_2208_11422_gb300 import lfd
    g, psf, _ = tiny()
    psf_d = torch.from_numpy(psf).cuda()
    for variant in ("fft", "direct"):
        lfd.lfd_debug_fail_allocs(1)
        try:
            with pytest.raises(lfd.LfdError) as ei:
                lfd.lfd_create(psf_d, g.P, g.nnum, g.nz, g.H, g.W, lfd.lfd_default_options(variant=variant))
            assert ei.value.status == lfd.LFD_ENOMEM
        finally:
            lfd.lfd_debug_fail_allocs(0)
        ctx = lfd.lfd_create(psf_d, g.P, g.nnum, g.nz, g.H, g.W, lfd.lfd_default_options(variant=variant))
        lfd.lfd_destroy(ctx)


def test_injected_allocation_failure_leaves_the_context_usable():
    import torch
    from paper_2208_11422_gb300 import lfd
    g, psf, y = tiny()
    with Ctx(psf, g.nnum, g.H, g.W, "fp32", variant="fft") as c:
        # reference: device buffers (no staging allocation)
        v_ref, *_ = c.rl(y, 3)
        # host buffers need the context's staging buffers: fail their allocation once
        y_h = np.ascontiguousarray(y, np.float32)
        v_h = np.ones((g.nz, g.H, g.W), np.float32)
        lfd.lfd_debug_fail_allocs(1)
        try:
            with pytest.raises(lfd.LfdError) as ei:
                lfd.lfd_rl_iterate(c.ctx, y_h, v_h, 3)
            assert ei.value.status == lfd.LFD_ENOMEM
        finally:
            lfd.lfd_debug_fail_allocs(0)
        assert (v_h == 1.0).all()
        lfd.lfd_rl_iterate(c.ctx, y_h, v_h, 3)
        torch.cuda.synchronize()
        assert rel_l2(v_h, v_ref) <= 1e-6


def test_server_arena_failure_then_recovery_and_poll_timeout():
    import torch
    from paper_2208_11422_gb300 import lfd
    g, psf, y = tiny()
    srv = lfd.lfd_server_create(lfd.lfd_server_default_options("bf16x3", opt_fft_size=32))
    try:
        sid = lfd.lfd_server_add_psf(srv, psf, g.P, g.nnum, g.nz, 300, 300)
        big = torch.from_numpy(synth.random_image(3, 300, 300)).cuda()
        v = torch.empty((g.nz, 300, 300), device="cuda")
        lfd.lfd_debug_fail_allocs(1)   # the arena is allocated at the first submit
        try:
            with pytest.raises(lfd.LfdError) as ei:
                lfd.lfd_submit(srv, sid, big, v, max_iter=30, stop_at_predicted=False)
            assert ei.value.status == lfd.LFD_ENOMEM
        finally:
            lfd.lfd_debug_fail_allocs(0)
        r = lfd.lfd_submit(srv, sid, big, v, max_iter=30, stop_at_predicted=False)
        assert lfd.lfd_poll(srv, r, 1000) is None      # 1 ms: 30 iterations are not done yet
        res = lfd.lfd_poll(srv, r, 120_000_000)
        assert res["status"] == lfd.LFD_OK and res["iters_done"] == 30
    finally:
        lfd.lfd_server_destroy(srv)
