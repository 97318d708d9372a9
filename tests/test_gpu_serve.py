"""Serving (lfd_submit / lfd_poll): frames of different shapes on two
resident PSF sets, batched continuously. Each request's result must be the
same as when its frame is reconstructed alone by an lfd_ctx made for its shape
(same precision and FFT size), including its stopping iteration. One frame is
also checked against the FP64 oracle, and the queue / cancel / admission
errors are exercised on the host side of the server."""
import ctypes

import numpy as np
import pytest

import oracle
from oracle import metric
from oracle import rl as orl
from paper_2208_11422_gb300 import synth

from gpu_util import Ctx, lib, rel_l2

pytestmark = pytest.mark.gpu

TOL_ORACLE = {"fp32": 1e-4, "bf16x3": 5e-4}


@pytest.fixture(scope="module", autouse=True)
def _built():
    lib()


def psf_sets():
    """(nnum, nz, P, psf, max_lenslets) of two small PSF sets."""
    a = (5, 5, 25, synth.make_psf(0), 48)
    b = (3, 4, 15, synth.psf_gaussian_spots(3, 4, 5, 2, 0.8, 0.6, 1), 40)
    return [a, b]


# (set, Ly, Lx, photon scale): one, two and four tiles per frame at F = 32
FRAMES = [(0, 15, 15, 200.0), (1, 20, 25, 500.0), (0, 30, 12, 1000.0), (1, 31, 8, 150.0),
          (0, 40, 29, 300.0), (0, 9, 33, 2000.0), (1, 12, 12, 800.0), (0, 27, 27, 100.0)]


def frame_data(sets, k, set_i, ly, lx, scale):
    nnum, nz, P, psf, _ = sets[set_i]
    v = synth.beads(500 + k, nz, ly * nnum, lx * nnum, 12, 1.5, 0.4)
    return synth.poisson_data(oracle.forward(psf, nnum, v), scale, 2.0, 600 + k)


def make_server(lfd, prec, sets, **kw):
    opt = lfd.lfd_server_default_options(prec, opt_fft_size=32, **kw)
    srv = lfd.lfd_server_create(opt)
    ids = [lfd.lfd_server_add_psf(srv, psf, P, nnum, nz, L * nnum, L * nnum)
           for nnum, nz, P, psf, L in sets]
    return srv, ids


# (precision, frames per set, columns per contraction): 16 columns with at most
# 3 frames per set, or 64 columns with all of a set's frames at once (the
# contraction then takes 32-column chunks)
@pytest.mark.parametrize("prec,mf,mc", [("bf16x3", 3, 16), ("fp32", 3, 16), ("bf16x3", 8, 64),
                                        ("bf16", 8, 64)])
def test_results_in_the_mix_equal_results_alone(prec, mf, mc):
    import torch
    from paper_2208_11422_gb300 import lfd
    sets = psf_sets()
    n = 12
    ys = [frame_data(sets, k, *f) for k, f in enumerate(FRAMES)]
    srv, ids = make_server(lfd, prec, sets, max_frames_per_set=mf, max_cols=mc, max_iter=n)
    outs, reqs = [], []
    try:
        for k, (si, ly, lx, _) in enumerate(FRAMES):
            nnum, nz = sets[si][0], sets[si][1]
            y = torch.from_numpy(ys[k]).pin_memory() if k % 2 else torch.from_numpy(ys[k]).cuda()
            v = torch.empty((nz, ly * nnum, lx * nnum)).pin_memory() if k % 3 else \
                torch.empty((nz, ly * nnum, lx * nnum), device="cuda")
            outs.append(v)
            reqs.append(lfd.lfd_submit(srv, ids[si], y, v, max_iter=n, stop_at_predicted=True))
        res = [lfd.lfd_poll(srv, r, 120_000_000) for r in reqs]
        stats = lfd.lfd_server_stats_get(srv)
        err = lfd.lfd_server_last_error(srv)
    finally:
        lfd.lfd_server_destroy(srv)
    assert stats["completed"] == len(FRAMES) and stats["in_flight"] == 0, (stats, res, err)
    torch.cuda.synchronize()
    stopped = 0
    for k, (si, ly, lx, _) in enumerate(FRAMES):
        nnum, nz, P, psf, _ = sets[si]
        r = res[k]
        assert r is not None and r["status"] == lfd.LFD_OK, (k, r)
        with Ctx(psf, nnum, ly * nnum, lx * nnum, prec, variant="fft", fft_size=32) as c:
            v1, d1, p1, e1, _ = c.rl(ys[k], n, stop=True)
        assert (r["iters_done"], r["predicted"]) == (d1, p1), (k, r, d1, p1)
        stopped += d1 < n
        assert rel_l2(outs[k].cpu().numpy(), v1) <= 1e-6, k
        ran = r["iters_run"]
        np.testing.assert_allclose(r["entropy"][:ran], e1[:ran], rtol=1e-9)
        assert np.isnan(r["entropy"][ran:]).all()
    assert stopped >= 3   # frames leave the batch at their own iterations


@pytest.mark.parametrize("prec", ["bf16x3", "fp32"])
def test_served_frame_matches_oracle(prec):
    import torch
    from paper_2208_11422_gb300 import lfd
    sets = psf_sets()
    nnum, nz, P, psf, _ = sets[0]
    g = synth.CONFIGS[0]
    y = synth.poisson_data(oracle.forward(psf, nnum, synth.ground_truth(0)), g.scale, g.background, 200)
    n = 5
    srv, ids = make_server(lfd, prec, sets)
    try:
        v = torch.empty((nz, g.H, g.W), device="cuda")
        r = lfd.lfd_poll(srv, lfd.lfd_submit(srv, ids[0], torch.from_numpy(y).cuda(), v, max_iter=n,
                                              stop_at_predicted=False), 60_000_000)
    finally:
        lfd.lfd_server_destroy(srv)
    assert r["status"] == lfd.LFD_OK and r["iters_done"] == n and r["iters_run"] == n
    XS, YS = metric.region_size(nnum, g.H, g.W)
    ref = orl.rl(psf, nnum, y.astype(np.float64), n, XS, YS)
    assert rel_l2(v.cpu().numpy(), ref.v) <= TOL_ORACLE[prec]
    np.testing.assert_allclose(r["entropy"], ref.entropy, rtol=1e-3)


def test_queue_cancel_and_admission_errors():
    import torch
    from paper_2208_11422_gb300 import lfd
    L = lfd.load()
    sets = psf_sets()[:1]
    nnum, nz = sets[0][0], sets[0][1]
    # one frame in flight at a time and a queue of two
    srv, ids = make_server(lfd, "bf16x3", sets, max_frames_per_set=1, max_queue=2, max_iter=30)
    try:
        y = torch.from_numpy(frame_data(sets, 0, 0, 40, 40, 500.0)).cuda()
        keep, busy = [], 0
        for _ in range(8):
            v = torch.empty((nz, 200, 200), device="cuda")
            try:
                keep.append(lfd.lfd_submit(srv, ids[0], y, v, max_iter=30, stop_at_predicted=False))
            except lfd.LfdError as e:
                assert e.status == lfd.LFD_EBUSY
                busy += 1
        assert busy >= 1 and len(keep) >= 2
        last = keep[-1]
        assert lfd.lfd_poll(srv, last, 0) is None           # still queued: not ready
        assert lfd.lfd_cancel(srv, last) == lfd.LFD_OK
        r = lfd.lfd_poll(srv, last, 0)
        assert r["status"] == lfd.LFD_ECANCELED and r["iters_run"] == 0
        assert L.lfd_poll(srv, last.ticket, 0, None) == lfd.LFD_EINVAL
        first = lfd.lfd_poll(srv, keep[0], 120_000_000)
        assert first["status"] == lfd.LFD_OK and first["iters_done"] == 30
        assert lfd.lfd_cancel(srv, keep[0]) == lfd.LFD_EINVAL   # released
        for q in keep[1:-1]:
            assert lfd.lfd_poll(srv, q, 120_000_000)["status"] == lfd.LFD_OK
        # shape and set errors, and PSF sets only before the first submit
        v = torch.empty((nz, 75, 75), device="cuda")
        for sid, yy in ((ids[0], torch.empty((74, 75), device="cuda")),
                        (ids[0], torch.empty((250, 250), device="cuda")),
                        (7, torch.empty((75, 75), device="cuda"))):
            with pytest.raises(lfd.LfdError) as ei:
                lfd.lfd_submit(srv, sid, yy, v, max_iter=3)
            assert ei.value.status == lfd.LFD_EINVAL
        with pytest.raises(lfd.LfdError) as ei:
            lfd.lfd_server_add_psf(srv, sets[0][3], sets[0][2], nnum, nz, 75, 75)
        assert ei.value.status == lfd.LFD_EBUSY
        st = lfd.lfd_server_stats_get(srv)
        assert st["cancelled"] == 1 and st["rejected"] >= busy + 3
    finally:
        lfd.lfd_server_destroy(srv)


def test_frame_larger_than_the_arena_is_rejected():
    import torch
    from paper_2208_11422_gb300 import lfd
    sets = psf_sets()[:1]
    nnum, nz = sets[0][0], sets[0][1]
    srv, ids = make_server(lfd, "bf16x3", sets, arena_bytes=1 << 20)
    try:
        y = torch.zeros((200, 200), device="cuda")
        v = torch.empty((nz, 200, 200), device="cuda")
        with pytest.raises(lfd.LfdError) as ei:
            lfd.lfd_submit(srv, ids[0], y, v, max_iter=3)
        assert ei.value.status == lfd.LFD_ENOMEM
    finally:
        lfd.lfd_server_destroy(srv)
