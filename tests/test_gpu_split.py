"""Depth split (Section 2.1, Fig. 1: depth layers and their PSF slices divided
among GPUs) through the library: contexts over depth ranges, the split entry
points (lfd_split_load / _forward / _update / _store, lfd_quality_mip) and the
orchestration in paper_2208_11422_gb300.depth_split. Here the parts share one
GPU and are reduced in-process; the cross-process reductions are tested on CPU
(tests/test_dist_cpu.py).

* the partial forward projections of the parts sum to the full context's
  projection (and to the oracle's, within the precision's bound);
* split RL equals unsplit RL: the same entropies, flux and stopping
  iteration, and a volume within the precision's bound of the oracle."""
import os
import types

import numpy as np
import pytest

import oracle
from oracle import metric
from oracle import rl as orl
from paper_2208_11422_gb300 import synth

from gpu_util import lib, rel_l2

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
TOL_PROJ = {"fp32": 1e-5, "bf16x3": 1e-4}
TOL_RL = {"fp32": 1e-4, "bf16x3": 5e-4}
PATHS = [("fft", "fp32"), ("fft", "bf16x3"), ("direct", "fp32"), ("direct", "bf16x3")]


@pytest.fixture(scope="module", autouse=True)
def _built():
    lib()


def shards_for(psf_d, g, ranges, variant, prec):
    from paper_2208_11422_gb300 import depth_split, lfd
    opt = lfd.lfd_default_options(precision=prec, variant=variant)
    return [depth_split.LibraryShard(psf_d, g.P, g.nnum, z0, z1, g.H, g.W, opt) for z0, z1 in ranges]


@pytest.mark.parametrize("variant,prec", PATHS)
def test_partial_forward_projections_sum_to_the_full_projection(variant, prec):
    import torch
    from paper_2208_11422_gb300 import lfd
    N, Ly, Lx, Nz, k = 5, 9, 12, 7, 5
    H, W, P = Ly * N, Lx * N, k * N
    psf = synth.random_psf(51, N, Nz, P, density=0.8)
    v = synth.random_volume(52, Nz, H, W)
    dev = torch.device("cuda:0")
    psf_d = torch.from_numpy(psf).to(dev)
    vd = torch.from_numpy(v).to(dev)
    g = types.SimpleNamespace(P=P, nnum=N, H=H, W=W)
    ranges = [(0, 2), (2, 3), (3, 7)]
    shards = shards_for(psf_d, g, ranges, variant, prec)
    full = lfd.lfd_create(psf_d, P, N, Nz, H, W, lfd.lfd_default_options(precision=prec, variant=variant))
    try:
        hv = torch.zeros((H, W), device=dev)
        part = torch.empty((H, W), device=dev)
        for s, (z0, z1) in zip(shards, ranges):
            s.load(vd[z0:z1].contiguous())
            s.forward(part)
            hv += part
        ref = torch.empty((H, W), device=dev)
        lfd.lfd_forward(full, vd, ref)
        torch.cuda.synchronize()
        got, ref_h = hv.cpu().numpy(), ref.cpu().numpy()
    finally:
        for s in shards:
            s.close()
        lfd.lfd_destroy(full)
    e_full = rel_l2(got, ref_h)
    e_orc = rel_l2(got, oracle.forward(psf, N, v))
    print("%s %s: summed parts vs full context %.2e, vs oracle %.2e" % (variant, prec, e_full, e_orc))
    assert e_full <= TOL_PROJ[prec] and e_orc <= TOL_PROJ[prec]


def spread_frame():
    """The tiny workload with a frame whose entropy peaks at iteration 7."""
    g = synth.CONFIGS[0]
    psf = synth.make_psf(0)
    vt = synth.timelapse_beads(0, 1, 300, step_sigma=1.0)[0]
    y = synth.poisson_data(oracle.forward(psf, g.nnum, vt), 100.0, g.background, 310)
    return g, psf, y


@pytest.mark.parametrize("stop", [False, True])
@pytest.mark.parametrize("variant,prec", PATHS)
def test_split_rl_equals_unsplit_rl(variant, prec, stop):
    import torch
    from paper_2208_11422_gb300 import depth_split, lfd
    g, psf, y = spread_frame()
    n = 12
    XS, YS = metric.region_size(g.nnum, g.H, g.W)
    ref = orl.rl(psf, g.nnum, y, n, XS, YS, keep_iterates=True)
    dev = torch.device("cuda:0")
    psf_d = torch.from_numpy(psf).to(dev)
    yd = torch.from_numpy(y).to(dev)
    ranges = depth_split.depth_ranges(g.nz, 2)
    shards = shards_for(psf_d, g, ranges, variant, prec)
    try:
        for s, (z0, z1) in zip(shards, ranges):
            s.load(torch.ones((z1 - z0, g.H, g.W), device=dev))
        res = depth_split.split_rl(shards, yd, n, stop)
        v = torch.empty((g.nz, g.H, g.W), device=dev)
        for s, (z0, z1) in zip(shards, ranges):
            part = torch.empty((z1 - z0, g.H, g.W), device=dev)
            s.store(part, res.previous)
            v[z0:z1] = part
        v_split = v.cpu().numpy()
    finally:
        for s in shards:
            s.close()
    full = lfd.lfd_create(psf_d, g.P, g.nnum, g.nz, g.H, g.W,
                          lfd.lfd_default_options(precision=prec, variant=variant))
    try:
        v1 = torch.ones((g.nz, g.H, g.W), device=dev)
        done, pred, ent, flux = lfd.lfd_rl_iterate(full, yd, v1, n, stop)
        v_full = v1.cpu().numpy()
    finally:
        lfd.lfd_destroy(full)
    e_full = rel_l2(v_split, v_full)
    e_orc = rel_l2(v_split, ref.iterates[res.iters_done - 1])
    print("%s %s stop=%s: split done %d predicted %d (unsplit %d / %d, oracle %d); rel-L2 vs unsplit "
          "%.2e, vs oracle %.2e" % (variant, prec, stop, res.iters_done, res.predicted, done, pred,
                                    ref.predicted, e_full, e_orc))
    assert res.predicted == pred == ref.predicted
    assert res.iters_done == done
    assert e_orc <= TOL_RL[prec] and e_full <= TOL_RL[prec]
    ran = len(res.entropy)
    np.testing.assert_allclose(res.entropy, ent[:ran], rtol=1e-5 if prec == "fp32" else 1e-3)
    np.testing.assert_allclose(res.flux, flux[:ran], rtol=1e-5 if prec == "fp32" else 1e-4)


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_split_rl_mid_size_against_stored_oracle_run(prec):
    """The 615 px, 31-depth workload in two depth parts (FFT variant): sampled
    voxels after 10 iterations and the predicted iteration of the stored FP64
    oracle run."""
    import torch
    from paper_2208_11422_gb300 import depth_split
    d = np.load(os.path.join(GOLDEN, "lf_mid_615px_31z_psf165.npz"))
    g = synth.CONFIGS[1]
    psf = synth.make_psf(1)
    y = (d["y_counts"].astype(np.float64) + float(d["background"])).astype(np.float32)
    n = int(d["n_iter"])
    dev = torch.device("cuda:0")
    psf_d = torch.from_numpy(psf).to(dev)
    ranges = depth_split.depth_ranges(g.nz, 2)
    shards = shards_for(psf_d, g, ranges, "fft", prec)
    try:
        for s, (z0, z1) in zip(shards, ranges):
            s.load(torch.ones((z1 - z0, g.H, g.W), device=dev))
        res = depth_split.split_rl(shards, torch.from_numpy(y).to(dev), n)
        v = torch.empty((g.nz, g.H, g.W), device=dev)
        for s, (z0, z1) in zip(shards, ranges):
            part = torch.empty((z1 - z0, g.H, g.W), device=dev)
            s.store(part)
            v[z0:z1] = part
        v = v.cpu().numpy()
    finally:
        for s in shards:
            s.close()
    vox = d["sample_vox"]
    e = rel_l2(v[vox[:, 0], vox[:, 1], vox[:, 2]], d["v_last"])
    print("615 px in 2 depth parts, fft %s: sampled rel-L2 %.2e, predicted %d (oracle %d)"
          % (prec, e, res.predicted, int(d["predicted"])))
    assert e <= TOL_RL[prec]
    assert res.predicted == int(d["predicted"])
    np.testing.assert_allclose(res.flux, d["flux"], rtol=1e-5 if prec == "fp32" else 1e-4)


def test_split_calls_check_their_state():
    import torch
    from paper_2208_11422_gb300 import lfd
    g, psf, y = spread_frame()
    dev = torch.device("cuda:0")
    ctx = lfd.lfd_create(torch.from_numpy(psf).to(dev), g.P, g.nnum, g.nz, g.H, g.W,
                         lfd.lfd_default_options(variant="fft"))
    try:
        hv = torch.zeros((g.H, g.W), device=dev)
        with pytest.raises(lfd.LfdError):          # nothing loaded yet
            lfd.lfd_split_forward(ctx, hv)
        lfd.lfd_split_load(ctx, np.ones((g.nz, g.H, g.W), np.float32))   # host volume
        v = np.zeros((g.nz, g.H, g.W), np.float32)
        with pytest.raises(lfd.LfdError):          # no update yet: no previous iterate
            lfd.lfd_split_store(ctx, v, previous=True)
        lfd.lfd_split_store(ctx, v)
        assert np.all(v == 1.0)
        with pytest.raises(ValueError):            # device memory required
            lfd.lfd_split_forward(ctx, torch.zeros((g.H, g.W)))
        lfd.lfd_forward(ctx, np.ones((g.nz, g.H, g.W), np.float32), np.zeros((g.H, g.W), np.float32))
        with pytest.raises(lfd.LfdError):          # lfd_forward reused the iterate buffers
            lfd.lfd_split_forward(ctx, hv)
    finally:
        lfd.lfd_destroy(ctx)
