"""Parity of the FP32 GPU path (CUDA cores) with the FP64 oracle, through the C ABI.

Tolerances (relative L2): 1e-5 per projection, 1e-4 after RL iterations; the
predicted iteration must equal the oracle's. Index work (the PSF repack) is
checked bit-exactly with delta inputs.
"""
import os

import numpy as np
import pytest

import oracle
from oracle import metric
from oracle import rl as orl
from paper_2208_11422_gb300 import synth

from gpu_util import Ctx, lib, rel_l2

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module", autouse=True)
def _built():
    lib()


# (Nnum, lenslets y, lenslets x, Nz, PSF lenslets): tiny, ragged, degenerate
SHAPES = [
    (5, 15, 15, 5, 5),     # the tiny workload's geometry
    (5, 7, 12, 3, 5),      # non-square, tiles partly filled
    (1, 40, 33, 2, 7),     # Nnum = 1: plain 2-D convolution per depth
    (3, 9, 9, 4, 1),       # PSF of one lenslet
    (5, 3, 3, 2, 9),       # PSF wider than the sensor
    (15, 5, 7, 31, 11),    # mid-size PSF and depths on a small sensor
    (5, 40, 40, 5, 5),     # several output tiles
    (3, 1, 1, 1, 1),       # a single lenslet
]


@pytest.mark.parametrize("shape", SHAPES)
def test_projections_match_oracle(shape):
    N, Ly, Lx, Nz, k = shape
    H, W, P = Ly * N, Lx * N, k * N
    psf = synth.random_psf(21, N, Nz, P, density=0.8)
    v = synth.random_volume(22, Nz, H, W)
    r = synth.random_image(23, H, W, 0.1, 2.0)
    with Ctx(psf, N, H, W) as c:
        hv = c.forward(v)
        ht = c.backward(r)
    assert rel_l2(hv, oracle.forward(psf, N, v)) <= 1e-5
    assert rel_l2(ht, oracle.backward(psf, N, r)) <= 1e-5


@pytest.mark.parametrize("pos", [(0, 0, 0), (2, 7, 13), (4, 74, 74), (1, 37, 0)])
def test_delta_voxel_is_exact(pos):
    """A unit voxel projects to its own PSF slice, bit for bit (repack index check)."""
    g = synth.CONFIGS[0]
    psf = synth.make_psf(0)
    v = np.zeros((g.nz, g.H, g.W), np.float32)
    v[pos] = 1.0
    with Ctx(psf, g.nnum, g.H, g.W) as c:
        hv = c.forward(v)
    assert np.array_equal(hv, oracle.forward(psf, g.nnum, v).astype(np.float32))


def test_backward_of_delta_pixel_is_exact():
    g = synth.CONFIGS[0]
    psf = synth.make_psf(0)
    r = np.zeros((g.H, g.W), np.float32)
    r[31, 44] = 1.0
    with Ctx(psf, g.nnum, g.H, g.W) as c:
        ht = c.backward(r)
    assert np.array_equal(ht, oracle.backward(psf, g.nnum, r).astype(np.float32))


def test_host_and_device_pointers_agree():
    g = synth.CONFIGS[0]
    psf = synth.make_psf(0)
    v = synth.random_volume(5, g.nz, g.H, g.W)
    y = synth.random_image(6, g.H, g.W, 1, 3)
    with Ctx(psf, g.nnum, g.H, g.W) as c:
        dev_out = c.forward(v)
        host_out = np.empty((g.H, g.W), np.float32)
        c.lfd.lfd_forward(c.ctx, v, host_out)
        assert np.array_equal(dev_out, host_out)
        vh = np.ones((g.nz, g.H, g.W), np.float32)
        c.lfd.lfd_rl_iterate(c.ctx, y, vh, 3)
        vd, *_ = c.rl(y, 3)
        assert np.array_equal(vh, vd)


def config0_data():
    g = synth.CONFIGS[0]
    psf = synth.make_psf(0)
    y = synth.poisson_data(oracle.forward(psf, g.nnum, synth.ground_truth(0)), g.scale,
                           g.background, 200)
    return g, psf, y


def test_rl_config0_matches_oracle():
    g, psf, y = config0_data()
    XS, YS = metric.region_size(g.nnum, g.H, g.W)
    ref = orl.rl(psf, g.nnum, y, g.iterations, XS, YS)
    with Ctx(psf, g.nnum, g.H, g.W) as c:
        v, done, pred, ent, flux = c.rl(y, g.iterations)
    assert done == g.iterations
    assert rel_l2(v, ref.v) <= 1e-4
    np.testing.assert_allclose(ent, ref.entropy, rtol=1e-5)
    np.testing.assert_allclose(flux, ref.flux, rtol=1e-5)
    assert pred == ref.predicted
    assert v.min() >= 0.0


def test_rl_resume_and_stop_are_exact():
    """Two calls of 2 + 3 iterations equal one call of 5, bit for bit; the
    stopping run returns the same bits as a run of exactly n* iterations."""
    g, psf, y = config0_data()
    with Ctx(psf, g.nnum, g.H, g.W) as c:
        v5, *_ = c.rl(y, 5)
        v2, *_ = c.rl(y, 2)
        v23, *_ = c.rl(y, 3, v0=v2)
        assert np.array_equal(v5, v23)
        vs, done, pred, ent, _ = c.rl(y, 8, stop=True)
        E = [e for e in ent if not np.isnan(e)]
        assert done == pred == metric.predicted_iteration(E)
        vn, *_ = c.rl(y, done)
        assert np.array_equal(vs, vn)


def test_rl_config1_matches_stored_oracle_run():
    """Mid-size workload (615x615 px, 31 depths, PSF 165 px), 10 iterations,
    against the oracle run stored by tests/golden/make_lf_mid_615px.py."""
    d = np.load(os.path.join(GOLDEN, "lf_mid_615px_31z_psf165.npz"))
    g = synth.CONFIGS[1]
    psf = synth.make_psf(1)
    y = (d["y_counts"].astype(np.float64) + float(d["background"])).astype(np.float32)
    vox = d["sample_vox"]
    with Ctx(psf, g.nnum, g.H, g.W) as c:
        v, done, pred, ent, flux = c.rl(y, int(d["n_iter"]))
        take = v[vox[:, 0], vox[:, 1], vox[:, 2]]
        assert rel_l2(take, d["v_last"]) <= 1e-4
        np.testing.assert_allclose(ent, d["entropy"], rtol=1e-5)
        np.testing.assert_allclose(flux, d["flux"], rtol=1e-5)
        assert pred == int(d["predicted"])
        vs, done_s, pred_s, _, _ = c.rl(y, int(d["n_iter"]), stop=True)
        assert done_s == pred_s == int(d["predicted"])
        assert rel_l2(vs[vox[:, 0], vox[:, 1], vox[:, 2]], d["v_pred"]) <= 1e-4


@pytest.mark.parametrize("l2_region", [1, 0])
def test_quality_matches_oracle(l2_region):
    g = synth.CONFIGS[0]
    psf = synth.make_psf(0)
    v = synth.ground_truth(0).astype(np.float32)
    with Ctx(psf, g.nnum, g.H, g.W, l2_over_region=l2_region) as c:
        e = c.lfd.lfd_quality(c.ctx, v)
        XS, YS = c.lfd.lfd_get_geometry(c.ctx)["XS"], c.lfd.lfd_get_geometry(c.ctx)["YS"]
    ref = metric.dct_entropy(metric.mip_z(v), XS, YS, bool(l2_region))
    assert abs(e - ref) <= 1e-9 * abs(ref)


@pytest.mark.parametrize("cfg", [1, 2])
def test_full_size_sampled_projections(cfg):
    """Full-size frames (615 and 2025 px): sampled outputs against the oracle's
    per-output sums."""
    g = synth.CONFIGS[cfg]
    psf = synth.make_psf(cfg)
    v = synth.beads(100 + cfg, g.nz, g.H, g.W, g.beads, g.bead_radius, g.amp_lo).astype(np.float32)
    r = synth.random_image(7, g.H, g.W, 0.5, 1.5)
    pix = synth.sample_indices(8, 256, (g.H, g.W))
    vox = synth.sample_indices(9, 256, (g.nz, g.H, g.W))
    # make sure the edges are sampled too
    pix[:4] = [[0, 0], [g.H - 1, g.W - 1], [0, g.W - 1], [g.H - 1, 0]]
    vox[:2] = [[0, 0, 0], [g.nz - 1, g.H - 1, g.W - 1]]
    with Ctx(psf, g.nnum, g.H, g.W) as c:
        hv = c.forward(v)
        ht = c.backward(r)
    assert rel_l2(hv[pix[:, 0], pix[:, 1]], oracle.forward_at(psf, g.nnum, v, pix)) <= 1e-5
    assert rel_l2(ht[vox[:, 0], vox[:, 1], vox[:, 2]], oracle.backward_at(psf, g.nnum, r, vox)) <= 1e-5


def test_invalid_calls_return_errors():
    g = synth.CONFIGS[0]
    psf = synth.make_psf(0)
    with Ctx(psf, g.nnum, g.H, g.W) as c:
        L = c.lfd.load()
        assert L.lfd_rl_iterate(c.ctx, None, None, 1, 0, None, None, None, None, None) == c.lfd.LFD_EINVAL
        y = np.ones((g.H, g.W), np.float32)
        v = np.ones((g.nz, g.H, g.W), np.float32)
        assert L.lfd_rl_iterate(c.ctx, y.ctypes.data, v.ctypes.data, 0, 0, None, None, None, None,
                                None) == c.lfd.LFD_EINVAL
        assert "n < 1" in c.lfd.lfd_last_error(c.ctx)
