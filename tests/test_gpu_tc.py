"""Parity of the tensor-core path (tcgen05: BF16, split BF16 and TF32) with the
FP64 oracle, through the C ABI.

Split BF16 (x = hi + lo, products hi*hi + hi*lo + lo*hi, FP32 accumulation):
relative L2 <= 1e-4 per projection and <= 5e-4 after RL iterations, predicted
iteration equal to the oracle's. Plain BF16: the error is reported and held
to <= 1e-2 per projection and <= 1e-2 after the iterations (BF16 keeps 8
significant bits, so single products carry ~2^-9 relative error). TF32 (PSF,
iterate and ratio rounded to nearest with a 10-bit mantissa, unit roundoff
2^-11): a product of two rounded non-negative operands is within 2^-10 of the
exact one, and so is a sum of such products, so each projection is held to
2^-10; after RL iterations the BF16 bound 1e-2 applies and the error is
reported.
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
TOL_PROJ = {"bf16x3": 1e-4, "bf16": 1e-2, "tf32": 2.0 ** -10}
TOL_RL = {"bf16x3": 5e-4, "bf16": 1e-2, "tf32": 1e-2}


@pytest.fixture(scope="module", autouse=True)
def _built():
    lib()


SHAPES = [
    (5, 15, 15, 5, 5),     # the tiny workload's geometry
    (5, 7, 12, 3, 5),      # non-square, tiles partly filled
    (1, 20, 17, 2, 7),     # Nnum = 1
    (3, 9, 9, 4, 1),       # PSF of one lenslet
    (5, 3, 3, 2, 9),       # PSF wider than the sensor
    (15, 5, 7, 31, 11),    # 225 phases: the widest forward tile (240 columns)
    (5, 40, 40, 5, 5),     # several row tiles
    (15, 3, 4, 3, 3),      # column tile of 704 channels: ragged last tile
]


@pytest.mark.parametrize("prec", ["bf16x3", "bf16", "tf32"])
@pytest.mark.parametrize("shape", SHAPES)
def test_projections_match_oracle(shape, prec):
    N, Ly, Lx, Nz, k = shape
    H, W, P = Ly * N, Lx * N, k * N
    psf = synth.random_psf(21, N, Nz, P, density=0.8)
    v = synth.random_volume(22, Nz, H, W)
    r = synth.random_image(23, H, W, 0.1, 2.0)
    with Ctx(psf, N, H, W, precision=prec) as c:
        hv = c.forward(v)
        ht = c.backward(r)
    ef = rel_l2(hv, oracle.forward(psf, N, v))
    eb = rel_l2(ht, oracle.backward(psf, N, r))
    print("%s %s forward %.2e backward %.2e" % (shape, prec, ef, eb))
    assert ef <= TOL_PROJ[prec] and eb <= TOL_PROJ[prec]


@pytest.mark.parametrize("prec", ["bf16x3", "bf16", "tf32"])
def test_rl_config0(prec):
    g = synth.CONFIGS[0]
    psf = synth.make_psf(0)
    y = synth.poisson_data(oracle.forward(psf, g.nnum, synth.ground_truth(0)), g.scale,
                           g.background, 200)
    XS, YS = metric.region_size(g.nnum, g.H, g.W)
    ref = orl.rl(psf, g.nnum, y, g.iterations, XS, YS)
    with Ctx(psf, g.nnum, g.H, g.W, precision=prec) as c:
        v, done, pred, ent, flux = c.rl(y, g.iterations)
    e = rel_l2(v, ref.v)
    print("config 0 %s: rel-L2 %.2e after %d iterations, predicted %d (oracle %d)"
          % (prec, e, done, pred, ref.predicted))
    assert e <= TOL_RL[prec]
    assert v.min() >= 0.0
    if prec == "bf16x3":
        assert pred == ref.predicted
        np.testing.assert_allclose(ent, ref.entropy, rtol=1e-3)


@pytest.mark.parametrize("prec", ["bf16x3", "bf16", "tf32"])
def test_rl_config1_against_stored_oracle_run(prec):
    d = np.load(os.path.join(GOLDEN, "lf_mid_615px_31z_psf165.npz"))
    g = synth.CONFIGS[1]
    psf = synth.make_psf(1)
    y = (d["y_counts"].astype(np.float64) + float(d["background"])).astype(np.float32)
    vox = d["sample_vox"]
    with Ctx(psf, g.nnum, g.H, g.W, precision=prec) as c:
        v, done, pred, ent, flux = c.rl(y, int(d["n_iter"]))
    e = rel_l2(v[vox[:, 0], vox[:, 1], vox[:, 2]], d["v_last"])
    print("config 1 %s: sampled rel-L2 %.2e after %d iterations, predicted %d (oracle %d)"
          % (prec, e, done, pred, int(d["predicted"])))
    assert e <= TOL_RL[prec]
    if prec == "bf16x3":
        assert pred == int(d["predicted"])
        np.testing.assert_allclose(ent, d["entropy"], rtol=1e-3)
        np.testing.assert_allclose(flux, d["flux"], rtol=1e-4)


@pytest.mark.parametrize("prec", ["bf16x3", "bf16", "tf32"])
def test_full_size_sampled_projections(prec):
    """2025x2025 px, 51 depths, PSF 345 px: sampled outputs against the oracle."""
    g = synth.CONFIGS[2]
    psf = synth.make_psf(2)
    v = synth.beads(102, g.nz, g.H, g.W, g.beads, g.bead_radius, g.amp_lo).astype(np.float32)
    r = synth.random_image(7, g.H, g.W, 0.5, 1.5)
    pix = synth.sample_indices(8, 256, (g.H, g.W))
    vox = synth.sample_indices(9, 256, (g.nz, g.H, g.W))
    pix[:4] = [[0, 0], [g.H - 1, g.W - 1], [0, g.W - 1], [g.H - 1, 0]]
    vox[:2] = [[0, 0, 0], [g.nz - 1, g.H - 1, g.W - 1]]
    with Ctx(psf, g.nnum, g.H, g.W, precision=prec) as c:
        hv = c.forward(v)
        ht = c.backward(r)
    ef = rel_l2(hv[pix[:, 0], pix[:, 1]], oracle.forward_at(psf, g.nnum, v, pix))
    eb = rel_l2(ht[vox[:, 0], vox[:, 1], vox[:, 2]], oracle.backward_at(psf, g.nnum, r, vox))
    print("config 2 %s: sampled forward %.2e backward %.2e" % (prec, ef, eb))
    assert ef <= TOL_PROJ[prec] and eb <= TOL_PROJ[prec]


def test_flux_invariant_holds_in_split_bf16():
    """sum(H^T1 v^k) = sum(y Hv/(Hv+eps)) ~= sum(y) for every iterate."""
    g = synth.CONFIGS[0]
    psf = synth.make_psf(0)
    y = synth.poisson_data(oracle.forward(psf, g.nnum, synth.ground_truth(0)), g.scale,
                           g.background, 200)
    with Ctx(psf, g.nnum, g.H, g.W, precision="bf16x3") as c:
        _, _, _, _, flux = c.rl(y, 4)
    total = float(np.sum(y.astype(np.float64)))
    for f in flux:
        assert abs(f - total) <= 1e-4 * total
