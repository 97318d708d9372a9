"""Accuracy of every projection path at the large frame (2025 x 2025 px, Nnum
15, 51 depths, PSF 345 px) against the FP64 oracle, dense on four seeded
256 x 256 crops: origins drawn with default_rng(300) uniformly over
[0, 2025 - 256]^2.

Each path computes the full-frame forward projection of the ground-truth
volume (5000 beads + 200 filaments) and the full-frame backprojection of a
ratio-like image (uniform in [0.5, 1.5]); the forward output is compared with
the oracle on every pixel of each crop, the backprojection at every depth of
each crop's voxels. The oracle values come from ``oracle.forward_crop`` and
``oracle.backward_block`` (the oracle's own sums over the crop, bit for bit
those of the full frame), computed in a background thread while the GPU works.

Bounds per projection (relative L2 per crop):
  FP32 (FFT and direct)             1e-5           (the FP32 bound)
  split BF16 (FFT and direct)       1e-4           (the split-BF16 bound)
  BF16 PSF spectra (FFT)            2^-9 ~ 2e-3    (one BF16 rounding per spectrum value)
  BF16 (direct)                     2^-8 ~ 3.9e-3  (both operands rounded to BF16)
  TF32 (direct)                     2^-10 ~ 9.8e-4 (both operands rounded to TF32)
The errors are printed for every path and crop."""
import threading

import numpy as np
import pytest

import oracle
from paper_2208_11422_gb300 import synth

from gpu_util import lib, rel_l2

pytestmark = pytest.mark.gpu

CROP = 256
NCROPS = 4
TOL = {("fft", "fp32"): 1e-5, ("fft", "bf16x3"): 1e-4, ("fft", "bf16"): 2.0 ** -9,
       ("direct", "fp32"): 1e-5, ("direct", "bf16x3"): 1e-4, ("direct", "bf16"): 2.0 ** -8,
       ("direct", "tf32"): 2.0 ** -10}


def crop_origins(H, W, n=NCROPS, size=CROP, seed=300):
    rng = np.random.default_rng(seed)
    return [(int(rng.integers(0, H - size + 1)), int(rng.integers(0, W - size + 1))) for _ in range(n)]


class _OracleCrops:
    """The oracle's forward and backward values on the crops, computed in a
    thread (the C oracle releases the interpreter lock)."""

    def __init__(self):
        g = synth.CONFIGS[2]
        self.g = g
        self.psf = synth.make_psf(2)
        self.v = synth.ground_truth(2).astype(np.float32)
        self.r = synth.random_image(7, g.H, g.W, 0.5, 1.5)
        self.origins = crop_origins(g.H, g.W)
        self.fwd, self.bwd = [], []
        self.err = None
        self.th = threading.Thread(target=self._run, daemon=True)
        self.th.start()

    def _run(self):
        try:
            g = self.g
            psf64 = self.psf.astype(np.float64)
            for (i0, j0) in self.origins:
                self.fwd.append(oracle.forward_crop(psf64, g.nnum, self.v, i0, i0 + CROP, j0, j0 + CROP))
                self.bwd.append(oracle.backward_block(psf64, g.nnum, self.r, 0, g.nz,
                                                      i0, i0 + CROP, j0, j0 + CROP))
        except Exception as e:  # reported by result()
            self.err = e

    def result(self):
        self.th.join()
        if self.err is not None:
            raise self.err
        return self.fwd, self.bwd


@pytest.fixture(scope="module")
def oracle_crops():
    lib()
    return _OracleCrops()


@pytest.mark.parametrize("variant,prec", list(TOL))
def test_large_frame_crops_match_oracle(oracle_crops, variant, prec):
    import torch
    from paper_2208_11422_gb300 import lfd
    oc = oracle_crops
    g = oc.g
    dev = torch.device("cuda:0")
    psf_d = torch.from_numpy(oc.psf).to(dev)
    ctx = lfd.lfd_create(psf_d, g.P, g.nnum, g.nz, g.H, g.W,
                         lfd.lfd_default_options(precision=prec, variant=variant))
    try:
        v = torch.from_numpy(oc.v).to(dev)
        r = torch.from_numpy(oc.r).to(dev)
        hv = torch.empty((g.H, g.W), device=dev)
        ht = torch.empty((g.nz, g.H, g.W), device=dev)
        lfd.lfd_forward(ctx, v, hv)
        lfd.lfd_backward(ctx, r, ht)
        torch.cuda.synchronize()
        got_f = [hv[i0:i0 + CROP, j0:j0 + CROP].cpu().numpy() for i0, j0 in oc.origins]
        got_b = [ht[:, i0:i0 + CROP, j0:j0 + CROP].cpu().numpy() for i0, j0 in oc.origins]
    finally:
        lfd.lfd_destroy(ctx)
        del psf_d
        torch.cuda.empty_cache()
    ref_f, ref_b = oc.result()
    ef = [rel_l2(a, b) for a, b in zip(got_f, ref_f)]
    eb = [rel_l2(a, b) for a, b in zip(got_b, ref_b)]
    print("2025 px %s %s: crops %s forward rel-L2 %s backward rel-L2 %s"
          % (variant, prec, oc.origins, ["%.2e" % e for e in ef], ["%.2e" % e for e in eb]))
    tol = TOL[(variant, prec)]
    assert max(ef) <= tol and max(eb) <= tol
