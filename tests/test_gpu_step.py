"""RL iterations on the context's resident iterate (lfd_rl_load / lfd_rl_step /
lfd_rl_store) through the C ABI. Stepping must give what lfd_rl_iterate gives
for the same number of iterations (the same kernels on the same data; within
1e-6 relative L2, as batch against single frames), and the FP64 oracle's RL
within the path's tolerance, with the oracle's entropies."""
import numpy as np
import pytest

import oracle
from oracle import metric
from oracle import rl as orl
from paper_2208_11422_gb300 import synth

from gpu_util import Ctx, lib, rel_l2

pytestmark = pytest.mark.gpu

TOL_RL = {("fft", "fp32"): 1e-4, ("fft", "bf16x3"): 5e-4, ("direct", "fp32"): 1e-4,
          ("direct", "bf16x3"): 5e-4}
ENT_RTOL = {"fp32": 1e-5, "bf16x3": 1e-3}


@pytest.fixture(scope="module", autouse=True)
def _built():
    lib()


def _config0():
    g = synth.CONFIGS[0]
    psf = synth.make_psf(0)
    y = synth.poisson_data(oracle.forward(psf, g.nnum, synth.ground_truth(0)), g.scale,
                           g.background, 200)
    return g, psf, y


@pytest.mark.parametrize("variant,prec", list(TOL_RL))
def test_steps_equal_iterate_and_oracle(variant, prec):
    import torch
    g, psf, y = _config0()
    XS, YS = metric.region_size(g.nnum, g.H, g.W)
    n = g.iterations
    ref = orl.rl(psf, g.nnum, y, n, XS, YS)
    with Ctx(psf, g.nnum, g.H, g.W, variant=variant, precision=prec) as c:
        lfd = c.lfd
        v_it, _, _, ent_it, flux_it = c.rl(y, n)
        yd = torch.from_numpy(y).to(c.dev)
        v0 = torch.ones((g.nz, g.H, g.W), device=c.dev)
        lfd.lfd_rl_load(c.ctx, v0)
        ent, flux = [], []
        for _ in range(n):                       # one iteration per call
            e, f = lfd.lfd_rl_step(c.ctx, yd, 1)
            ent += e
            flux += f
        out = torch.empty_like(v0)
        lfd.lfd_rl_store(c.ctx, out)
        torch.cuda.synchronize()
        v_st = out.cpu().numpy()
    assert rel_l2(v_st, v_it) <= 1e-6
    np.testing.assert_allclose(ent, ent_it, rtol=1e-9)
    np.testing.assert_allclose(flux, flux_it, rtol=1e-9)
    e = rel_l2(v_st, ref.v)
    print("config 0 %s %s stepped: rel-L2 %.2e from the oracle" % (variant, prec, e))
    assert e <= TOL_RL[(variant, prec)]
    assert v_st.min() >= 0.0
    np.testing.assert_allclose(ent, ref.entropy, rtol=ENT_RTOL[prec])
    assert metric.predicted_iteration(ent) == ref.predicted


def test_host_buffers_and_multi_iteration_steps():
    """Host image and volumes; one call of n iterations equals n calls of one;
    a stepped run continues where the previous call stopped."""
    g, psf, y = _config0()
    with Ctx(psf, g.nnum, g.H, g.W, variant="fft", precision="bf16x3") as c:
        lfd = c.lfd
        v0 = np.ones((g.nz, g.H, g.W), np.float32)
        lfd.lfd_rl_load(c.ctx, v0)
        e3, _ = lfd.lfd_rl_step(c.ctx, y, 3)
        e2, _ = lfd.lfd_rl_step(c.ctx, y, 2)
        a = np.empty_like(v0)
        lfd.lfd_rl_store(c.ctx, a)
        lfd.lfd_rl_load(c.ctx, v0)
        e1 = []
        for _ in range(5):
            e1 += lfd.lfd_rl_step(c.ctx, y, 1)[0]
        b = np.empty_like(v0)
        lfd.lfd_rl_store(c.ctx, b)
        v_it, _, _, ent_it, _ = c.rl(y, 5)
    assert rel_l2(a, b) <= 1e-6 and rel_l2(a, v_it) <= 1e-6
    np.testing.assert_allclose(e3 + e2, e1, rtol=1e-9)
    np.testing.assert_allclose(e1, ent_it, rtol=1e-9)


def test_step_needs_a_loaded_iterate():
    g, psf, y = _config0()
    with Ctx(psf, g.nnum, g.H, g.W, variant="fft", precision="bf16x3") as c:
        L = c.lfd.load()
        yd = np.ascontiguousarray(y)
        yp = yd.__array_interface__["data"][0]
        assert L.lfd_rl_step(c.ctx, yp, 1, None, None, None) == 1      # nothing loaded
        c.lfd.lfd_rl_load(c.ctx, np.ones((g.nz, g.H, g.W), np.float32))
        assert L.lfd_rl_step(c.ctx, yp, 0, None, None, None) == 1      # n < 1
        assert L.lfd_rl_step(c.ctx, None, 1, None, None, None) == 1    # no image
        assert L.lfd_rl_step(c.ctx, yp, 1, None, None, None) == 0
        c.rl(y, 1)                                                     # reuses the buffers
        assert L.lfd_rl_step(c.ctx, yp, 1, None, None, None) == 1
