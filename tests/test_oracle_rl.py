"""Pins for the oracle's Richardson-Lucy iteration."""
import numpy as np
import pytest
from scipy.signal import convolve2d

from oracle import rl as orl
from paper_2208_11422_gb300 import synth


def test_delta_psf_one_depth_gives_data():
    """Delta PSF, Nz = 1: H = identity, H^T 1 = 1, so v^1 = 1 * y / (1 + eps)."""
    N, L, P = 3, 4, 3
    H = W = N * L
    psf = np.zeros((1, N, N, P, P))
    psf[..., 1, 1] = 1.0
    y = synth.random_image(1, H, W, 1.0, 5.0).astype(np.float64)
    res = orl.rl(psf, N, y, 1, 2, 2)
    np.testing.assert_allclose(res.v[0], y / (1.0 + orl.EPS), rtol=1e-15)


def test_delta_psf_many_depths_splits_evenly():
    """Delta PSF, Nz depths: Hv^0 = Nz, so v^1_z = y / (Nz + eps) in every depth."""
    N, L, P, Nz = 3, 3, 9, 4
    H = W = N * L
    psf = np.zeros((Nz, N, N, P, P))
    psf[..., 4, 4] = 1.0
    y = synth.random_image(2, H, W, 0.5, 2.0).astype(np.float64)
    res = orl.rl(psf, N, y, 1, 2, 2)
    for z in range(Nz):
        np.testing.assert_allclose(res.v[z], y / (Nz + orl.EPS), rtol=1e-15)


def test_nnum1_single_depth_is_textbook_rl():
    """Nnum = 1, Nz = 1 reduces to 2-D RL with one kernel K:
    v <- v * conv(y / (conv(v, K) + eps), flip K) / conv(1, flip K)."""
    H, W, P = 17, 13, 5
    K = synth.random_psf(3, 1, 1, P)[0, 0, 0].astype(np.float64)
    y = synth.random_image(4, H, W, 0.2, 3.0).astype(np.float64)
    Kf = K[::-1, ::-1]
    v = np.ones((H, W))
    norm = convolve2d(np.ones((H, W)), Kf, mode="same")
    for _ in range(3):
        v = v * convolve2d(y / (convolve2d(v, K, mode="same") + orl.EPS), Kf, mode="same") / norm
    res = orl.rl(K[None, None, None], 1, y, 3, 2, 2)
    np.testing.assert_allclose(res.v[0], v, rtol=1e-12)


def test_nonnegative_and_flux_invariant(orc):
    """sum(H^T1 * v^k) = <v^{k-1}, H^T r> = <H v^{k-1}, r> = sum y Hv/(Hv+eps)."""
    g = synth.CONFIGS[0]
    psf = synth.make_psf(0)
    vt = synth.ground_truth(0)
    y = synth.poisson_data(orc.forward(psf, g.nnum, vt), g.scale, g.background, 200)
    ht1 = orl.ht_one(psf, g.nnum, g.H, g.W)
    v = np.ones((g.nz, g.H, g.W))
    for _ in range(4):
        vn, hv = orl.rl_step(psf, g.nnum, y, v, ht1)
        assert vn.min() >= 0.0
        lhs = float(np.sum(ht1 * vn))
        rhs = float(np.sum(y * hv / (hv + orl.EPS)))
        assert abs(lhs - rhs) <= 1e-12 * rhs
        assert abs(lhs - float(np.sum(y))) <= 1e-6 * float(np.sum(y))
        v = vn


def test_rl_metric_history_config0(orc):
    """Five iterations of the tiny configuration: entropies finite, prediction
    consistent with the history."""
    g = synth.CONFIGS[0]
    psf = synth.make_psf(0)
    y = synth.poisson_data(orc.forward(psf, g.nnum, synth.ground_truth(0)), g.scale, g.background, 200)
    from oracle.metric import predicted_iteration, region_size
    XS, YS = region_size(g.nnum, g.H, g.W)
    res = orl.rl(psf, g.nnum, y, g.iterations, XS, YS)
    assert len(res.entropy) == g.iterations
    assert all(np.isfinite(res.entropy))
    assert res.predicted == predicted_iteration(res.entropy)


@pytest.mark.parametrize("world", [2])
def test_depth_split_reduction(world, orc):
    """Depth-split projection (Section 2.1: depths divided among devices): the
    partial forward projections of disjoint depth ranges sum to the full one, and
    the partial z-maxima combine by max into the full MIP (exact)."""
    N, L, Nz, k = 5, 6, 5, 3
    H = W = N * L
    psf = synth.random_psf(12, N, Nz, k * N).astype(np.float64)
    v = synth.random_volume(13, Nz, H, W).astype(np.float64)
    full = orc.forward(psf, N, v)
    bounds = [Nz * r // world for r in range(world + 1)]
    parts = [orc.forward(psf[a:b], N, v[a:b]) for a, b in zip(bounds, bounds[1:])]
    np.testing.assert_allclose(sum(parts), full, rtol=1e-13)
    mips = [v[a:b].max(axis=0) for a, b in zip(bounds, bounds[1:])]
    assert np.array_equal(np.maximum.reduce(mips), v.max(axis=0))
