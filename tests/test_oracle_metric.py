"""Pins for the oracle's DCT-entropy metric and stopping rule (Section 2.2)."""
import math

import numpy as np
import pytest
import scipy.fft

from oracle import metric


@pytest.mark.parametrize("shape", [(1, 1), (7, 11), (16, 16), (5, 3)])
def test_dct_matches_direct_sum_and_scipy(shape):
    rng = np.random.default_rng(0)
    f = rng.normal(size=shape)
    F = metric.dct2(f)
    np.testing.assert_allclose(F, scipy.fft.dctn(f, type=2, norm="ortho"), rtol=1e-12, atol=1e-12)
    # direct double sum of Eqs. 1-4 on one coefficient per axis pair
    H, W = shape

    def c(k, Z):
        return math.sqrt(1.0 / Z) if k == 0 else math.sqrt(2.0 / Z)

    for (v, u) in [(0, 0), (H - 1, W - 1), (H // 2, W // 3)]:
        s = 0.0
        for y in range(H):
            for x in range(W):
                s += (f[y, x] * c(u, W) * math.cos((2 * x + 1) * math.pi * u / (2 * W))
                      * c(v, H) * math.cos((2 * y + 1) * math.pi * v / (2 * H)))
        assert abs(F[v, u] - s) < 1e-12


def test_parseval_and_constant_image():
    rng = np.random.default_rng(1)
    f = rng.uniform(size=(12, 9))
    F = metric.dct2(f)
    assert abs(np.sum(F * F) - np.sum(f * f)) < 1e-12 * np.sum(f * f)
    const = np.full((10, 14), 3.5)
    Fc = metric.dct2(const)
    assert abs(Fc[0, 0] - 3.5 * math.sqrt(140)) < 1e-12
    Fc[0, 0] = 0
    assert np.max(np.abs(Fc)) < 1e-12
    assert abs(metric.dct_entropy(const, 4, 4)) < 1e-12


def basis_image(H, W, v, u):
    return np.outer(metric.dct_basis(H)[v], metric.dct_basis(W)[u])


def test_entropy_single_coefficient_is_zero():
    f = 2.0 * basis_image(20, 24, 1, 2)
    assert abs(metric.dct_entropy(f, 6, 5)) < 1e-12


@pytest.mark.parametrize("n", [2, 3, 5])
def test_entropy_equal_magnitudes(n):
    """n coefficients of equal magnitude in S: p = 1/sqrt(n) each, so
    E = -(1/G_S) * n * (1/sqrt n) * log2(1/sqrt n) = sqrt(n) log2(n) / (2 G_S)."""
    H, W, XS, YS = 30, 26, 8, 6
    inside = [(0, 0), (1, 0), (0, 1), (2, 3), (1, 4)]
    mask = metric.region_mask(XS, YS)
    f = np.zeros((H, W))
    for q, (v, u) in enumerate(inside[:n]):
        assert mask[v, u]
        f += (-1.0) ** q * 0.7 * basis_image(H, W, v, u)
    G = XS * YS / 2.0
    expect = math.sqrt(n) * math.log2(n) / 2.0 / G
    assert abs(metric.dct_entropy(f, XS, YS) - expect) < 1e-12


def test_entropy_norm_domain():
    """With l2 over the whole DCT, energy outside S lowers every |p|."""
    H, W, XS, YS = 16, 16, 4, 4
    f = basis_image(H, W, 0, 0) + basis_image(H, W, 0, 1) + math.sqrt(2) * basis_image(H, W, 10, 10)
    G = XS * YS / 2.0
    # in S: two coefficients of 1; norm over S = sqrt 2, over all = 2
    e_region = metric.dct_entropy(f, XS, YS, l2_over_region=True)
    e_all = metric.dct_entropy(f, XS, YS, l2_over_region=False)
    assert abs(e_region - (-2 * (1 / math.sqrt(2)) * math.log2(1 / math.sqrt(2)) / G)) < 1e-12
    assert abs(e_all - (-2 * 0.5 * math.log2(0.5) / G)) < 1e-12


def test_region_mask_is_the_triangle():
    for n in range(1, 9):
        assert metric.region_mask(n, n).sum() == n * (n + 1) // 2
    m = metric.region_mask(6, 3)  # u*3 + v*6 < 18
    expect = [[1, 1, 1, 1, 1, 1], [1, 1, 1, 1, 0, 0], [1, 1, 0, 0, 0, 0]]
    assert m.astype(int).tolist() == expect


def test_region_size_from_optics():
    """X_S = P_u * W / d_psf with P_u = d_ML/(Q Nnum) and d_psf = 1.22 lambda Nnum / NA
    (Eqs. 7, 9, 11). With d_ML = 150 um, Q = 40, NA = 0.95, lambda = 0.525 um:
      Nnum 5,  W 75:   150*0.95*75   / (1.22*0.525*40*25)  = 10687.5 / 640.5  = 16.69 -> 16
      Nnum 15, W 615:  150*0.95*615  / (1.22*0.525*40*225) = 87637.5 / 5764.5 = 15.20 -> 15
      Nnum 15, W 2025: 150*0.95*2025 / (1.22*0.525*40*225) = 288562.5/ 5764.5 = 50.06 -> 50
    """
    assert metric.region_size(5, 75, 75) == (16, 16)
    assert metric.region_size(15, 615, 615) == (15, 15)
    assert metric.region_size(15, 2025, 2025) == (50, 50)
    assert metric.region_size(15, 615, 2025) == (50, 15)
    assert metric.region_size(15, 15, 15) == (2, 2)   # clamped below
    assert metric.region_size(1, 3, 1, dML_um=1e4) == (1, 3)  # clamped to the size


@pytest.mark.parametrize("E,expect", [
    ([1.0, 2.0, 3.0, 2.5, 4.0], 3),
    ([5.0, 4.0], 1),
    ([1.0, 1.0, 0.5], 2),          # a tie is not a decrease
    ([1.0, 2.0, 3.0], 3),          # never decreases: argmax
    ([2.0, 2.0, 2.0], 1),          # argmax, first of equals
    ([0.7], 1),
])
def test_predicted_iteration(E, expect):
    assert metric.predicted_iteration(E) == expect


def test_mip():
    v = np.zeros((3, 2, 2))
    v[0, 0, 0] = 1
    v[2, 0, 0] = 5
    v[1, 1, 1] = 2
    assert metric.mip_z(v).tolist() == [[5, 0], [0, 2]]
