"""Pins for the oracle's light-field projections (forward H, backward H^T).

Each check is independent of the oracle's own C loops: a dense matrix built by
placing single-voxel PSFs with numpy slicing, the textbook 2-D convolution of
scipy (the phase-masked form of Prevedel et al. 2014 that the paper's
deconvolution uses, Section 1), the adjoint identity, delta inputs and
closed-form sums.
"""
import numpy as np
import pytest
from scipy.signal import convolve2d

from paper_2208_11422_gb300 import synth


def dense_matrix(psf, N, H, W):
    """A[(i,j), (z,i',j')] by placing PSF_{phase(i',j'), z} centred on (i',j')."""
    Nz, _, _, P, _ = psf.shape
    c = (P - 1) // 2
    A = np.zeros((H * W, Nz * H * W))
    for z in range(Nz):
        for ip in range(H):
            for jp in range(W):
                img = np.zeros((H + 2 * c, W + 2 * c))
                img[ip:ip + P, jp:jp + P] = psf[z, ip % N, jp % N]
                A[:, (z * H + ip) * W + jp] = img[c:c + H, c:c + W].ravel()
    return A


GEOMS = [  # (Nnum, lenslets y, lenslets x, Nz, PSF lenslets)
    (3, 4, 4, 2, 3),
    (3, 4, 3, 2, 5),   # PSF wider than the sensor, non-square sensor
    (1, 6, 5, 2, 3),   # Nnum = 1: plain convolution per depth
    (5, 2, 3, 1, 1),   # PSF of a single lenslet
]


@pytest.mark.parametrize("geom", GEOMS)
def test_forward_backward_equal_dense_matrix(orc, geom):
    N, Ly, Lx, Nz, k = geom
    H, W, P = Ly * N, Lx * N, k * N
    psf = synth.random_psf(7, N, Nz, P).astype(np.float64)
    A = dense_matrix(psf, N, H, W)
    rng = np.random.default_rng(3)
    v = rng.uniform(0, 1, (Nz, H, W))
    y = rng.uniform(0, 1, (H, W))
    hv = orc.forward(psf, N, v)
    np.testing.assert_allclose(hv.ravel(), A @ v.ravel(), rtol=1e-12, atol=1e-14)
    ht = orc.backward(psf, N, y)
    np.testing.assert_allclose(ht.ravel(), A.T @ y.ravel(), rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("geom", [(3, 5, 4, 2, 3), (5, 6, 6, 3, 3), (5, 15, 15, 5, 5)])
def test_forward_equals_phase_masked_convolution(orc, geom):
    """Hv = sum_z sum_{aa,bb} conv2(v_z masked to phase (aa,bb), K[z,aa,bb], 'same');
    H^T r = sum over phases of mask * conv2(r, flipped K, 'same')."""
    N, Ly, Lx, Nz, k = geom
    H, W, P = Ly * N, Lx * N, k * N
    psf = synth.random_psf(11, N, Nz, P, density=0.7).astype(np.float64)
    rng = np.random.default_rng(5)
    v = rng.uniform(0, 1, (Nz, H, W))
    r = rng.uniform(0, 1, (H, W))
    ref_f = np.zeros((H, W))
    ref_b = np.zeros((Nz, H, W))
    for z in range(Nz):
        for aa in range(N):
            for bb in range(N):
                mask = np.zeros((H, W))
                mask[aa::N, bb::N] = 1.0
                ref_f += convolve2d(v[z] * mask, psf[z, aa, bb], mode="same")
                ref_b[z] += mask * convolve2d(r, psf[z, aa, bb][::-1, ::-1], mode="same")
    np.testing.assert_allclose(orc.forward(psf, N, v), ref_f, rtol=1e-11, atol=1e-13)
    np.testing.assert_allclose(orc.backward(psf, N, r), ref_b, rtol=1e-11, atol=1e-13)


def test_adjoint_identity(orc):
    N, L, Nz, k = 5, 7, 3, 3
    H = W = L * N
    psf = synth.random_psf(1, N, Nz, k * N).astype(np.float64)
    rng = np.random.default_rng(9)
    v = rng.normal(size=(Nz, H, W))
    y = rng.normal(size=(H, W))
    lhs = float(np.sum(orc.forward(psf, N, v) * y))
    rhs = float(np.sum(v * orc.backward(psf, N, y)))
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


@pytest.mark.parametrize("pos", [(0, 0, 0), (1, 7, 3), (2, 14, 14), (1, 0, 9)])
def test_delta_voxel_reproduces_psf_slice(orc, pos):
    N, L, Nz, k = 5, 3, 3, 3
    H = W = L * N
    P = k * N
    c = (P - 1) // 2
    psf = synth.make_psf(synth.Geometry("t", N, L, Nz, k, 1, 0.8, 0.6, 1, 0, 1, 1, 0, 1, 0, 1)).astype(np.float64)
    z, ip, jp = pos
    v = np.zeros((Nz, H, W))
    v[z, ip, jp] = 1.0
    img = np.zeros((H + 2 * c, W + 2 * c))
    img[ip:ip + P, jp:jp + P] = psf[z, ip % N, jp % N]
    expect = img[c:c + H, c:c + W]
    assert np.array_equal(orc.forward(psf, N, v), expect)


def test_delta_psf_closed_forms(orc):
    """A centred delta PSF makes Hv = sum_z v_z and H^T r = r in every depth."""
    N, L, Nz, k = 3, 4, 4, 3
    H = W = L * N
    P = k * N
    c = (P - 1) // 2
    psf = np.zeros((Nz, N, N, P, P))
    psf[:, :, :, c, c] = 1.0
    rng = np.random.default_rng(2)
    v = rng.uniform(size=(Nz, H, W))
    r = rng.uniform(size=(H, W))
    assert np.allclose(orc.forward(psf, N, v), v.sum(axis=0), rtol=1e-15, atol=0)
    assert np.array_equal(orc.backward(psf, N, r), np.broadcast_to(r, (Nz, H, W)))


def test_sampled_outputs_match_full(orc):
    N, L, Nz, k = 5, 6, 3, 3
    H = W = L * N
    psf = synth.random_psf(4, N, Nz, k * N).astype(np.float64)
    rng = np.random.default_rng(8)
    v = rng.uniform(size=(Nz, H, W))
    r = rng.uniform(size=(H, W))
    full_f = orc.forward(psf, N, v)
    full_b = orc.backward(psf, N, r)
    pix = synth.sample_indices(1, 50, (H, W))
    vox = synth.sample_indices(2, 50, (Nz, H, W))
    np.testing.assert_allclose(orc.forward_at(psf, N, v, pix), full_f[pix[:, 0], pix[:, 1]], rtol=1e-13)
    np.testing.assert_allclose(orc.backward_at(psf, N, r, vox),
                               full_b[vox[:, 0], vox[:, 1], vox[:, 2]], rtol=1e-13)


def test_thread_count_does_not_change_result(orc):
    N, L, Nz, k = 5, 5, 2, 3
    H = W = L * N
    psf = synth.random_psf(6, N, Nz, k * N).astype(np.float64)
    v = synth.random_volume(3, Nz, H, W).astype(np.float64)
    a = orc.forward(psf, N, v, nthreads=1)
    b = orc.forward(psf, N, v, nthreads=7)
    assert np.array_equal(a, b)


def test_mac_count(orc):
    """Interior count is H*W*Nz*P^2 when the PSF never leaves the sensor... and
    the exact clipped count matches a brute-force tally."""
    P, Nz, H, W = 9, 2, 12, 7
    c = (P - 1) // 2
    brute = 0
    for i in range(H):
        for j in range(W):
            for mi in range(P):
                for mj in range(P):
                    if 0 <= i + mi - c < H and 0 <= j + mj - c < W:
                        brute += 1
    assert orc.macs_per_projection(P, Nz, H, W) == Nz * brute


# crops (i0, i1, j0, j1) of a 60 x 75 px sensor: interior, at the borders,
# origins not on the lenslet grid, a single pixel, the whole sensor
CROPS = [(20, 41, 31, 52), (0, 13, 0, 9), (47, 60, 61, 75), (7, 8, 44, 45), (0, 60, 0, 75)]


@pytest.mark.parametrize("crop", CROPS)
def test_forward_crop_equals_full_forward(orc, crop):
    """forward_crop runs the forward model over a window of the volume; inside
    the crop it adds the same terms in the same order as the full frame."""
    N, Nz, P = 3, 3, 15
    H, W = 60, 75
    psf = synth.random_psf(31, N, Nz, P).astype(np.float64)
    v = synth.random_volume(32, Nz, H, W).astype(np.float64)
    v[v < 0.6] = 0.0                 # sparse, like the bead volumes
    i0, i1, j0, j1 = crop
    full = orc.forward(psf, N, v)
    assert np.array_equal(orc.forward_crop(psf, N, v, i0, i1, j0, j1), full[i0:i1, j0:j1])


@pytest.mark.parametrize("crop", CROPS)
def test_backward_block_equals_full_backward(orc, crop):
    """backward_block gives every voxel of the block the sum backward_at forms;
    the block's rows mix voxels whose windows are cut by the sensor and voxels
    computed eight side by side."""
    N, Nz, P = 3, 3, 15
    H, W = 60, 75
    psf = synth.random_psf(33, N, Nz, P).astype(np.float64)
    r = synth.random_image(34, H, W, 0.1, 2.0).astype(np.float64)
    i0, i1, j0, j1 = crop
    full = orc.backward(psf, N, r)
    blk = orc.backward_block(psf, N, r, 1, Nz, i0, i1, j0, j1)
    assert np.array_equal(blk, full[1:, i0:i1, j0:j1])
    zz, ii, jj = np.meshgrid(np.arange(1, Nz), np.arange(i0, i1), np.arange(j0, j1), indexing="ij")
    vox = np.stack([zz.ravel(), ii.ravel(), jj.ravel()], 1)
    assert np.array_equal(orc.backward_at(psf, N, r, vox), blk.ravel())
