"""Seeded synthetic inputs for light-field deconvolution: PSFs, volumes, data.

This module holds input generation only. It contains none of the projection,
Richardson-Lucy or metric arithmetic, imports nothing from the CUDA binding or
from the oracle, and is the one module both the tests' oracle side and the GPU
side read their inputs from.

The paper's own data (Prevedel et al. 2014 C. elegans, beads, MCF10A cells;
Sections 1 and 3.2) are not available; these generators stand in for them with
the shapes of the paper's setting: Nnum = 5..15 virtual pixels per lenslet,
tens of depths, PSFs several lenslets wide, sparse bright objects on a dark
background, Poisson photon noise plus a constant background.

PSF (per depth z and lenslet phase (aa, bb), window P = k*Nnum, centre c):
    spots on the lenslet-centre grid c + Nnum*(m, n) with m^2 + n^2 <= R(z)^2,
    each moved by ((aa - a_c), (bb - a_c)) * (z - z_c) / 2 pixels
    (a_c = (Nnum-1)/2), amplitude exp(-(m^2 + n^2)/4), a Gaussian of width
    sigma(z) sampled at integer pixel centres, truncated to the window, then
    each (z, aa, bb) slice normalised to unit sum in FP64 and stored as FP32.
    The PSF is deterministic (no random draws).
Beads:      sum of A exp(-|p - c|^2 / (2 r^2)), truncated at |p - c| <= 4 r,
            centres uniform over the volume, A uniform.
Filaments:  random walks of unit steps, direction d <- normalise(d + 0.3 N(0,I)),
            reflected at the walls; value max over centreline points of
            A exp(-dist^2 / (2 * 1.5^2)) truncated at 4 * 1.5.
Data:       y = float32(Poisson(scale * expected) + background).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Geometry:
    name: str
    nnum: int          # virtual pixels per lenslet (odd)
    lenslets: int      # lenslets per side (square sensor)
    nz: int            # depths
    psf_lenslets: int  # PSF window width in lenslets (odd)
    z_c: int           # depth of the focal plane in the PSF generator
    sigma0: float      # sigma(z) = sigma0 + sigma1 * |z - z_c|
    sigma1: float
    radius_div: int    # R(z) = ceil(|z - z_c| / radius_div) lenslets
    beads: int
    bead_radius: float
    amp_lo: float
    filaments: int
    scale: float       # photons per unit of expected signal
    background: float
    iterations: int

    @property
    def H(self) -> int:
        return self.lenslets * self.nnum

    @property
    def W(self) -> int:
        return self.lenslets * self.nnum

    @property
    def P(self) -> int:
        return self.psf_lenslets * self.nnum


CONFIGS = {
    # tiny: Nnum 5, 75x75 px, 5 depths, PSF 25 px
    0: Geometry("lf_tiny_75px_5z_psf25", 5, 15, 5, 5, 2, 0.8, 0.6, 1,
                8, 1.5, 0.5, 0, 200.0, 2.0, 5),
    # mid size: Nnum 15, 615x615 px, 31 depths, PSF 165 px
    1: Geometry("lf_mid_615px_31z_psf165", 15, 41, 31, 11, 15, 1.0, 0.4, 3,
                300, 2.0, 0.3, 0, 500.0, 5.0, 10),
    # large frame: Nnum 15, 2025x2025 px, 51 depths, PSF 345 px
    2: Geometry("lf_large_2025px_51z_psf345", 15, 135, 51, 23, 25, 1.0, 0.4, 3,
                5000, 2.0, 0.3, 200, 1000.0, 10.0, 30),
}


def psf_gaussian_spots(nnum: int, nz: int, psf_lenslets: int, z_c: int,
                       sigma0: float, sigma1: float, radius_div: int,
                       z_range=None) -> np.ndarray:
    """PSF array [Nz][Nnum][Nnum][P][P] float32 (see module docstring).

    ``radius_div`` = 1 gives R(z) = |z - z_c|; otherwise ceil(|z-z_c|/div).
    ``z_range`` restricts generation to a slice of depths (same values)."""
    N = nnum
    P = psf_lenslets * N
    c = (P - 1) // 2
    a_c = (N - 1) / 2.0
    zs = range(nz) if z_range is None else z_range
    out = np.zeros((len(zs), N, N, P, P), np.float32)
    pix = np.arange(P, dtype=np.float64)
    for zi, z in enumerate(zs):
        sigma = sigma0 + sigma1 * abs(z - z_c)
        R = abs(z - z_c) if radius_div == 1 else int(math.ceil(abs(z - z_c) / radius_div))
        ms = np.arange(-R, R + 1)
        nmax = np.array([math.isqrt(R * R - int(m) * int(m)) for m in ms])
        sz = (z - z_c) / 2.0
        shifts = (np.arange(N) - a_c) * sz                  # per phase
        # Gy[a, m, i] = exp(-m^2/4) g(i - c - N m - dy_a)
        dy = pix[None, None, :] - c - N * ms[None, :, None] - shifts[:, None, None]
        Gy = np.exp(-(ms[None, :, None] ** 2) / 4.0) * np.exp(-dy * dy / (2 * sigma * sigma))
        # Gx[b, m, j] = sum_{|n| <= nmax(m)} exp(-n^2/4) g(j - c - N n - dx_b)
        ns = ms
        dx = pix[None, None, :] - c - N * ns[None, :, None] - shifts[:, None, None]
        gx_n = np.exp(-(ns[None, :, None] ** 2) / 4.0) * np.exp(-dx * dx / (2 * sigma * sigma))
        inside = (np.abs(ns)[None, :] <= nmax[:, None]).astype(np.float64)  # [m, n]
        Gx = np.einsum("mn,bnj->bmj", inside, gx_n)
        A = Gy.transpose(0, 2, 1).reshape(N * P, len(ms))   # (a,i) x m
        B = Gx.transpose(1, 0, 2).reshape(len(ms), N * P)   # m x (b,j)
        sl = (A @ B).reshape(N, P, N, P).transpose(0, 2, 1, 3)
        sums = sl.sum(axis=(2, 3), keepdims=True)
        out[zi] = (sl / sums).astype(np.float32)
    return out


def make_psf(cfg: int | Geometry) -> np.ndarray:
    g = CONFIGS[cfg] if isinstance(cfg, int) else cfg
    return psf_gaussian_spots(g.nnum, g.nz, g.psf_lenslets, g.z_c, g.sigma0,
                              g.sigma1, g.radius_div)


def _gauss_blob(v: np.ndarray, cz, cy, cx, amp, r, combine="add"):
    """Add (or max) amp*exp(-d^2/(2r^2)) within d <= 4r of (cz, cy, cx)."""
    Nz, H, W = v.shape
    rad = 4.0 * r
    z0, z1 = max(0, int(math.floor(cz - rad))), min(Nz, int(math.ceil(cz + rad)) + 1)
    y0, y1 = max(0, int(math.floor(cy - rad))), min(H, int(math.ceil(cy + rad)) + 1)
    x0, x1 = max(0, int(math.floor(cx - rad))), min(W, int(math.ceil(cx + rad)) + 1)
    if z0 >= z1 or y0 >= y1 or x0 >= x1:
        return
    zz = np.arange(z0, z1)[:, None, None] - cz
    yy = np.arange(y0, y1)[None, :, None] - cy
    xx = np.arange(x0, x1)[None, None, :] - cx
    d2 = zz * zz + yy * yy + xx * xx
    blob = np.where(d2 <= rad * rad, amp * np.exp(-d2 / (2.0 * r * r)), 0.0)
    sub = v[z0:z1, y0:y1, x0:x1]
    if combine == "add":
        sub += blob
    else:
        np.maximum(sub, blob, out=sub)


def beads(seed: int, nz: int, H: int, W: int, count: int, radius: float,
          amp_lo: float, amp_hi: float = 1.0) -> np.ndarray:
    """Bead volume [Nz][H][W] float64; draws x, y, z centres then amplitudes."""
    rng = np.random.default_rng(seed)
    cx = rng.uniform(0, W, count)
    cy = rng.uniform(0, H, count)
    cz = rng.uniform(0, nz, count)
    amp = rng.uniform(amp_lo, amp_hi, count)
    v = np.zeros((nz, H, W), np.float64)
    for q in range(count):
        _gauss_blob(v, cz[q], cy[q], cx[q], amp[q], radius)
    return v


def beads_device(seed: int, nz: int, H: int, W: int, count: int, radius: float,
                 amp_lo: float, amp_hi: float = 1.0, device="cuda", out=None):
    """The volume of ``beads`` built on a torch device (float32): the same seeded
    draws, each bead splatted over the grid points within 4r of its centre.
    Equal to ``beads`` up to float rounding; for timing inputs that must be
    made quickly (serving pools). out: a zeroed [Nz][H][W] tensor to fill."""
    import torch
    rng = np.random.default_rng(seed)
    cx = rng.uniform(0, W, count)
    cy = rng.uniform(0, H, count)
    cz = rng.uniform(0, nz, count)
    amp = rng.uniform(amp_lo, amp_hi, count)
    v = torch.zeros((nz, H, W), dtype=torch.float32, device=device) if out is None else out
    rad = 4.0 * radius
    k = int(math.ceil(rad)) + 1
    off = torch.arange(-k, k + 1, device=device, dtype=torch.float64)
    c = torch.tensor(np.stack([cz, cy, cx], 1), device=device, dtype=torch.float64)   # [n, 3]
    a = torch.tensor(amp, device=device, dtype=torch.float64)
    base = torch.floor(c)                                                             # [n, 3]
    for chunk in range(0, count, 512):
        cc, bb, aa = c[chunk:chunk + 512], base[chunk:chunk + 512], a[chunk:chunk + 512]
        pz = bb[:, 0, None] + off[None, :]          # [m, 2k+1] candidate grid coordinates
        py = bb[:, 1, None] + off[None, :]
        px = bb[:, 2, None] + off[None, :]
        dz = pz - cc[:, 0, None]
        dy = py - cc[:, 1, None]
        dx = px - cc[:, 2, None]
        d2 = dz[:, :, None, None] ** 2 + dy[:, None, :, None] ** 2 + dx[:, None, None, :] ** 2
        val = aa[:, None, None, None] * torch.exp(-d2 / (2.0 * radius * radius))
        ok = (d2 <= rad * rad) & (pz >= 0)[:, :, None, None] & (pz < nz)[:, :, None, None] \
            & (py >= 0)[:, None, :, None] & (py < H)[:, None, :, None] \
            & (px >= 0)[:, None, None, :] & (px < W)[:, None, None, :]
        zi = pz[:, :, None, None].expand_as(d2)[ok].long()
        yi = py[:, None, :, None].expand_as(d2)[ok].long()
        xi = px[:, None, None, :].expand_as(d2)[ok].long()
        v.index_put_((zi, yi, xi), val[ok].to(torch.float32), accumulate=True)
    return v


def filaments(seed: int, nz: int, H: int, W: int, count: int, radius: float = 1.5,
              amp_lo: float = 0.3, amp_hi: float = 1.0) -> np.ndarray:
    """Tubular random-walk filaments [Nz][H][W] float64 (max-combined)."""
    rng = np.random.default_rng(seed)
    dims = np.array([nz, H, W], np.float64)
    v = np.zeros((nz, H, W), np.float64)
    for _ in range(count):
        p = rng.uniform(0, 1, 3) * dims
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        steps = int(rng.integers(50, 301))
        amp = rng.uniform(amp_lo, amp_hi)
        for _s in range(steps):
            _gauss_blob(v, p[0], p[1], p[2], amp, radius, combine="max")
            d = d + 0.3 * rng.normal(size=3)
            d /= np.linalg.norm(d)
            p = p + d
            for a in range(3):
                if p[a] < 0:
                    p[a] = -p[a]
                    d[a] = -d[a]
                elif p[a] > dims[a] - 1:
                    p[a] = 2 * (dims[a] - 1) - p[a]
                    d[a] = -d[a]
    return v


def ground_truth(cfg: int | Geometry, seed: int | None = None) -> np.ndarray:
    """Ground-truth volume [Nz][H][W] float64 for a configuration."""
    g = CONFIGS[cfg] if isinstance(cfg, int) else cfg
    idx = cfg if isinstance(cfg, int) else 0
    s = 100 + idx if seed is None else seed
    v = beads(s, g.nz, g.H, g.W, g.beads, g.bead_radius, g.amp_lo)
    if g.filaments:
        v = v + filaments(s + 1000, g.nz, g.H, g.W, g.filaments)
    return v


def timelapse_beads(cfg: int | Geometry, frames: int, seed: int, step_sigma: float = 0.5,
                    seed_offset: int = 0):
    """Bead volumes of a time-lapse: frame 0 has the configuration's beads, and
    every later frame moves each bead centre by an N(0, step_sigma^2) step per
    axis (cumulative). Returns a list of float64 volumes [Nz][H][W]."""
    g = CONFIGS[cfg] if isinstance(cfg, int) else cfg
    rng = np.random.default_rng(seed)
    cx = rng.uniform(0, g.W, g.beads)
    cy = rng.uniform(0, g.H, g.beads)
    cz = rng.uniform(0, g.nz, g.beads)
    amp = rng.uniform(g.amp_lo, 1.0, g.beads)
    vols = []
    for _f in range(frames):
        v = np.zeros((g.nz, g.H, g.W), np.float64)
        for q in range(g.beads):
            _gauss_blob(v, cz[q], cy[q], cx[q], amp[q], g.bead_radius)
        vols.append(v)
        cx = cx + rng.normal(0, step_sigma, g.beads)
        cy = cy + rng.normal(0, step_sigma, g.beads)
        cz = cz + rng.normal(0, step_sigma, g.beads)
    return vols


def timelapse_scales(frames: int, seed: int, lo: float = 100.0, hi: float = 2000.0) -> np.ndarray:
    """Photon scale of every frame, uniform in [lo, hi]."""
    return np.random.default_rng(seed).uniform(lo, hi, frames)


def poisson_data(expected, scale: float, background: float, seed: int) -> np.ndarray:
    """y = float32(Poisson(scale * expected) + background)."""
    rng = np.random.default_rng(seed)
    lam = np.maximum(np.asarray(expected, np.float64), 0.0) * scale
    return (rng.poisson(lam).astype(np.float64) + background).astype(np.float32)


def random_volume(seed: int, nz: int, H: int, W: int, lo: float = 0.0,
                  hi: float = 1.0) -> np.ndarray:
    """Dense uniform random volume [Nz][H][W] float32 (parity inputs)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, (nz, H, W)).astype(np.float32)


def random_image(seed: int, H: int, W: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, (H, W)).astype(np.float32)


def random_psf(seed: int, nnum: int, nz: int, P: int, density: float = 1.0) -> np.ndarray:
    """Random non-negative PSF [Nz][Nnum][Nnum][P][P] float32 (parity inputs);
    ``density`` < 1 zeroes a random share of taps."""
    rng = np.random.default_rng(seed)
    k = rng.uniform(0.0, 1.0, (nz, nnum, nnum, P, P))
    if density < 1.0:
        k *= rng.uniform(0, 1, k.shape) < density
    k /= np.maximum(k.sum(axis=(3, 4), keepdims=True), 1e-300)
    return k.astype(np.float32)


def sample_indices(seed: int, count: int, dims) -> np.ndarray:
    """count random index tuples within dims (int32 [count][len(dims)])."""
    rng = np.random.default_rng(seed)
    return np.stack([rng.integers(0, d, count) for d in dims], axis=1).astype(np.int32)


# ----------------------------------------------------------------- serving --
SERVE_NNUM = (11, 13, 15)
SERVE_NZ = (21, 31, 41, 51)
SERVE_PSF_LENSLETS = 11
SERVE_LENSLETS = (33, 121)     # lenslet grid per axis, uniform integers


def serve_psf_set(j: int):
    """PSF set j (1..4) of the serving workload: (Nnum, Nz) drawn with
    default_rng(j), a PSF window 11 lenslets wide with the mid-size workload's
    sigma(z) = 1 + 0.4 |z - z_c|, R(z) = ceil(|z - z_c| / 3), z_c = Nz // 2.
    Returns (nnum, nz, P, psf)."""
    rng = np.random.default_rng(j)
    nnum = int(rng.choice(SERVE_NNUM))
    nz = int(rng.choice(SERVE_NZ))
    psf = psf_gaussian_spots(nnum, nz, SERVE_PSF_LENSLETS, nz // 2, 1.0, 0.4, 3)
    return nnum, nz, SERVE_PSF_LENSLETS * nnum, psf


@dataclass(frozen=True)
class ServeRequest:
    index: int
    arrival_s: float   # Poisson arrivals
    set_id: int        # 1..4
    ly: int            # lenslet grid
    lx: int
    beads: int         # 50..5000
    scale: float       # photons per unit signal, log-uniform [100, 5000]
    seed: int


def serve_requests(n: int, seed: int, rate_hz: float = 20.0, sets: int = 4):
    """n requests of the serving workload: exponential inter-arrival times of
    mean 1 / rate_hz, a PSF set uniform in 1..sets, lenslet grid uniform in
    33..121 per axis, 50..5000 beads, photon scale log-uniform over [100, 5000]."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, n))
    set_id = rng.integers(1, sets + 1, n)
    ly = rng.integers(SERVE_LENSLETS[0], SERVE_LENSLETS[1] + 1, n)
    lx = rng.integers(SERVE_LENSLETS[0], SERVE_LENSLETS[1] + 1, n)
    nb = rng.integers(50, 5001, n)
    scale = np.exp(rng.uniform(math.log(100.0), math.log(5000.0), n))
    return [ServeRequest(i, float(t[i]), int(set_id[i]), int(ly[i]), int(lx[i]), int(nb[i]),
                         float(scale[i]), seed * 100003 + i) for i in range(n)]


def serve_volume(req: ServeRequest, nnum: int, nz: int) -> np.ndarray:
    """Bead volume [Nz][ly*Nnum][lx*Nnum] of a serving request (radius 2,
    amplitudes U[0.3, 1]), float32."""
    return beads(req.seed, nz, req.ly * nnum, req.lx * nnum, req.beads, 2.0, 0.3).astype(np.float32)
