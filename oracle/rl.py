"""Richardson-Lucy deconvolution for the light-field model, FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper names RL deconvolution (Sections 1 and 2.1) without writing the
update; it is restated here in the usual multiplicative form:

    v^0     = 1 (every voxel)
    r       = y / (H v^{k-1} + eps)        (0 where the denominator is <= 0)
    v^k     = v^{k-1} * (H^T r) / (H^T 1)  (0 where H^T 1 == 0)
    v^k     = max(0, v^k), NaN -> 0
    E_k     = DCT entropy of max_z v^k     (Section 2.2)
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import backward, forward
from .metric import dct_entropy, mip_z, predicted_iteration

EPS = 1e-6


@dataclass
class RLResult:
    v: np.ndarray                         # final iterate v^n, FP64 [Nz][H][W]
    entropy: list = field(default_factory=list)   # E_1..E_n
    flux: list = field(default_factory=list)      # sum(H^T1 * v^k), k=1..n
    predicted: int = 0                    # predicted iteration n*
    iterates: list = field(default_factory=list)  # v^k, only if kept


def ht_one(psf, nnum: int, H: int, W: int, nthreads=None) -> np.ndarray:
    """H^T 1: the backprojection of an all-ones sensor image."""
    return backward(psf, nnum, np.ones((H, W)), nthreads)


def rl_step(psf, nnum, y, v, ht1, eps=EPS, nthreads=None):
    """One RL iteration; returns (v_new, Hv of the old iterate)."""
    hv = forward(psf, nnum, v, nthreads)
    den = hv + eps
    with np.errstate(divide="ignore", invalid="ignore"):
        r = np.where(den > 0, np.asarray(y, np.float64) / den, 0.0)
    x = backward(psf, nnum, r, nthreads)
    with np.errstate(divide="ignore", invalid="ignore"):
        vn = np.where(ht1 > 0, v * x / ht1, 0.0)
    vn = np.where(np.isnan(vn), 0.0, np.maximum(vn, 0.0))
    return vn, hv


def rl(psf, nnum: int, y, n: int, XS: int, YS: int, eps: float = EPS,
       v0=None, l2_over_region: bool = True, keep_iterates: bool = False,
       nthreads=None) -> RLResult:
    """n RL iterations from v0 (default: ones), with the metric per iteration."""
    y = np.asarray(y, np.float64)
    H, W = y.shape
    Nz = np.asarray(psf).shape[0]
    v = np.ones((Nz, H, W)) if v0 is None else np.array(v0, np.float64)
    ht1 = ht_one(psf, nnum, H, W, nthreads)
    res = RLResult(v=v)
    for _ in range(n):
        v, _ = rl_step(psf, nnum, y, v, ht1, eps, nthreads)
        res.entropy.append(dct_entropy(mip_z(v), XS, YS, l2_over_region))
        res.flux.append(float(np.sum(ht1 * v)))
        if keep_iterates:
            res.iterates.append(v.copy())
    res.v = v
    res.predicted = predicted_iteration(res.entropy)
    return res
