"""Helpers shared by the GPU parity tests (test side only)."""
from __future__ import annotations

import numpy as np


def rel_l2(got, ref) -> float:
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    den = np.linalg.norm(ref)
    return float(np.linalg.norm(got - ref) / (den if den > 0 else 1.0))


def lib():
    from paper_2208_11422_gb300 import build, lfd
    build.build()
    return lfd


class Ctx:
    """Context manager around lfd_create / lfd_destroy with torch device buffers."""

    def __init__(self, psf, nnum, H, W, precision="fp32", **opt):
        self.ctx = None
        import torch
        from paper_2208_11422_gb300 import lfd
        self.lfd = lfd
        self.torch = torch
        self.dev = torch.device("cuda:0")
        psf = np.ascontiguousarray(psf, np.float32)
        self.Nz, _, _, self.P, _ = psf.shape
        self.nnum, self.H, self.W = nnum, H, W
        self.psf_dev = torch.from_numpy(psf).to(self.dev)
        self.ctx = lfd.lfd_create(self.psf_dev, self.P, nnum, self.Nz, H, W,
                                  lfd.lfd_default_options(precision=precision, **opt))

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.lfd.lfd_destroy(self.ctx)
        self.ctx = None

    def forward(self, v):
        t = self.torch
        vd = t.from_numpy(np.ascontiguousarray(v, np.float32)).to(self.dev)
        y = t.empty((self.H, self.W), device=self.dev)
        self.lfd.lfd_forward(self.ctx, vd, y)
        t.cuda.synchronize()
        return y.cpu().numpy()

    def backward(self, r):
        t = self.torch
        rd = t.from_numpy(np.ascontiguousarray(r, np.float32)).to(self.dev)
        v = t.empty((self.Nz, self.H, self.W), device=self.dev)
        self.lfd.lfd_backward(self.ctx, rd, v)
        t.cuda.synchronize()
        return v.cpu().numpy()

    def rl(self, y, n, v0=None, stop=False):
        t = self.torch
        yd = t.from_numpy(np.ascontiguousarray(y, np.float32)).to(self.dev)
        if v0 is None:
            v = t.ones((self.Nz, self.H, self.W), device=self.dev)
        else:
            v = t.from_numpy(np.ascontiguousarray(v0, np.float32)).to(self.dev)
        done, pred, ent, flux = self.lfd.lfd_rl_iterate(self.ctx, yd, v, n, stop)
        t.cuda.synchronize()
        return v.cpu().numpy(), done, pred, ent, flux
