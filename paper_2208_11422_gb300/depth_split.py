"""Depth-split Richardson-Lucy: the depth layers of the volume, and the PSF
slices that belong to them, are divided among workers (Section 2.1 and Fig. 1:
depth layers and PSF slices divided among GPUs).

Each worker owns a context over its depth range [z0, z1) (the PSF slice
psf[z0:z1]) and the matching part of the volume. One RL iteration then needs
two exchanges:

  1. the forward projection is the sum of the parts' partial projections
     (all-reduce, sum, of an [H][W] image);
  2. after each part's backprojection and update (per depth, no exchange),
     the z-maximum projection is the maximum of the parts' (all-reduce, max,
     of an [H][W] image) and the flux the sum of theirs (all-reduce, sum, of
     one double).

The entropy of the reduced projection image and the stopping rule are those
of ``lfd_rl_iterate``. The arithmetic runs in the library (``lfd_split_*``
and ``lfd_quality_mip``); this module only orders the calls and the
reductions. Parts owned by this process are combined in list order, then
across processes through ``torch.distributed`` (NCCL for CUDA tensors, or
gloo, staged through host memory).
"""
from __future__ import annotations

from dataclasses import dataclass, field

from . import lfd


def depth_ranges(nz: int, parts: int) -> list[tuple[int, int]]:
    """Split depths 0..nz-1 into `parts` contiguous ranges of near-equal size."""
    if parts < 1 or parts > nz:
        raise ValueError("need 1 <= parts <= nz")
    return [(nz * p // parts, nz * (p + 1) // parts) for p in range(parts)]


class Reducer:
    """Sum / max of a tensor over the processes of a torch.distributed group
    (identity when there is no group or only one process)."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.active = dist.is_available() and dist.is_initialized() and \
            dist.get_world_size(group) > 1
        self.stage = self.active and dist.get_backend(group) == "gloo"

    def _all_reduce(self, t, op):
        if not self.active:
            return t
        if self.stage and t.is_cuda:
            h = t.cpu()
            self.dist.all_reduce(h, op=op, group=self.group)
            t.copy_(h)
        else:
            self.dist.all_reduce(t, op=op, group=self.group)
        return t

    def sum_(self, t):
        return self._all_reduce(t, self.dist.ReduceOp.SUM)

    def max_(self, t):
        return self._all_reduce(t, self.dist.ReduceOp.MAX)


class LibraryShard:
    """A context over the depths [z0, z1) of a PSF held on the device."""

    def __init__(self, psf_dev, P: int, nnum: int, z0: int, z1: int, H: int, W: int,
                 opt: lfd.lfd_options | None = None, stream=None):
        part = psf_dev[z0:z1]
        if not part.is_contiguous():
            raise ValueError("the PSF must be contiguous [Nz][Nnum][Nnum][P][P]")
        self.z0, self.z1, self.H, self.W = z0, z1, H, W
        self.stream = stream
        self.ctx = lfd.lfd_create(part, P, nnum, z1 - z0, H, W, opt, stream)

    def load(self, v_part):
        lfd.lfd_split_load(self.ctx, v_part, self.stream)

    def forward(self, hv_part):
        lfd.lfd_split_forward(self.ctx, hv_part, self.stream)

    def update(self, y, hv, mip_part, flux_part):
        lfd.lfd_split_update(self.ctx, y, hv, mip_part, flux_part, self.stream)

    def quality(self, mip) -> float:
        return lfd.lfd_quality_mip(self.ctx, mip, self.stream)

    def store(self, v_part, previous: bool = False):
        lfd.lfd_split_store(self.ctx, v_part, previous, self.stream)

    def close(self):
        if self.ctx is not None:
            lfd.lfd_destroy(self.ctx)
            self.ctx = None


@dataclass
class SplitResult:
    iters_done: int = 0          # iterations whose result the parts hold (see previous)
    predicted: int = 0           # first k with E_{k+1} < E_k, else the first argmax
    previous: bool = False       # the result is each part's previous iterate
    entropy: list = field(default_factory=list)   # E_1 .. E_ran
    flux: list = field(default_factory=list)      # sum(H^T 1 v^k) over all depths


def predict_stop(E) -> int:
    """The library's stopping rule (lfd_predict_stop) on an entropy history."""
    import ctypes
    arr = (ctypes.c_double * len(E))(*E)
    return int(lfd.load().lfd_predict_stop(arr, len(E)))


def split_rl(shards, y, n: int, stop_at_predicted: bool = False, reducer: Reducer | None = None,
             predict=None) -> SplitResult:
    """Up to n RL iterations over the depth parts `shards` (this process's,
    each already loaded with its part of v^0) and those of the other processes
    of `reducer`. y is the [H][W] image (on the parts' device). With
    stop_at_predicted the iterations stop once the entropy falls
    (E_{k+1} < E_k) and the result is v^k, each part's previous iterate
    (SplitResult.previous); fetch the parts with shard.store(v, previous)."""
    import torch
    if n < 1 or not shards:
        raise ValueError("need n >= 1 and at least one part")
    reducer = reducer or Reducer()
    predict = predict or predict_stop
    hv = torch.zeros_like(y)
    part = torch.zeros_like(y)
    mip = torch.zeros_like(y)
    mpart = torch.zeros_like(y)
    flux = torch.zeros(1, dtype=torch.float64, device=y.device)
    fpart = torch.zeros(1, dtype=torch.float64, device=y.device)
    res = SplitResult()
    for k in range(n):
        hv.zero_()
        for s in shards:                       # partial forward projections
            s.forward(part)
            hv.add_(part)
        reducer.sum_(hv)
        mip.zero_()                            # iterates are >= 0
        flux.zero_()
        for s in shards:                       # ratio, backprojection, update per part
            s.update(y, hv, mpart, fpart)
            torch.maximum(mip, mpart, out=mip)
            flux.add_(fpart)
        reducer.max_(mip)
        reducer.sum_(flux)
        res.entropy.append(float(shards[0].quality(mip)))
        res.flux.append(float(flux.item()))
        res.iters_done = k + 1
        if stop_at_predicted and k >= 1 and res.entropy[k] < res.entropy[k - 1]:
            res.iters_done = k
            res.previous = True
            break
    res.predicted = predict(res.entropy)
    return res
