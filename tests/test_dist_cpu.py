"""Multi-process paths on CPU with the gloo backend (world size 2).

* bench.py's rank logic: the slowest rank's time sets the job time and the
  throughput counts every rank's units (independent replicas, weak scaling).
* the depth split of Section 2.1 (depth ranges divided among devices): each
  rank projects its own depth range with the oracle, one all-reduce(sum) gives
  Hv, one all-reduce(max) gives the MIP; both match the single-process result.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    import oracle
    from paper_2208_11422_gb300 import synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # bench aggregation: rank r pretends to take (r+1) seconds for 4 steps
        tmax = bench.dist_max(float(rank + 1), world)
        value = bench.aggregate(4, world, tmax)
        # depth split
        N, L, Nz, k = 5, 6, 5, 3
        H = W = N * L
        psf = synth.random_psf(12, N, Nz, k * N).astype(np.float64)
        v = synth.random_volume(13, Nz, H, W).astype(np.float64)
        a, b = Nz * rank // world, Nz * (rank + 1) // world
        part = torch.from_numpy(oracle.forward(psf[a:b], N, v[a:b], nthreads=2))
        dist.all_reduce(part, op=dist.ReduceOp.SUM)
        mip = torch.from_numpy(v[a:b].max(axis=0).copy())
        dist.all_reduce(mip, op=dist.ReduceOp.MAX)
        q.put((rank, tmax, value, part.numpy(), mip.numpy()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_gloo_ranks(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    import oracle
    from paper_2208_11422_gb300 import synth
    N, L, Nz, k = 5, 6, 5, 3
    H = W = N * L
    psf = synth.random_psf(12, N, Nz, k * N).astype(np.float64)
    v = synth.random_volume(13, Nz, H, W).astype(np.float64)
    full = oracle.forward(psf, N, v)
    for rank, tmax, value, hv, mip in res:
        assert tmax == float(world)
        assert value == 4 * world / float(world)
        np.testing.assert_allclose(hv, full, rtol=1e-13)
        assert np.array_equal(mip, v.max(axis=0))


# ------------------------------------------------ depth-split orchestration --
# The library's depth-split loop (paper_2208_11422_gb300.depth_split: the call
# order, the local and cross-process sum / max reductions, the stopping rule)
# driven over shards whose arithmetic is the FP64 oracle's, on CPU.
# the tiny workload's geometry (Nnum 5, 75 px, 5 depths, PSF 25 px) with a
# frame whose entropy peaks at iteration 7, so the stopping rule acts
SPLIT_CASE = dict(N=5, L=15, Nz=5, k=5, n=12)


def _split_problem():
    import oracle
    from paper_2208_11422_gb300 import synth
    g = synth.CONFIGS[0]
    psf = synth.make_psf(0).astype(np.float64)
    vt = synth.timelapse_beads(0, 1, 300, step_sigma=1.0)[0]
    y = synth.poisson_data(oracle.forward(psf, g.nnum, vt), 100.0, g.background, 310).astype(np.float64)
    return psf, y


class OracleShard:
    """A depth part [z0, z1) computed with the FP64 oracle (test side)."""

    def __init__(self, psf, N, z0, z1, H, W, XS, YS):
        from oracle import rl as orl
        self.psf, self.N, self.XS, self.YS = psf[z0:z1], N, XS, YS
        self.ht1 = orl.ht_one(self.psf, N, H, W)
        self.v = self.prev = None

    def load(self, v):
        self.v = np.array(v, np.float64)

    def forward(self, out):
        import oracle
        out.copy_(torch.from_numpy(oracle.forward(self.psf, self.N, self.v)))

    def update(self, y, hv, mip_out, flux_out):
        import oracle
        from oracle.rl import EPS
        yy, h = y.numpy(), hv.numpy()
        den = h + EPS
        with np.errstate(divide="ignore", invalid="ignore"):
            r = np.where(den > 0, yy / den, 0.0)
            x = oracle.backward(self.psf, self.N, r)
            vn = np.where(self.ht1 > 0, self.v * x / self.ht1, 0.0)
        vn = np.where(np.isnan(vn), 0.0, np.maximum(vn, 0.0))
        self.prev, self.v = self.v, vn
        mip_out.copy_(torch.from_numpy(vn.max(axis=0)))
        flux_out.fill_(float(np.sum(self.ht1 * vn)))

    def quality(self, mip):
        from oracle import metric
        return metric.dct_entropy(mip.numpy(), self.XS, self.YS)

    def part(self, previous):
        return self.prev if previous else self.v


def _split_run(shard_ranges, stop, reducer=None):
    from oracle import metric
    from paper_2208_11422_gb300 import depth_split
    psf, y = _split_problem()
    c = SPLIT_CASE
    H = W = c["N"] * c["L"]
    XS, YS = metric.region_size(c["N"], H, W)
    shards = []
    for z0, z1 in shard_ranges:
        s = OracleShard(psf, c["N"], z0, z1, H, W, XS, YS)
        s.load(np.ones((z1 - z0, H, W)))
        shards.append(s)
    res = depth_split.split_rl(shards, torch.from_numpy(y), c["n"], stop, reducer)
    return res, [s.part(res.previous) for s in shards]


def _split_worker(rank, world, port, stop, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    from paper_2208_11422_gb300 import depth_split
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rng = depth_split.depth_ranges(SPLIT_CASE["Nz"], world)[rank]
        res, parts = _split_run([rng], stop, depth_split.Reducer())
        q.put((rank, rng, res.iters_done, res.predicted, res.previous, res.entropy, res.flux, parts[0]))
    finally:
        dist.destroy_process_group()


def _oracle_reference(stop):
    from oracle import metric
    from oracle import rl as orl
    psf, y = _split_problem()
    c = SPLIT_CASE
    H = c["N"] * c["L"]
    XS, YS = metric.region_size(c["N"], H, H)
    ref = orl.rl(psf, c["N"], y, c["n"], XS, YS, keep_iterates=True)
    done = c["n"]
    if stop:
        for k in range(1, c["n"]):
            if ref.entropy[k] < ref.entropy[k - 1]:
                done = k
                break
    return ref, done


def test_split_depth_ranges():
    from paper_2208_11422_gb300 import depth_split
    assert depth_split.depth_ranges(51, 2) == [(0, 25), (25, 51)]
    r = depth_split.depth_ranges(51, 8)
    assert r[0][0] == 0 and r[-1][1] == 51 and all(a[1] == b[0] for a, b in zip(r, r[1:]))
    assert max(b - a for a, b in r) - min(b - a for a, b in r) <= 1
    with pytest.raises(ValueError):
        depth_split.depth_ranges(3, 4)


@pytest.mark.parametrize("stop", [False, True])
def test_split_rl_local_parts_match_oracle_rl(stop):
    """Three depth parts in one process (local reductions only) against the
    oracle's unsplit RL loop."""
    ref, done = _oracle_reference(stop)
    res, parts = _split_run([(0, 1), (1, 3), (3, 5)], stop)
    assert res.iters_done == done == (7 if stop else SPLIT_CASE["n"])
    assert res.previous == stop
    assert res.predicted == ref.predicted
    np.testing.assert_allclose(res.entropy, ref.entropy[:len(res.entropy)], rtol=1e-12)
    np.testing.assert_allclose(res.flux, ref.flux[:len(res.flux)], rtol=1e-12)
    v = np.concatenate(parts)
    np.testing.assert_allclose(v, ref.iterates[done - 1], rtol=1e-11, atol=1e-14)


@pytest.mark.parametrize("stop", [False, True])
def test_split_rl_gloo_ranks_match_oracle_rl(stop):
    """Two gloo ranks, one depth part each: the all-reduces of the forward
    projection (sum), the z-maximum (max) and the flux (sum) give every rank
    the unsplit iteration's entropies, flux and stopping iteration."""
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_split_worker, args=(r, world, port, stop, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ref, done = _oracle_reference(stop)
    for rank, (z0, z1), iters_done, pred, previous, ent, flux, part in res:
        assert iters_done == done and previous == stop
        assert done == (7 if stop else SPLIT_CASE["n"])
        assert pred == ref.predicted
        np.testing.assert_allclose(ent, ref.entropy[:len(ent)], rtol=1e-12)
        np.testing.assert_allclose(flux, ref.flux[:len(flux)], rtol=1e-12)
        np.testing.assert_allclose(part, ref.iterates[done - 1][z0:z1], rtol=1e-11, atol=1e-14)
