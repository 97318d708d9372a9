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
