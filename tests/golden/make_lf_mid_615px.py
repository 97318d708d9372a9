"""Writes lf_mid_615px_31z_psf165.npz: the oracle's 10-iteration RL run on the
mid-size light-field workload (Nnum 15, 41x41 lenslets = 615x615 px, 31 depths,
PSF 165 px, 300 beads, y = Poisson(500 Hv) + 5, v^0 = 1, eps = 1e-6).

Calls only ``oracle`` and the seeded generators; nothing here touches the CUDA
path. Run from the repository root:  python tests/golden/make_lf_mid_615px.py
(about 6 minutes on 8 cores).
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from oracle import rl as orl  # noqa: E402
from oracle.metric import region_size  # noqa: E402
from paper_2208_11422_gb300 import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lf_mid_615px_31z_psf165.npz")
NSAMP = 20000


def main():
    g = synth.CONFIGS[1]
    t0 = time.time()
    psf = synth.make_psf(1)
    vt = synth.ground_truth(1)
    hv_true = oracle.forward(psf, g.nnum, vt)
    y = synth.poisson_data(hv_true, g.scale, g.background, 201)
    counts = y.astype(np.float64) - g.background
    assert counts.min() >= 0 and counts.max() < 65535
    assert np.array_equal((counts + g.background).astype(np.float32), y)
    XS, YS = region_size(g.nnum, g.H, g.W)
    res = orl.rl(psf, g.nnum, y, g.iterations, XS, YS, keep_iterates=True)
    vox = synth.sample_indices(301, NSAMP, (g.nz, g.H, g.W))
    take = lambda v: v[vox[:, 0], vox[:, 1], vox[:, 2]]  # noqa: E731
    np.savez_compressed(
        OUT,
        y_counts=counts.astype(np.uint16), background=g.background,
        n_iter=g.iterations, eps=orl.EPS, XS=XS, YS=YS,
        entropy=np.array(res.entropy), flux=np.array(res.flux),
        predicted=res.predicted, sample_vox=vox,
        v_last=take(res.v), v_pred=take(res.iterates[res.predicted - 1]),
        v_first=take(res.iterates[0]),
        mip_last_l2=float(np.linalg.norm(res.v.max(axis=0))),
    )
    print("wrote", OUT, "in %.0f s" % (time.time() - t0), "entropy", res.entropy,
          "predicted", res.predicted)


if __name__ == "__main__":
    main()
