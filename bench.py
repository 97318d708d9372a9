"""Benchmark: Richardson-Lucy iterations per second on the large light-field
workload (2025x2025 px sensor, Nnum 15, 51 depths, PSF 345 px; 5000 beads + 200
filaments, y = Poisson(1000 Hv) + 10), one step = one RL iteration (forward
projection, ratio, backprojection, update + MIP + flux, DCT-entropy metric).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision P] [--impl lfd|reference]

Prints one JSON line (rank 0). With N > 1 (torchrun, one process per GPU)
every rank reconstructs its own frame (independent replicas, weak scaling);
the time is the maximum over ranks. ``--impl reference`` times the FP64 CPU
oracle on a bounded sample of the same workload (the reference arm).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD_CFG = 2
CROP_LENSLETS = 13      # CPU-baseline sample: 195x195 px crop of the frame


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=None)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="lfd", choices=["lfd", "reference"])
    p.add_argument("--precision", default=None, choices=["fp32", "tf32", "bf16", "bf16x3"])
    p.add_argument("--variant", default="fft", choices=["fft", "direct"])
    p.add_argument("--config", type=int, default=WORKLOAD_CFG)
    p.add_argument("--workload", default="large", choices=["large", "batch", "serve"],
                   help="large: one 2025x2025 px frame; batch: 64-frame time-lapse at 615x615 px; "
                        "serve: Poisson request stream over 4 PSF sets")
    p.add_argument("--frames", type=int, default=64)
    p.add_argument("--requests", type=int, default=2000, help="serving: requests in the stream")
    p.add_argument("--rate", type=float, default=20.0, help="serving: mean arrivals per second")
    p.add_argument("--pool", type=int, default=256, help="serving: distinct frames")
    p.add_argument("--serve-requests", type=int, default=600,
                   help="requests of the serving run inside the default (large-frame) line")
    p.add_argument("--no-serve", action="store_true",
                   help="default line without its serving run")
    p.add_argument("--no-batch", action="store_true",
                   help="default line without its time-lapse batch run")
    p.add_argument("--serve-frames", type=int, default=32, help="serving: frames per PSF set batch")
    p.add_argument("--cap", type=int, default=40)
    p.add_argument("--depths", type=int, default=None,
                   help="override the number of depths (small cases for profiler captures)")
    p.add_argument("--lenslets", type=int, default=None,
                   help="override the lenslets per side (small cases for profiler captures)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--skip-fp32-ref", action="store_true")
    return p.parse_args()


# ------------------------------------------------------------ distributed --
def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl"
        try:
            import torch
            if not torch.cuda.is_available():
                backend = "gloo"
        except Exception:
            backend = "gloo"
        dist.init_process_group(backend=backend)
    return rank, world, local


def dist_barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def dist_max(x: float, world: int, device=None) -> float:
    """Maximum of a float over ranks (the slowest rank sets the job time)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(units_per_rank: float, world: int, max_seconds: float) -> float:
    """Whole-job throughput: units every rank processed over the slowest rank's time."""
    return units_per_rank * world / max_seconds


# ------------------------------------------------------------------ clocks --
class ClockSampler:
    """Samples nvidia-smi SM clocks and throttle reasons while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            if self.thread:
                self.thread.join(timeout=2)

    def summary(self):
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = max(smax, float(f[2]))
            except ValueError:
                continue
            for n, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": smax or None, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


# ------------------------------------------------------------------ inputs --
def make_inputs(cfg: int, depths=None, lenslets=None):
    """PSF, ground truth and the seeded parameters of the workload (optionally
    with another number of depths or lenslets, for small profiler cases)."""
    import dataclasses
    from paper_2208_11422_gb300 import synth
    g = synth.CONFIGS[cfg]
    if lenslets:
        g = dataclasses.replace(g, lenslets=lenslets,
                                beads=max(1, g.beads * lenslets ** 2 // g.lenslets ** 2),
                                filaments=g.filaments * lenslets // g.lenslets,
                                name=g.name + "_%dl" % lenslets)
    if depths:
        g = dataclasses.replace(g, nz=depths, z_c=depths // 2,
                                beads=max(1, g.beads * depths // g.nz),
                                filaments=g.filaments * depths // g.nz,
                                name=g.name + "_%dz" % depths)
    psf = synth.make_psf(g)
    vt = synth.ground_truth(g, seed=100 + cfg)
    return g, psf, vt


def algorithmic_flops_per_projection(g) -> float:
    # 2 flops per multiply-add, H*W*Nz*P^2 multiply-adds
    return 2.0 * g.H * g.W * g.nz * g.P * g.P


# ------------------------------------------------------------- CPU baseline --
def cpu_baseline_sample(cfg: int, psf=None):
    """One oracle RL iteration on a 195x195 px crop of the workload (13x13
    lenslets, same Nnum, depths and PSF), scaled to the full frame by the exact
    ratio of multiply-adds. Returns (iterations/s, seconds, sample text, cores)."""
    import oracle
    from oracle import rl as orl
    from paper_2208_11422_gb300 import synth
    g = synth.CONFIGS[cfg]
    Lc = min(CROP_LENSLETS, g.lenslets)
    Hc = Wc = Lc * g.nnum
    psf = (synth.make_psf(cfg) if psf is None else psf).astype(np.float64)
    vt = synth.beads(100 + cfg, g.nz, Hc, Wc, max(1, g.beads * Lc * Lc // (g.lenslets ** 2)),
                     g.bead_radius, g.amp_lo)
    y = synth.poisson_data(oracle.forward(psf, g.nnum, vt), g.scale, g.background, 200 + cfg)
    ht1 = orl.ht_one(psf, g.nnum, Hc, Wc)
    v = np.ones((g.nz, Hc, Wc))
    cores = oracle.default_threads()
    t0 = time.perf_counter()
    vn, _ = orl.rl_step(psf, g.nnum, y, v, ht1)
    from oracle.metric import dct_entropy, mip_z, region_size
    XS, YS = region_size(g.nnum, Hc, Wc)
    dct_entropy(mip_z(vn), XS, YS)
    dt = time.perf_counter() - t0
    ratio = oracle.macs_per_projection(g.P, g.nz, g.H, g.W) / oracle.macs_per_projection(g.P, g.nz, Hc, Wc)
    it_s = 1.0 / (dt * ratio)
    sample = ("one FP64 RL iteration (forward, ratio, backward, update, metric) on a %dx%d px crop "
              "(%dx%d lenslets, Nz %d, PSF %d px) took %.2f s; scaled to the full %dx%d frame by the "
              "exact multiply-add ratio %.1f" % (Hc, Wc, Lc, Lc, g.nz, g.P, dt, g.W, g.H, ratio))
    return it_s, dt, sample, cores


# ------------------------------------------------------ accuracy vs oracle --
ACC_CROP = 256     # crop 0 of the four seeded 256x256 test crops (default_rng(300))
ACC_BLOCK = 64     # backprojection checked at every depth of the crop's central 64x64 voxels


def accuracy_regions(g):
    """(i0, j0) of the forward crop and of the backprojection block."""
    rng = np.random.default_rng(300)
    i0 = int(rng.integers(0, g.H - ACC_CROP + 1))
    j0 = int(rng.integers(0, g.W - ACC_CROP + 1))
    d = (ACC_CROP - ACC_BLOCK) // 2
    return (i0, j0), (i0 + d, j0 + d)


def ratio_like_image(g):
    """The backprojection's input for the accuracy check: uniform in [0.5, 1.5]."""
    from paper_2208_11422_gb300 import synth
    return synth.random_image(7, g.H, g.W, 0.5, 1.5)


def gpu_crop_outputs(lfd, torch, ctx, g, vt_d, r_d):
    """A path's full-frame forward of the ground truth and backprojection of
    the ratio-like image, cut to the accuracy regions (host arrays)."""
    (i0, j0), (b0, b1) = accuracy_regions(g)
    hv = torch.empty((g.H, g.W), device=vt_d.device)
    ht = torch.empty((g.nz, g.H, g.W), device=vt_d.device)
    lfd.lfd_forward(ctx, vt_d, hv)
    lfd.lfd_backward(ctx, r_d, ht)
    torch.cuda.synchronize()
    f = hv[i0:i0 + ACC_CROP, j0:j0 + ACC_CROP].cpu().numpy()
    b = ht[:, b0:b0 + ACC_BLOCK, b1:b1 + ACC_BLOCK].cpu().numpy()
    del hv, ht
    return f, b


def oracle_crop_values(g, psf, vt, r):
    """The FP64 oracle on the accuracy regions (part of the CPU-baseline leg)."""
    import oracle
    (i0, j0), (b0, b1) = accuracy_regions(g)
    psf64 = psf.astype(np.float64)
    f = oracle.forward_crop(psf64, g.nnum, vt, i0, i0 + ACC_CROP, j0, j0 + ACC_CROP)
    b = oracle.backward_block(psf64, g.nnum, r, 0, g.nz, b0, b0 + ACC_BLOCK, b1, b1 + ACC_BLOCK)
    return f, b


def rel_l2(a, b) -> float:
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


# ---------------------------------------------------------------- GPU arm --
PATH_NAMES = {("fft", "fp32"): "fft_fp32", ("fft", "bf16x3"): "fft_bf16x3", ("fft", "bf16"): "fft_bf16",
              ("direct", "bf16x3"): "direct_bf16x3", ("direct", "bf16"): "direct_bf16",
              ("direct", "tf32"): "direct_tf32", ("direct", "fp32"): "direct_fp32"}


def fft_plan_numbers(g, plan):
    """(F, bins, tiles, Cf, S, C) of the FFT tiling the library chose (lfd_get_fft_plan)."""
    N = g.nnum
    S, C = N * N, g.nz * N * N
    return plan["F"], plan["bins"], plan["tiles"], (C + 7) // 8 * 8, S, C


# DRAM bytes (read + write) per launch from one ncu capture, by (workload,
# precision, kernel); each entry names its summary under profiles/ and is
# removed when that kernel changes. The volume transforms' traffic grows in
# proportion to the channels C, so their 4-depth capture is scaled by
# 11475 / 900; the contractions' does not (the share of kept lo tiles and the
# transformed volume's re-reads depend on the depths), so they have no entry.
NCU_TRAFFIC = {
    # 4-depth case (C = 900 channels, 1024 transformed); reads scale with the
    # channels read (C for the volume, Cf = 904 for the spectra), writes with
    # the channels written (Cw = 1024 for the planes, C for the volume)
    ("lf_large_2025px_51z_psf345", "bf16x3", "forward volume transform"):
        (84.584e6 * 11475 / 900 + 213.216e6 * 11520 / 1024, "profiles/fft_lf_large_2025px_51z_psf345_bf16x3.md"),
}


# dense tensor rates relative to BF16 (nominal: TF32 1.1, BF16 2.25 PFLOP/s)
TF32_OVER_BF16 = 1.1 / 2.25


def direct_tensor_roofline(g, prec, st_ms):
    """Tensor-pipe fraction of the direct (implicit GEMM) projections: the
    algorithmic flops 2*H*W*Nz*P^2 per projection, and the executed ones (the
    dense tap union (k+2)^2/k^2, three products per term in split BF16),
    against the sustained BF16 peak (the projections run inside a long step);
    TF32 against that peak times the nominal TF32 / BF16 ratio."""
    peaks, src = measured_peaks()
    k = g.psf_lenslets
    fl = algorithmic_flops_per_projection(g)
    ex = fl * ((k + 2) / k) ** 2 * (3 if prec == "bf16x3" else 1)
    ms = max(st_ms[0], st_ms[2])
    peak = peaks["bf16_tflops_sustained"] * (TF32_OVER_BF16 if prec == "tf32" else 1.0)
    if prec == "tf32":
        src += ", x %.3f nominal TF32/BF16" % TF32_OVER_BF16
    return {"kernel": "forward projection" if st_ms[0] >= st_ms[2] else "backprojection",
            "algorithmic_TFLOPs": fl / (ms / 1e3) / 1e12, "executed_TFLOPs": ex / (ms / 1e3) / 1e12,
            "peak": peak, "frac_algorithmic": fl / (ms / 1e3) / 1e12 / peak,
            "frac_executed": ex / (ms / 1e3) / 1e12 / peak,
            "peak_source": "bf16_tflops_sustained (%s)" % src}


def fft_kernel_work(g, plan, prec, spectra=None):
    """Algorithmic bytes (and contraction flops) per launch of the FFT
    variant's four large kernels. Data spectra are 8 bytes per complex value
    (BF16 hi/lo planes of real and imaginary part, or complex64); the PSF
    spectra are the bytes of the planes the contraction streams
    (lfd_get_spectra: 8 bytes per value in split BF16, less with adaptive lo
    planes, 4 with BF16 spectra), else 8 bytes per complex64 value. Executed
    flops count every tensor-core product (three per term in split BF16, two
    with BF16 PSF spectra)."""
    F, bins, nt, _, S, C = fft_plan_numbers(g, plan)
    L2 = (g.H // g.nnum) * (g.W // g.nnum)
    vol = 4.0 * C * L2
    xs, ys = 8.0 * bins * nt * C, 8.0 * bins * nt * S
    ws = float(spectra["bytes"]) if spectra and spectra.get("bytes") else 8.0 * bins * S * C
    flops = 8.0 * bins * S * nt * C * {"bf16x3": 3, "bf16": 2}.get(prec, 1)
    return {"volume_r2c": {"bytes": vol + xs, "slot": 8, "kernel": "forward volume transform"},
            "forward_contraction": {"bytes": ws + xs + ys, "flops": flops, "slot": 5,
                                    "kernel": "forward contraction"},
            "backward_contraction": {"bytes": ws + ys + xs, "flops": flops, "slot": 6,
                                     "kernel": "backward contraction"},
            "volume_c2r": {"bytes": xs + vol, "slot": 9, "kernel": "backward volume transform"},
            # fused update: read v, H^T r, 1 / H^T 1, write v (4 B each per voxel), write the MIP
            "update": {"bytes": 4.0 * vol + 4.0 * g.H * g.W, "slot": 3, "kernel": "fused update + MIP + flux"}}, \
        {"F": F, "bins": bins, "tiles": nt}


def fft_roofline(g, plan, prec, stage, peaks, peak_src, fp32_peak, smax, spectra=None):
    """Roofline of the slowest of the FFT variant's kernels (by the stage
    times measured with CUDA events), and every kernel's fractions beside it."""
    work, shape = fft_kernel_work(g, plan, prec, spectra)
    kern = {}
    for name, w in work.items():
        ms = stage[w["slot"]]
        if ms <= 0:
            continue
        gbs = w["bytes"] / (ms / 1e3) / 1e9
        e = {"ms": ms, "algorithmic_bytes": w["bytes"], "GBps": gbs, "hbm_frac": gbs / peaks["hbm_gbs"]}
        t = NCU_TRAFFIC.get((g.name, prec, w["kernel"]))
        e["traffic"] = t[0] if t else None
        if "flops" in w:
            tf = w["flops"] / (ms / 1e3) / 1e12
            e["TFLOPs"] = tf
            if prec == "fp32":
                e["alu_frac"] = tf / fp32_peak
        kern[name] = e
    dom = max(kern, key=lambda k: kern[k]["ms"])
    d = kern[dom]
    if prec == "fp32" and "alu_frac" in d and d["alu_frac"] > d["hbm_frac"]:
        roof = {"bound": "alu", "achieved": d["TFLOPs"], "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": d["alu_frac"],
                "peak_source": "FP32 FMA: 152 SMs x 128 lanes x 2 flop x %g MHz" % smax}
    else:
        roof = {"bound": "hbm", "achieved": d["GBps"], "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": d["hbm_frac"], "peak_source": "hbm_gbs (%s, of measured)" % peak_src
                if peak_src == "measured" else "hbm_gbs (fallback)"}
    roof["kernel"] = work[dom]["kernel"]
    roof["algorithmic_per_launch"] = dict(shape, bytes=work[dom]["bytes"],
                                          **({"flops": work[dom]["flops"]} if "flops" in work[dom] else {}))
    t = NCU_TRAFFIC.get((g.name, prec, work[dom]["kernel"]))
    roof["traffic"] = t[0] if t else None
    if t:
        roof["traffic_source"] = t[1]
    roof["kernels"] = kern
    return roof


def time_path(lfd, torch, dev, psf_d, g, y_d, variant, precision, iters, warm, stream, acc=None):
    """RL iterations/s of one path; returns (it/s, stage times, final volume,
    crop outputs for the accuracy check or None). acc: (vt_d, r_d) or None."""
    ctx = lfd.lfd_create(psf_d, g.P, g.nnum, g.nz, g.H, g.W,
                         lfd.lfd_default_options(precision=precision, variant=variant))
    try:
        crops = gpu_crop_outputs(lfd, torch, ctx, g, *acc) if acc else None
        v = torch.ones((g.nz, g.H, g.W), device=dev)
        if warm:
            lfd.lfd_rl_iterate(ctx, y_d, v, warm)
            v.fill_(1.0)
        torch.cuda.synchronize()
        lfd.lfd_set_profiling(ctx, True)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        lfd.lfd_rl_iterate(ctx, y_d, v, iters, False, stream)
        b.record(stream)
        torch.cuda.synchronize()
        return iters / (a.elapsed_time(b) / 1e3), lfd.lfd_stage_times(ctx), v, crops
    finally:
        lfd.lfd_destroy(ctx)


def run_lfd(args, rank, world, local):
    import torch
    from paper_2208_11422_gb300 import build, lfd, synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()
    lfd.load()
    variant = args.variant
    prec = args.precision or "bf16x3"
    steps = args.steps if args.steps is not None else 5
    warm = max(3, args.warmup)
    g, psf, vt = make_inputs(args.config, args.depths, args.lenslets)
    psf_d = torch.from_numpy(psf).to(dev)
    stream = torch.cuda.current_stream()

    ctx = lfd.lfd_create(psf_d, g.P, g.nnum, g.nz, g.H, g.W,
                         lfd.lfd_default_options(precision=prec, variant=variant))
    fft_plan = lfd.lfd_get_fft_plan(ctx)
    spectra = lfd.lfd_get_spectra(ctx)
    # data: y = Poisson(scale * H v_true) + background; H v_true by this path's
    # forward projection (an input for timing, never an expected value)
    vt_d = torch.from_numpy(vt.astype(np.float32)).to(dev)
    hv = torch.empty((g.H, g.W), device=dev)
    lfd.lfd_forward(ctx, vt_d, hv)
    torch.cuda.synchronize()
    y = synth.poisson_data(hv.cpu().numpy(), g.scale, g.background, 200 + args.config)
    del hv
    y_d = torch.from_numpy(y).to(dev)
    # accuracy against the oracle (rank 0 at N = 1, with the CPU-baseline leg):
    # every path's forward of the ground truth and backprojection of a
    # ratio-like image on crop 0 of the four seeded test crops
    do_acc = rank == 0 and world == 1 and not args.no_cpu_baseline and not args.depths \
        and not args.lenslets
    acc_in = None
    gpu_crops = {}
    if do_acc:
        r_img = ratio_like_image(g)
        acc_in = (vt_d, torch.from_numpy(r_img).to(dev))
        gpu_crops[(variant, prec)] = gpu_crop_outputs(lfd, torch, ctx, g, *acc_in)
    else:
        del vt_d
    v = torch.ones((g.nz, g.H, g.W), device=dev)

    # warm-up (untimed)
    lfd.lfd_rl_iterate(ctx, y_d, v, warm)
    v.fill_(1.0)
    torch.cuda.synchronize()

    # device-resident timed region: one call of `steps` iterations
    lfd.lfd_set_profiling(ctx, True)
    launches0 = lfd.lfd_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        dist_barrier(world)
        torch.cuda.synchronize()
        e0.record(stream)
        done, pred, ent, flux = lfd.lfd_rl_iterate(ctx, y_d, v, steps, False, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        dist_barrier(world)
    launches = lfd.lfd_launch_count() - launches0
    secs = e0.elapsed_time(e1) / 1e3
    stage = lfd.lfd_stage_times(ctx)
    lfd.lfd_set_profiling(ctx, False)
    tmax = dist_max(secs, world, dev)
    value = aggregate(steps, world, tmax)
    v_head = v.clone()

    # end to end through the C ABI, one iteration per call: every step uploads
    # the step's input (the light-field image y) from pinned host memory and
    # reads back its result (the entropy and flux of the new iterate); the
    # volume is the iteration's state and stays in the context (lfd_rl_load
    # before the first step and lfd_rl_store after the last are timed too)
    e2e = None
    e2e_rt = None
    if not args.no_e2e:
        y_h = torch.from_numpy(y).pin_memory()
        v.fill_(1.0)
        lfd.lfd_rl_load(ctx, v)
        lfd.lfd_rl_step(ctx, y_h, 1)          # warm the staging buffers and graphs
        v.fill_(1.0)
        torch.cuda.synchronize()
        dist_barrier(world)
        t0 = time.perf_counter()
        lfd.lfd_rl_load(ctx, v)
        for _ in range(steps):
            ent_k, flux_k = lfd.lfd_rl_step(ctx, y_h, 1)
        lfd.lfd_rl_store(ctx, v)
        torch.cuda.synchronize()
        t_e2e = time.perf_counter() - t0
        dist_barrier(world)
        t_e2e = dist_max(t_e2e, world, dev)
        e2e = {"value": aggregate(steps, world, t_e2e), "unit": "RL iterations/s",
               "h2d_bytes_per_step": int(y_h.numel() * 4), "d2h_bytes_per_step": 16,
               "step": "lfd_rl_step(y in pinned host memory, n=1) on the resident iterate; reads back "
                       "the iterate's entropy and flux (lfd_rl_load of v^0 before the first step and "
                       "lfd_rl_store of the result after the last inside the timed region)"}
        # the same with the whole volume through host memory every iteration
        v_h = torch.ones((g.nz, g.H, g.W)).pin_memory()
        lfd.lfd_rl_iterate(ctx, y_h, v_h, 1)
        v_h.fill_(1.0)
        dist_barrier(world)
        t0 = time.perf_counter()
        for _ in range(steps):
            lfd.lfd_rl_iterate(ctx, y_h, v_h, 1)
        t_rt = time.perf_counter() - t0
        dist_barrier(world)
        t_rt = dist_max(t_rt, world, dev)
        e2e_rt = {"value": aggregate(steps, world, t_rt), "unit": "RL iterations/s",
                  "h2d_bytes_per_step": int(y_h.numel() * 4 + v_h.numel() * 4),
                  "d2h_bytes_per_step": int(v_h.numel() * 4)}
        del y_h, v_h
    lfd.lfd_destroy(ctx)
    del v

    # the other formulations and precisions on the same GPU and data, with the
    # relative L2 distance of their v^steps from this path's
    # (the FFT variant with FP32 contractions runs first: every path's v^steps
    # is also compared with it, the metric's FP32 reference)
    paths = {}
    head_vs_fp32 = None
    if not args.skip_fp32_ref:
        v_fp32 = None
        for var, pr in (("fft", "fp32"), ("fft", "bf16x3"), ("fft", "bf16"), ("direct", "bf16x3"),
                        ("direct", "bf16"), ("direct", "tf32"), ("direct", "fp32")):
            if (var, pr) == (variant, prec):
                continue
            n_it = 1 if (var, pr) == ("direct", "fp32") else steps
            it_s, st_ms, vo, crops = time_path(lfd, torch, dev, psf_d, g, y_d, var, pr, n_it,
                                               0 if n_it == 1 else 2, stream, acc_in)
            if crops is not None:
                gpu_crops[(var, pr)] = crops
            rel = rel32 = None
            if n_it == steps:
                rel = float(torch.linalg.vector_norm(vo - v_head) / torch.linalg.vector_norm(v_head))
                if (var, pr) == ("fft", "fp32"):
                    v_fp32 = vo
                    head_vs_fp32 = rel * float(torch.linalg.vector_norm(v_head) / torch.linalg.vector_norm(vo))
                elif v_fp32 is not None:
                    rel32 = float(torch.linalg.vector_norm(vo - v_fp32) / torch.linalg.vector_norm(v_fp32))
            paths[PATH_NAMES[(var, pr)]] = {
                "value": it_s, "unit": "RL iterations/s", "iterations": n_it,
                "forward_ms": st_ms[0], "backward_ms": st_ms[2],
                "rel_l2_vs_headline_after_%d_iterations" % steps: rel,
                "rel_l2_vs_fft_fp32_after_%d_iterations" % steps: rel32}
            if var == "direct" and pr in ("bf16", "bf16x3", "tf32"):
                paths[PATH_NAMES[(var, pr)]]["tensor_roofline"] = direct_tensor_roofline(g, pr, st_ms)
            if vo is not v_fp32:
                del vo
            torch.cuda.empty_cache()
        del v_fp32
        torch.cuda.empty_cache()

    peaks, peak_src = measured_peaks()
    smax = peaks.get("sm_max_mhz", 2070.0)
    fp32_peak = 152 * 128 * 2 * smax * 1e6 / 1e12   # FP32 FMA lanes x 2 flop x max clock
    fl = algorithmic_flops_per_projection(g)
    stage_names = ["forward", "ratio", "backward", "update", "metric", "forward_contraction",
                   "backward_contraction", "fft_transforms", "volume_r2c", "volume_c2r",
                   "exact_low_sensitivity"]
    stage_ms = dict(zip(stage_names, stage))
    if variant == "fft":
        roof = fft_roofline(g, fft_plan, prec, stage, peaks, peak_src, fp32_peak, smax, spectra)
        roof["psf_spectra"] = spectra
    elif prec == "fp32":
        dom_ms = max(stage[0], stage[2])
        dom = "forward projection" if stage[0] >= stage[2] else "backprojection"
        roof = {"bound": "alu", "kernel": dom, "achieved": fl / (dom_ms / 1e3) / 1e12,
                "peak": fp32_peak, "unit": "TFLOP/s",
                "peak_source": "FP32 FMA: 152 SMs x 128 lanes x 2 x %g MHz" % smax}
        roof["frac"] = roof["achieved"] / roof["peak"]
    else:
        dom_ms = max(stage[0], stage[2])
        dom = "forward projection" if stage[0] >= stage[2] else "backprojection"
        ratio = TF32_OVER_BF16 if prec == "tf32" else 1.0
        peak = peaks["bf16_tflops_sustained"] * ratio
        roof = {"bound": "tensor", "kernel": dom, "achieved": fl / (dom_ms / 1e3) / 1e12,
                "peak": peak, "unit": "TFLOP/s",
                "peak_source": "bf16_tflops_sustained (%s)%s" % (
                    peak_src, " x %.3f nominal TF32/BF16" % ratio if prec == "tf32" else "")}
        roof["frac"] = roof["achieved"] / roof["peak"]
    roof.setdefault("traffic", None)
    roof["stage_ms"] = stage_ms

    cpu = None
    accuracy = None
    if do_acc:
        del acc_in, vt_d
        torch.cuda.empty_cache()
        it_s, dt, sample, cores = cpu_baseline_sample(args.config, psf)
        cpu = {"value": it_s, "unit": "RL iterations/s", "cores": cores, "kind": "oracle",
               "sample": sample, "extrapolated": True, "sample_seconds": dt}
        t0 = time.perf_counter()
        ref_f, ref_b = oracle_crop_values(g, psf, vt, r_img)
        (i0, j0), (b0, b1) = accuracy_regions(g)
        accuracy = {"forward_crop": [i0, j0, ACC_CROP], "backward_block": [b0, b1, ACC_BLOCK, g.nz],
                    "inputs": "forward: the ground-truth volume; backprojection: an image uniform "
                              "in [0.5, 1.5]; oracle: FP64 direct summation",
                    "oracle_seconds": time.perf_counter() - t0, "paths": {}}
        for (var, pr), (gf, gb) in gpu_crops.items():
            accuracy["paths"][PATH_NAMES[(var, pr)]] = {"forward_rel_l2": rel_l2(gf, ref_f),
                                                        "backward_rel_l2": rel_l2(gb, ref_b)}

    clocks = clk.summary()
    # the metric's other two parts on the same GPU (N = 1, full workload only):
    # serving p50 / p99 under a bounded Poisson stream, and the 64-frame time-lapse
    full = world == 1 and not args.depths and not args.lenslets
    torch.cuda.empty_cache()
    serve = batch = None
    if full and not args.no_serve:
        serve = measure_serve(args, rank, world, local, args.serve_requests, args.pool)
    if full and not args.no_batch:
        batch = measure_batch(args, rank, world, local, ("bf16x3", "fp32"))
    out = {
        "metric": "RL iterations/s, 2025x2025 px x 51 depths, PSF 345 px (Nnum 15)",
        "value": value, "unit": "RL iterations/s", "n_gpus": world, "steps": steps,
        "warmup": warm, "ms_per_step": tmax * 1e3 / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "tf32": "tf32", "bf16": "bf16", "bf16x3": "bf16x3"}[prec],
        "data": "synthetic (seeded beads + filaments, Poisson noise)",
        "config": frame_config(g, world), "path": {"variant": variant, "precision": prec},
        "e2e": e2e, "e2e_volume_roundtrip": e2e_rt, "gpu_launches": launches, "clocks": clocks,
        "roofline": roof, "cpu_baseline": cpu, "paths": paths, "accuracy_vs_oracle": accuracy,
        "rel_l2_vs_fft_fp32_after_%d_iterations" % steps: head_vs_fp32,
        "entropy": ent, "predicted_iteration": pred,
        "serve": serve,
        "batch": {"workload": "lf_timelapse_%dx615px_31z_psf165" % args.frames, "frames": args.frames,
                  "cap": args.cap, "paths": batch} if batch else None,
    }
    if rank == 0:
        print(json.dumps(out), flush=True)


def measure_batch(args, rank, world, local, precisions=("bf16x3", "bf16", "fp32")):
    """Time-lapse batch: frames of the 615 px geometry sharing one PSF, beads
    drifting by N(0, 0.5) voxel per frame, photon scale per frame U[100, 2000];
    all frames advance together (one launch per stage, one CUDA graph per
    iteration) and each stops at its own predicted iteration (cap --cap).
    Returns {precision: result} (frames/s over all ranks, the tuned FFT size,
    stopping iterations)."""
    import torch
    from paper_2208_11422_gb300 import lfd, synth

    dev = torch.device("cuda", local)
    g = synth.CONFIGS[1]
    nf, cap = args.frames, args.cap
    psf = synth.make_psf(1)
    psf_d = torch.from_numpy(psf).to(dev)
    vols = synth.timelapse_beads(1, nf, 103 + 1000 * rank)
    scales = synth.timelapse_scales(nf, 203 + 1000 * rank)
    ctx = lfd.lfd_create(psf_d, g.P, g.nnum, g.nz, g.H, g.W,
                         lfd.lfd_default_options(precision="fp32", variant="fft"))
    hv = torch.empty((g.H, g.W), device=dev)
    ys = []
    for f in range(nf):
        lfd.lfd_forward(ctx, torch.from_numpy(vols[f].astype(np.float32)).to(dev), hv)
        torch.cuda.synchronize()
        ys.append(synth.poisson_data(hv.cpu().numpy(), scales[f], 5.0, 303 + f + 1000 * rank))
    lfd.lfd_destroy(ctx)
    del vols
    y_d = torch.from_numpy(np.stack(ys)).to(dev)
    stream = torch.cuda.current_stream()
    results = {}
    for prec in precisions:
        opt = lfd.lfd_default_options(precision=prec, variant="fft", max_frames=nf)
        tune_ms, _ = lfd.lfd_autotune_options(psf_d, g.P, g.nnum, g.nz, g.H, g.W, opt)
        best, cols = opt.fft_size, opt.contraction_cols
        ctx = lfd.lfd_create(psf_d, g.P, g.nnum, g.nz, g.H, g.W, opt)
        v = torch.ones((nf, g.nz, g.H, g.W), device=dev)
        lfd.lfd_rl_iterate_batch(ctx, nf, y_d, v, 1)   # warm-up
        v.fill_(1.0)
        l0 = lfd.lfd_launch_count()
        with ClockSampler(local) as clk:
            dist_barrier(world)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            done, pred, ent, _ = lfd.lfd_rl_iterate_batch(ctx, nf, y_d, v, cap, True, stream)
            b.record(stream)
            torch.cuda.synchronize()
            dist_barrier(world)
        secs = dist_max(a.elapsed_time(b) / 1e3, world, dev)
        ran = max(sum(1 for e in row if e == e) for row in ent)
        results[prec] = {"frames_per_s": aggregate(nf, world, secs), "seconds": secs,
                         "iterations_run": ran, "iters_done": done,
                         "frame_iterations_per_s": aggregate(nf * ran, world, secs),
                         "fft_size": best, "contraction_cols": cols or "widest needed",
                         "autotune_ms_per_iteration": tune_ms,
                         "gpu_launches": lfd.lfd_launch_count() - l0, "clocks": clk.summary()}
        lfd.lfd_destroy(ctx)
        if prec == precisions[0]:
            # the same run with one launch per stage instead of a CUDA-graph
            # replay per iteration: what the launches cost between the kernels
            opt.use_graph = 0
            ctx = lfd.lfd_create(psf_d, g.P, g.nnum, g.nz, g.H, g.W, opt)
            v.fill_(1.0)
            lfd.lfd_rl_iterate_batch(ctx, nf, y_d, v, 1)
            v.fill_(1.0)
            torch.cuda.synchronize()
            a.record(stream)
            lfd.lfd_rl_iterate_batch(ctx, nf, y_d, v, cap, True, stream)
            b.record(stream)
            torch.cuda.synchronize()
            results[prec]["plain_launches_seconds"] = a.elapsed_time(b) / 1e3
            lfd.lfd_destroy(ctx)
        del v
        torch.cuda.empty_cache()
    if "fp32" in results:
        for prec in results:   # frames whose stopping iteration equals the FP32 run's
            if prec != "fp32":
                results[prec]["stops_equal_to_fp32"] = sum(
                    int(d == e) for d, e in zip(results[prec]["iters_done"], results["fp32"]["iters_done"]))
    del psf_d, y_d
    torch.cuda.empty_cache()
    return results


def run_batch(args, rank, world, local):
    import torch
    from paper_2208_11422_gb300 import build, lfd
    torch.cuda.set_device(local)
    build.build()
    lfd.load()
    nf, cap = args.frames, args.cap
    results = measure_batch(args, rank, world, local)
    head = results["bf16x3"]
    out = {
        "metric": "RL frames/s, %d-frame time-lapse 615x615 px x 31 depths, PSF 165 px, each frame "
                  "stopped at its predicted iteration (cap %d)" % (nf, cap),
        "value": head["frames_per_s"], "unit": "frames/s", "n_gpus": world, "steps": 1, "warmup": 1,
        "ms_per_step": head["seconds"] * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16x3", "data": "synthetic (drifting beads, Poisson noise)",
        "config": {"workload": "lf_timelapse_%dx615px_31z_psf165" % nf, "frames": nf, "cap": cap,
                   "variant": "fft", "precision": "bf16x3"},
        "gpu_launches": head["gpu_launches"], "clocks": head["clocks"], "paths": results,
    }
    if rank == 0:
        print(json.dumps(out), flush=True)


def measure_serve(args, rank, world, local, requests, pool_size):
    """Serving: a Poisson stream of `requests` requests (mean --rate per second)
    over 4 resident PSF sets (Nnum, Nz drawn per set, PSF 11 lenslets wide).
    Each request has its own lenslet grid (33..121 per axis), bead count
    (50..5000) and photon scale (log-uniform 100..5000). The server admits
    requests by device footprint, batches them per PSF set in split BF16 and
    stops each at its predicted iteration (cap --cap). The frames' data come
    from a pool of `pool_size` distinct requests (bead volumes made on the
    device, projected once before the run); arrival i uses pool entry
    i mod pool_size. Host buffers are page-locked. Returns the summary."""
    import collections
    import torch
    from paper_2208_11422_gb300 import lfd, synth

    dev = torch.device("cuda", local)
    sets = [synth.serve_psf_set(j) for j in (1, 2, 3, 4)]
    pool = synth.serve_requests(pool_size, 910 + rank)
    arrivals = synth.serve_requests(requests, 920 + rank, args.rate)
    Lmax = synth.SERVE_LENSLETS[1]
    # pool data: y = Poisson(scale * H v) + 5 with H v from an FP32 context at the
    # largest sensor of the set (the volume is zero outside the request's frame,
    # so the crop is the frame's own projection)
    ys = [None] * len(pool)
    t_prep = time.perf_counter()
    for si, (nnum, nz, P, psf) in enumerate(sets):
        Hm = Lmax * nnum
        ctx = lfd.lfd_create(torch.from_numpy(psf).to(dev), P, nnum, nz, Hm, Hm,
                             lfd.lfd_default_options(precision="fp32", variant="fft"))
        vbig = torch.zeros((nz, Hm, Hm), device=dev)
        hv = torch.empty((Hm, Hm), device=dev)
        for k, rq in enumerate(pool):
            if rq.set_id != si + 1:
                continue
            H, W = rq.ly * nnum, rq.lx * nnum
            vbig.zero_()
            synth.beads_device(rq.seed, nz, H, W, rq.beads, 2.0, 0.3, device=dev, out=vbig[:, :H, :W])
            lfd.lfd_forward(ctx, vbig, hv)
            torch.cuda.synchronize()
            ys[k] = torch.from_numpy(synth.poisson_data(hv[:H, :W].cpu().numpy(), rq.scale, 5.0,
                                                        rq.seed + 7)).pin_memory()
        lfd.lfd_destroy(ctx)
        del vbig, hv
        torch.cuda.empty_cache()
    t_prep = time.perf_counter() - t_prep

    opt = lfd.lfd_server_default_options("bf16x3", max_iter=args.cap,
                                         max_frames_per_set=args.serve_frames)
    srv = lfd.lfd_server_create(opt)
    ids = [lfd.lfd_server_add_psf(srv, torch.from_numpy(psf).to(dev), P, nnum, nz, Lmax * nnum, Lmax * nnum)
           for nnum, nz, P, psf in sets]
    torch.cuda.synchronize()
    free_v = collections.defaultdict(list)   # pool entry -> page-locked result buffers

    def v_buffer(k):
        if free_v[k]:
            return free_v[k].pop()
        rq = pool[k]
        nnum, nz = sets[rq.set_id - 1][0], sets[rq.set_id - 1][1]
        return torch.empty((nz, rq.ly * nnum, rq.lx * nnum)).pin_memory()

    pending = collections.deque()
    cv = threading.Condition()
    done_rec = []
    submitted = len(arrivals)

    def collector():
        for _ in range(submitted):
            with cv:
                while not pending:
                    cv.wait()
                i, k, req, v, t_arr, t_sub = pending.popleft()
            if req is None:
                done_rec.append((i, None, t_arr, t_sub, time.perf_counter()))
                continue
            r = lfd.lfd_poll(srv, req, -1)
            done_rec.append((i, r, t_arr, t_sub, time.perf_counter()))
            with cv:
                free_v[k].append(v)

    l0 = lfd.lfd_launch_count()
    th = threading.Thread(target=collector)
    th.start()
    rejected = 0
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        for i, a in enumerate(arrivals):
            dt = t0 + a.arrival_s - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            k = i % len(pool)
            rq = pool[k]
            with cv:
                v = v_buffer(k)
            t_sub = time.perf_counter()
            try:
                req = lfd.lfd_submit(srv, ids[rq.set_id - 1], ys[k], v, max_iter=args.cap,
                                     stop_at_predicted=True, entropy_hist=True)
            except lfd.LfdError:
                req = None
                rejected += 1
            with cv:
                pending.append((i, k, req, v, t0 + a.arrival_s, t_sub))
                cv.notify()
        th.join()
        t_end = max(rec[4] for rec in done_rec)
    stats = lfd.lfd_server_stats_get(srv)
    lfd.lfd_server_destroy(srv)
    del ys, free_v
    torch.cuda.empty_cache()
    ok = [rec for rec in done_rec if rec[1] is not None and rec[1]["status"] == lfd.LFD_OK]
    lat = np.array([r["latency_us"] / 1e3 + (t_sub - t_arr) * 1e3 for _, r, t_arr, t_sub, _ in ok])
    queue = np.array([r["queue_us"] / 1e3 for _, r, _, _, _ in ok])
    iters = np.array([r["iters_run"] for _, r, _, _, _ in ok])
    span = t_end - t0
    return {
        "frames_per_s": len(ok) / span, "requests": len(arrivals), "pool": len(pool),
        "rate_req_s": args.rate, "cap": args.cap, "max_frames_per_set": args.serve_frames,
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p90": float(np.percentile(lat, 90)),
                       "p99": float(np.percentile(lat, 99)), "mean": float(lat.mean())},
        "queue_ms_mean": float(queue.mean()),
        "offered_req_s": len(arrivals) / max(a.arrival_s for a in arrivals),
        "achieved_req_s": len(ok) / span,
        "completed": len(ok), "rejected": rejected, "iterations_mean": float(iters.mean()),
        "frame_iterations_per_s": float(iters.sum() / span), "seconds": span,
        "pool_preparation_s": t_prep,
        "server": {k: stats[k] for k in ("ticks", "frame_iterations", "columns", "arena_bytes",
                                         "arena_peak_bytes", "resident_bytes")},
        "psf_sets": [{"Nnum": n, "Nz": z, "P": p} for n, z, p, _ in sets],
        "gpu_launches": lfd.lfd_launch_count() - l0, "clocks": clk.summary(),
    }


def run_serve(args, rank, world, local):
    import torch
    from paper_2208_11422_gb300 import build, lfd
    torch.cuda.set_device(local)
    build.build()
    lfd.load()
    r = measure_serve(args, rank, world, local, args.requests, args.pool)
    out = {
        "metric": "served frames/s, Poisson stream of %d requests at %g req/s over 4 resident PSF sets "
                  "(mixed sensor sizes, Nnum 11-15, 21-51 depths), split BF16, predicted stop (cap %d)"
                  % (r["requests"], args.rate, args.cap),
        "value": r["frames_per_s"], "unit": "frames/s", "n_gpus": world, "steps": r["requests"],
        "warmup": 0, "ms_per_step": r["seconds"] * 1e3 / max(1, r["completed"]), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3",
        "data": "synthetic (beads, Poisson noise; %d distinct frames reused)" % r["pool"],
        "config": {"workload": "lf_serve_4sets_poisson%greq_s" % args.rate, "requests": r["requests"],
                   "rate_req_s": args.rate, "cap": args.cap, "pool": r["pool"],
                   "max_frames_per_set": args.serve_frames, "psf_sets": r["psf_sets"]},
        "gpu_launches": r["gpu_launches"], "clocks": r["clocks"], "serve": r,
    }
    if rank == 0:
        print(json.dumps(out), flush=True)


def frame_config(g, world):
    """The `config` object of the frame workload (both arms print the same; the
    arithmetic each arm ran is in its `dtype` and `path`)."""
    return {"workload": g.name, "H": g.H, "W": g.W, "Nnum": g.nnum, "Nz": g.nz, "P": g.P,
            "parallelism": "replicas" if world > 1 else "single GPU",
            "l2": "inputs larger than L2 (volume %.2f GB)" % (g.nz * g.H * g.W * 4 / 1e9)}


def run_reference(args, rank, world):
    """Reference arm: the FP64 CPU oracle on bounded samples of the workload.
    One step is one oracle RL iteration on a 195x195 px crop (all depths, the
    full PSF); `ms_per_step` is that measured crop iteration, and `value` the
    full frame's iterations/s extrapolated by the exact multiply-add ratio."""
    if rank != 0:
        return
    steps = args.steps if args.steps is not None else 1
    warm = args.warmup
    for _ in range(warm):
        cpu_baseline_sample(args.config)
    vals = []
    sample = cores = None
    for _ in range(steps):
        it_s, dt, sample, cores = cpu_baseline_sample(args.config)
        vals.append(dt)
    from paper_2208_11422_gb300 import synth
    import oracle
    g = synth.CONFIGS[args.config]
    Hc = CROP_LENSLETS * g.nnum
    ratio = oracle.macs_per_projection(g.P, g.nz, g.H, g.W) / oracle.macs_per_projection(g.P, g.nz, Hc, Hc)
    value = 1.0 / (statistics.mean(vals) * ratio)
    out = {
        "impl": "reference",
        "metric": "RL iterations/s, 2025x2025 px x 51 depths, PSF 345 px (Nnum 15)",
        "value": value, "unit": "RL iterations/s", "n_gpus": world, "steps": steps, "warmup": warm,
        "ms_per_step": statistics.mean(vals) * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": frame_config(g, world), "path": {"variant": "oracle", "precision": "f64"},
        "extrapolated": True,
        "extrapolation": {"step": "one FP64 RL iteration on a %dx%d px crop (measured: ms_per_step)"
                                  % (Hc, Hc), "multiply_add_ratio_to_full_frame": ratio},
        "cpu_baseline": {"value": value, "unit": "RL iterations/s", "cores": cores,
                         "kind": "oracle", "sample": sample, "extrapolated": True},
        "e2e": {"value": value, "unit": "RL iterations/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    rank, world, local = dist_init()
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "batch":
        run_batch(args, rank, world, local)
    elif args.workload == "serve":
        run_serve(args, rank, world, local)
    else:
        run_lfd(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
