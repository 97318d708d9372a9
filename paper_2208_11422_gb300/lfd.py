"""ctypes binding of liblfd (include/lfd.h), one Python function per C entry point.

Argument marshalling only: every step of the computation runs in the CUDA
library. Array arguments may be torch tensors (CUDA or CPU, contiguous
float32), numpy float32 arrays, or raw integer addresses; streams may be a
``torch.cuda.Stream``, a raw ``cudaStream_t`` integer or None (default stream).
``load()`` raises ``LfdError`` when the library is missing: there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "liblfd.so")

LFD_OK, LFD_EINVAL, LFD_ENOMEM, LFD_ECUDA, LFD_ENOTREADY, LFD_ETIMEDOUT, LFD_EBUSY, \
    LFD_EINTERNAL, LFD_EUNSUPPORTED, LFD_ECANCELED = range(10)
LFD_FP32, LFD_TF32, LFD_BF16, LFD_BF16X3 = range(4)
PRECISIONS = {"fp32": LFD_FP32, "tf32": LFD_TF32, "bf16": LFD_BF16, "bf16x3": LFD_BF16X3}
LFD_DIRECT, LFD_FFT = 0, 1
VARIANTS = {"direct": LFD_DIRECT, "fft": LFD_FFT}


class LfdError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(msg)
        self.status = status


class lfd_options(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int),
        ("eps", ctypes.c_float),
        ("dML_um", ctypes.c_double),
        ("Q", ctypes.c_double),
        ("NA", ctypes.c_double),
        ("lambda_um", ctypes.c_double),
        ("XS", ctypes.c_int),
        ("YS", ctypes.c_int),
        ("l2_over_region", ctypes.c_int),
        ("variant", ctypes.c_int),
        ("max_frames", ctypes.c_int),
        ("use_graph", ctypes.c_int),
        ("fft_size", ctypes.c_int),
        ("spectra_lo_tau", ctypes.c_float),
        ("contraction_cols", ctypes.c_int),
    ]


class lfd_server_options(ctypes.Structure):
    _fields_ = [
        ("opt", lfd_options),
        ("arena_bytes", ctypes.c_int64),
        ("max_frames_per_set", ctypes.c_int),
        ("max_cols", ctypes.c_int),
        ("max_queue", ctypes.c_int),
        ("max_iter", ctypes.c_int),
    ]


class lfd_request(ctypes.Structure):
    _fields_ = [
        ("set_id", ctypes.c_int),
        ("H", ctypes.c_int),
        ("W", ctypes.c_int),
        ("y", ctypes.c_void_p),
        ("v_out", ctypes.c_void_p),
        ("max_iter", ctypes.c_int),
        ("stop_at_predicted", ctypes.c_int),
        ("entropy_hist", ctypes.POINTER(ctypes.c_double)),
    ]


class lfd_result(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int),
        ("iters_done", ctypes.c_int),
        ("iters_run", ctypes.c_int),
        ("predicted", ctypes.c_int),
        ("queue_us", ctypes.c_int64),
        ("latency_us", ctypes.c_int64),
    ]


class lfd_server_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in (
        "submitted", "admitted", "completed", "rejected", "cancelled", "frame_iterations", "ticks",
        "columns", "arena_bytes", "arena_peak_bytes", "resident_bytes")] + [
        ("queued", ctypes.c_int), ("in_flight", ctypes.c_int)]


_lock = threading.Lock()
_lib = None

_VP = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_SIGS = {
    "lfd_default_options": (None, [ctypes.POINTER(lfd_options)]),
    "lfd_create": (_I, [_VP, _I, _I, _I, _I, _I, ctypes.POINTER(lfd_options), _VP,
                        ctypes.POINTER(_VP)]),
    "lfd_forward": (_I, [_VP, _VP, _VP, _VP]),
    "lfd_backward": (_I, [_VP, _VP, _VP, _VP]),
    "lfd_rl_iterate": (_I, [_VP, _VP, _VP, _I, _I, ctypes.POINTER(_I), ctypes.POINTER(_I),
                            ctypes.POINTER(_D), ctypes.POINTER(_D), _VP]),
    "lfd_rl_iterate_batch": (_I, [_VP, _I, _VP, _VP, _I, _I, ctypes.POINTER(_I), ctypes.POINTER(_I),
                                  ctypes.POINTER(_D), ctypes.POINTER(_D), _VP]),
    "lfd_quality": (_I, [_VP, _VP, ctypes.POINTER(_D), _VP]),
    "lfd_autotune": (_I, [_VP, _I, _I, _I, _I, _I, ctypes.POINTER(lfd_options), _VP,
                          ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_float)]),
    "lfd_autotune_options": (_I, [_VP, _I, _I, _I, _I, _I, ctypes.POINTER(lfd_options), _VP,
                                  ctypes.POINTER(ctypes.c_float), ctypes.POINTER(_I)]),
    "lfd_quality_mip_static": (_I, [_VP, _I, _I, _I, _I, _I, _VP, _VP]),
    "lfd_quality_mip": (_I, [_VP, _VP, ctypes.POINTER(_D), _VP]),
    "lfd_rl_load": (_I, [_VP, _VP, _VP]),
    "lfd_rl_step": (_I, [_VP, _VP, _I, ctypes.POINTER(_D), ctypes.POINTER(_D), _VP]),
    "lfd_rl_store": (_I, [_VP, _VP, _VP]),
    "lfd_split_load": (_I, [_VP, _VP, _VP]),
    "lfd_split_forward": (_I, [_VP, _VP, _VP]),
    "lfd_split_update": (_I, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "lfd_split_store": (_I, [_VP, _VP, _I, _VP]),
    "lfd_destroy": (None, [_VP]),
    "lfd_last_error": (ctypes.c_char_p, [_VP]),
    "lfd_status_string": (ctypes.c_char_p, [_I]),
    "lfd_region_size": (_I, [_I, _I, _I, _D, _D, _D, _D, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "lfd_predict_stop": (_I, [ctypes.POINTER(_D), _I]),
    "lfd_get_geometry": (_I, [_VP, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I),
                              ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_int64)]),
    "lfd_get_fft_plan": (_I, [_VP, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I),
                              ctypes.POINTER(_I)]),
    "lfd_get_exact_plan": (_I, [_VP] + [ctypes.POINTER(ctypes.c_int64)] * 4),
    "lfd_get_spectra": (_I, [_VP] + [ctypes.POINTER(ctypes.c_int64)] * 3),
    "lfd_launch_count": (ctypes.c_uint64, []),
    "lfd_debug_fail_allocs": (None, [_I]),
    "lfd_selftest_bounded_wait": (_I, [ctypes.c_int64, ctypes.POINTER(_I)]),
    "lfd_selftest_freelist": (_I, [_I, _I]),
    "lfd_selftest_exact_runs": (_I, [_I, _I, _I, _I, _I]),
    "lfd_selftest_balanced_ranges": (_I, [_I, _I, _I]),
    "lfd_server_default_options": (None, [ctypes.POINTER(lfd_server_options)]),
    "lfd_server_create": (_I, [ctypes.POINTER(lfd_server_options), ctypes.POINTER(_VP)]),
    "lfd_server_add_psf": (_I, [_VP, _VP, _I, _I, _I, _I, _I, ctypes.POINTER(_I)]),
    "lfd_submit": (_I, [_VP, ctypes.POINTER(lfd_request), ctypes.POINTER(ctypes.c_uint64)]),
    "lfd_poll": (_I, [_VP, ctypes.c_uint64, ctypes.c_int64, ctypes.POINTER(lfd_result)]),
    "lfd_cancel": (_I, [_VP, ctypes.c_uint64]),
    "lfd_server_stats_get": (_I, [_VP, ctypes.POINTER(lfd_server_stats)]),
    "lfd_server_last_error": (ctypes.c_char_p, [_VP]),
    "lfd_server_destroy": (None, [_VP]),
    "lfd_set_profiling": (_I, [_VP, _I]),
    "lfd_stage_times": (_I, [_VP, ctypes.POINTER(ctypes.c_float), _I]),
}


def load(path: str | None = None):
    """Load liblfd.so (built by ``paper_2208_11422_gb300.build``); raises if absent."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise LfdError(LFD_EINTERNAL, "liblfd.so not built: run "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
            lib = ctypes.CDLL(p)
            for name, (res, args) in _SIGS.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def exported_names():
    return list(_SIGS)


# ----------------------------------------------------------- marshalling --
def _ptr(x):
    """Address of a contiguous float32 tensor / array, or an int address."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):  # torch.Tensor
        import torch
        if x.dtype != torch.float32 or not x.is_contiguous():
            raise ValueError("tensor must be contiguous float32")
        return x.data_ptr()
    if hasattr(x, "__array_interface__"):
        import numpy as np
        if x.dtype != np.float32 or not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous float32")
        return x.__array_interface__["data"][0]
    raise TypeError("unsupported array argument %r" % type(x))


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return getattr(s, "cuda_stream", s)


def _check(status: int, ctx=None):
    if status != LFD_OK:
        lib = load()
        msg = lib.lfd_last_error(ctx).decode() if ctx else ""
        raise LfdError(status, "%s: %s" % (lib.lfd_status_string(status).decode(), msg))


# ------------------------------------------------------------- entry points --
def lfd_default_options(**overrides) -> lfd_options:
    o = lfd_options()
    load().lfd_default_options(ctypes.byref(o))
    for k, v in overrides.items():
        if k == "precision" and isinstance(v, str):
            v = PRECISIONS[v]
        if k == "variant" and isinstance(v, str):
            v = VARIANTS[v]
        setattr(o, k, v)
    return o


def lfd_create(psf, P: int, Nnum: int, Nz: int, H: int, W: int, opt: lfd_options | None = None,
               stream=None):
    out = _VP()
    st = load().lfd_create(_ptr(psf), P, Nnum, Nz, H, W,
                           ctypes.byref(opt) if opt is not None else None, _stream(stream),
                           ctypes.byref(out))
    if st != LFD_OK:
        raise LfdError(st, "lfd_create failed: %s" % load().lfd_status_string(st).decode())
    return out.value


def lfd_forward(ctx, v, y_out, stream=None):
    _check(load().lfd_forward(ctx, _ptr(v), _ptr(y_out), _stream(stream)), ctx)


def lfd_backward(ctx, r, v_out, stream=None):
    _check(load().lfd_backward(ctx, _ptr(r), _ptr(v_out), _stream(stream)), ctx)


def lfd_rl_iterate(ctx, y, v, n: int, stop_at_predicted: bool = False, stream=None):
    """Returns (iters_done, predicted, entropy list, flux list)."""
    done, pred = _I(0), _I(0)
    ent = (_D * n)()
    flux = (_D * n)()
    _check(load().lfd_rl_iterate(ctx, _ptr(y), _ptr(v), n, int(bool(stop_at_predicted)),
                                 ctypes.byref(done), ctypes.byref(pred), ent, flux,
                                 _stream(stream)), ctx)
    return done.value, pred.value, list(ent), list(flux)


def lfd_rl_load(ctx, v, stream=None):
    """Puts the start volume v [Nz][H][W] into the context as its resident iterate."""
    _check(load().lfd_rl_load(ctx, _ptr(v), _stream(stream)), ctx)


def lfd_rl_step(ctx, y, n: int = 1, stream=None):
    """n RL iterations of the resident iterate with image y; returns
    (entropy list, flux list) of those iterations."""
    ent = (_D * n)()
    flux = (_D * n)()
    _check(load().lfd_rl_step(ctx, _ptr(y), n, ent, flux, _stream(stream)), ctx)
    return list(ent), list(flux)


def lfd_rl_store(ctx, v, stream=None):
    """Writes the resident iterate into v [Nz][H][W]."""
    _check(load().lfd_rl_store(ctx, _ptr(v), _stream(stream)), ctx)


def lfd_rl_iterate_batch(ctx, nframes: int, y, v, n: int, stop_at_predicted: bool = False,
                         stream=None):
    """Returns (iters_done[F], predicted[F], entropy[F][n], flux[F][n])."""
    done = (_I * nframes)()
    pred = (_I * nframes)()
    ent = (_D * (nframes * n))()
    flux = (_D * (nframes * n))()
    _check(load().lfd_rl_iterate_batch(ctx, nframes, _ptr(y), _ptr(v), n,
                                       int(bool(stop_at_predicted)), done, pred, ent, flux,
                                       _stream(stream)), ctx)
    e = list(ent)
    f = list(flux)
    return (list(done), list(pred), [e[i * n:(i + 1) * n] for i in range(nframes)],
            [f[i * n:(i + 1) * n] for i in range(nframes)])


def lfd_quality(ctx, v, stream=None) -> float:
    e = _D(0)
    _check(load().lfd_quality(ctx, _ptr(v), ctypes.byref(e), _stream(stream)), ctx)
    return e.value


def lfd_quality_mip_static(mip, H: int, W: int, XS: int, YS: int, l2_over_region: int,
                           entropy_out, stream=None):
    """Allocation-free DCT entropy of a device image ``mip`` [H][W]; the result is
    written to ``entropy_out`` (a float64 CUDA tensor of one element, or an address)."""
    for name, x in (("mip", mip), ("entropy_out", entropy_out)):
        if not isinstance(x, int) and not getattr(x, "is_cuda", False):
            raise ValueError("lfd_quality_mip_static: %s must be a CUDA tensor or a device "
                             "address (the call stages nothing)" % name)
    out = entropy_out if isinstance(entropy_out, int) else entropy_out.data_ptr()
    st = load().lfd_quality_mip_static(_ptr(mip), H, W, XS, YS, int(l2_over_region), out,
                                       _stream(stream))
    if st != LFD_OK:
        raise LfdError(st, "lfd_quality_mip_static: %s" % lfd_status_string(st))


def lfd_quality_mip(ctx, mip, stream=None) -> float:
    """DCT entropy of a z-maximum projection image with the context's tables."""
    e = _D(0)
    _check(load().lfd_quality_mip(ctx, _ptr(mip), ctypes.byref(e), _stream(stream)), ctx)
    return e.value


def _dptr(x):
    """Address of a device buffer (CUDA tensor of any dtype, or an int address)."""
    if isinstance(x, int):
        return x
    if getattr(x, "is_cuda", False) and x.is_contiguous():
        return x.data_ptr()
    raise ValueError("expected a contiguous CUDA tensor or a device address")


def lfd_split_load(ctx, v, stream=None):
    _check(load().lfd_split_load(ctx, _ptr(v), _stream(stream)), ctx)


def lfd_split_forward(ctx, hv_part, stream=None):
    _check(load().lfd_split_forward(ctx, _dptr(hv_part), _stream(stream)), ctx)


def lfd_split_update(ctx, y, hv, mip_part, flux_part, stream=None):
    """flux_part: a float64 CUDA tensor of one element (or a device address)."""
    _check(load().lfd_split_update(ctx, _dptr(y), _dptr(hv), _dptr(mip_part), _dptr(flux_part),
                                   _stream(stream)), ctx)


def lfd_split_store(ctx, v, previous: bool = False, stream=None):
    _check(load().lfd_split_store(ctx, _ptr(v), int(bool(previous)), _stream(stream)), ctx)


def lfd_autotune(psf, P: int, Nnum: int, Nz: int, H: int, W: int, opt: lfd_options, stream=None):
    """Returns (best FFT size, measured ms per batched iteration)."""
    best = _I(0)
    ms = ctypes.c_float(0)
    st = load().lfd_autotune(_ptr(psf), P, Nnum, Nz, H, W, ctypes.byref(opt), _stream(stream),
                             ctypes.byref(best), ctypes.byref(ms))
    if st != LFD_OK:
        raise LfdError(st, "lfd_autotune failed: %s" % lfd_status_string(st))
    return best.value, ms.value


def lfd_autotune_options(psf, P: int, Nnum: int, Nz: int, H: int, W: int, opt: lfd_options, stream=None):
    """Tunes opt.fft_size and opt.contraction_cols in place; returns
    (ms per batched iteration of the winner, whether it came from the cache)."""
    ms = ctypes.c_float(0)
    cached = _I(0)
    st = load().lfd_autotune_options(_ptr(psf), P, Nnum, Nz, H, W, ctypes.byref(opt), _stream(stream),
                                     ctypes.byref(ms), ctypes.byref(cached))
    if st != LFD_OK:
        raise LfdError(st, "lfd_autotune_options failed: %s" % lfd_status_string(st))
    return ms.value, bool(cached.value)


def lfd_destroy(ctx):
    if ctx:
        load().lfd_destroy(ctx)


def lfd_last_error(ctx) -> str:
    return load().lfd_last_error(ctx).decode()


def lfd_status_string(s: int) -> str:
    return load().lfd_status_string(s).decode()


def lfd_region_size(Nnum, H, W, dML_um=150.0, Q=40.0, NA=0.95, lambda_um=0.525):
    xs, ys = _I(0), _I(0)
    _check(load().lfd_region_size(Nnum, H, W, dML_um, Q, NA, lambda_um, ctypes.byref(xs),
                                  ctypes.byref(ys)))
    return xs.value, ys.value


def lfd_predict_stop(E) -> int:
    arr = (_D * len(E))(*E)
    return load().lfd_predict_stop(arr, len(E))


def lfd_get_geometry(ctx) -> dict:
    xs, ys, taps, prec = _I(0), _I(0), _I(0), _I(0)
    nbytes = ctypes.c_int64(0)
    _check(load().lfd_get_geometry(ctx, ctypes.byref(xs), ctypes.byref(ys), ctypes.byref(taps),
                                   ctypes.byref(prec), ctypes.byref(nbytes)), ctx)
    return {"XS": xs.value, "YS": ys.value, "taps": taps.value, "precision": prec.value,
            "device_bytes": nbytes.value}


def lfd_get_fft_plan(ctx) -> dict:
    F, B, nt, bins = _I(0), _I(0), _I(0), _I(0)
    _check(load().lfd_get_fft_plan(ctx, ctypes.byref(F), ctypes.byref(B), ctypes.byref(nt),
                                   ctypes.byref(bins)), ctx)
    return {"F": F.value, "B": B.value, "tiles": nt.value, "bins": bins.value}


def lfd_get_exact_plan(ctx) -> dict:
    v = [ctypes.c_int64(0) for _ in range(4)]
    _check(load().lfd_get_exact_plan(ctx, *[ctypes.byref(x) for x in v]), ctx)
    return dict(zip(("n_low", "in_runs", "runs", "single"), (x.value for x in v)))


def lfd_get_spectra(ctx) -> dict:
    v = [ctypes.c_int64(0) for _ in range(3)]
    _check(load().lfd_get_spectra(ctx, *[ctypes.byref(x) for x in v]), ctx)
    return dict(zip(("bytes", "lo_tiles_kept", "lo_tiles"), (x.value for x in v)))


def lfd_debug_fail_allocs(n: int):
    load().lfd_debug_fail_allocs(n)


def lfd_selftest_bounded_wait(limit_ns: int):
    """(status, error word) of the bounded-wait self-test kernel."""
    code = _I(0)
    st = load().lfd_selftest_bounded_wait(limit_ns, ctypes.byref(code))
    return st, code.value


def lfd_launch_count() -> int:
    return int(load().lfd_launch_count())


def lfd_set_profiling(ctx, on: bool = True):
    _check(load().lfd_set_profiling(ctx, int(bool(on))), ctx)


def lfd_stage_times(ctx):
    """Mean stage times (ms): forward, ratio, backward, update, metric, forward
    contraction, backward contraction, FFT transforms, volume R2C, volume C2R,
    exact low-sensitivity backprojection."""
    arr = (ctypes.c_float * 11)()
    _check(load().lfd_stage_times(ctx, arr, 11), ctx)
    return list(arr)


# --------------------------------------------------------------- serving --
def _check_srv(status: int, srv):
    if status != LFD_OK:
        lib = load()
        msg = lib.lfd_server_last_error(srv).decode() if srv else ""
        raise LfdError(status, "%s: %s" % (lib.lfd_status_string(status).decode(), msg))


def lfd_server_default_options(precision: str = "bf16x3", **kw) -> lfd_server_options:
    """Server options; ``opt_*`` keywords go to the embedded lfd_options
    (e.g. opt_fft_size=32), the others to the server fields."""
    o = lfd_server_options()
    load().lfd_server_default_options(ctypes.byref(o))
    o.opt.precision = PRECISIONS[precision]
    for k, v in kw.items():
        if k.startswith("opt_"):
            setattr(o.opt, k[4:], v)
        else:
            setattr(o, k, v)
    return o


def lfd_server_create(opt: lfd_server_options | None = None):
    srv = _VP()
    _check(load().lfd_server_create(ctypes.byref(opt) if opt is not None else None, ctypes.byref(srv)))
    return srv


def lfd_server_add_psf(srv, psf, P: int, nnum: int, nz: int, max_H: int, max_W: int) -> int:
    sid = _I(0)
    _check_srv(load().lfd_server_add_psf(srv, _ptr(psf), P, nnum, nz, max_H, max_W, ctypes.byref(sid)), srv)
    return sid.value


class Request:
    """A submitted request; keeps its buffers alive until it is polled."""

    def __init__(self, ticket, y, v_out, hist):
        self.ticket, self.y, self.v_out, self.hist = ticket, y, v_out, hist


def lfd_submit(srv, set_id: int, y, v_out, max_iter: int = 0, stop_at_predicted: bool = True,
               entropy_hist: bool = True) -> Request:
    """Queues y ([H][W]) for reconstruction into v_out ([Nz][H][W]); returns a
    Request whose ``hist`` holds the entropy history once it is polled."""
    shape = tuple(y.shape)
    r = lfd_request()
    r.set_id, r.H, r.W = set_id, shape[-2], shape[-1]
    r.y, r.v_out = _ptr(y), _ptr(v_out)
    r.max_iter = max_iter
    r.stop_at_predicted = int(bool(stop_at_predicted))
    hist = None
    if entropy_hist:
        n = max_iter if max_iter > 0 else 64
        hist = (ctypes.c_double * n)()
        if max_iter <= 0:
            raise ValueError("entropy_hist needs an explicit max_iter")
        r.entropy_hist = hist
    t = ctypes.c_uint64(0)
    _check_srv(load().lfd_submit(srv, ctypes.byref(r), ctypes.byref(t)), srv)
    return Request(t.value, y, v_out, hist)


def lfd_poll(srv, req, timeout_us: int = -1):
    """None if not finished within the timeout, else a dict of the result."""
    res = lfd_result()
    ticket = req.ticket if isinstance(req, Request) else int(req)
    st = load().lfd_poll(srv, ticket, timeout_us, ctypes.byref(res))
    if st in (LFD_ENOTREADY, LFD_ETIMEDOUT):
        return None
    _check_srv(st, srv)
    out = {"status": res.status, "iters_done": res.iters_done, "iters_run": res.iters_run,
           "predicted": res.predicted, "queue_us": res.queue_us, "latency_us": res.latency_us}
    if isinstance(req, Request) and req.hist is not None:
        out["entropy"] = list(req.hist)
    return out


def lfd_cancel(srv, req) -> int:
    ticket = req.ticket if isinstance(req, Request) else int(req)
    return load().lfd_cancel(srv, ticket)


def lfd_server_stats_get(srv) -> dict:
    st = lfd_server_stats()
    _check_srv(load().lfd_server_stats_get(srv, ctypes.byref(st)), srv)
    return {n: getattr(st, n) for n, _ in lfd_server_stats._fields_}


def lfd_server_last_error(srv) -> str:
    return load().lfd_server_last_error(srv).decode()


def lfd_server_destroy(srv):
    load().lfd_server_destroy(srv)
