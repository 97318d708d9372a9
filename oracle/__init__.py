"""FP64 CPU oracle for light-field Richardson-Lucy deconvolution.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this package. The
product library (``paper_2208_11422_gb300``) never imports, links or calls it,
and the two share no code: this package reads only its own C file
(``lfd_oracle.c``) and numpy.

Contents
  * ``forward`` / ``backward`` (+ ``*_at`` sampled variants, ``forward_crop``
    and ``backward_block`` for dense blocks): the light-field projection H and
    its transpose, direct FP64 summation (lfd_oracle.c).
  * ``metric``: z-MIP, orthonormal 2-D DCT (Eqs. 1-4), region size (Eqs. 6-11),
    DCT entropy (Eqs. 5 and 12), stopping rule (Section 2.2).
  * ``rl``: the Richardson-Lucy iteration built from the pieces above.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against brute force, closed forms or library routines; none is "parity
unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lfd_oracle.c")
_LIB = os.path.join(_HERE, "liblfd_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile lfd_oracle.c into liblfd_oracle.so beside it (gcc, -O3, no FMA
    contraction so x86 and Arm produce identical bits)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(
            ["gcc", "-O3", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
             "-pthread", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            i = ctypes.c_int
            for name in ("orc_forward", "orc_backward"):
                f = getattr(lib, name)
                f.argtypes = [dp, i, i, i, i, i, dp, dp, i]
                f.restype = None
            for name in ("orc_forward_at", "orc_backward_at"):
                f = getattr(lib, name)
                f.argtypes = [dp, i, i, i, i, i, dp, ctypes.c_long, ip, dp, i]
                f.restype = None
            lib.orc_backward_block.argtypes = [dp, i, i, i, i, i, dp, i, i, i, i, i, i, dp, i]
            lib.orc_backward_block.restype = None
            lib.orc_macs.argtypes = [i, i, i, i]
            lib.orc_macs.restype = ctypes.c_double
            _lib = lib
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def _geom(psf: np.ndarray, nnum: int):
    Nz, N1, N2, P, P2 = psf.shape
    if N1 != nnum or N2 != nnum or P != P2 or P % 2 == 0:
        raise ValueError("psf must be [Nz][Nnum][Nnum][P][P] with P odd")
    return Nz, P


def forward(psf, nnum: int, v, nthreads: int | None = None) -> np.ndarray:
    """Hv for a volume v[Nz][H][W]; returns the FP64 sensor image [H][W]."""
    psf = _f64(psf)
    v = _f64(v)
    Nz, P = _geom(psf, nnum)
    if v.ndim != 3 or v.shape[0] != Nz:
        raise ValueError("v must be [Nz][H][W]")
    H, W = v.shape[1:]
    out = np.zeros((H, W), np.float64)
    _load().orc_forward(_dptr(psf), P, nnum, Nz, H, W, _dptr(v), _dptr(out),
                        nthreads or default_threads())
    return out


def backward(psf, nnum: int, r, nthreads: int | None = None) -> np.ndarray:
    """H^T r for a sensor image r[H][W]; returns the FP64 volume [Nz][H][W]."""
    psf = _f64(psf)
    r = _f64(r)
    Nz, P = _geom(psf, nnum)
    H, W = r.shape
    out = np.zeros((Nz, H, W), np.float64)
    _load().orc_backward(_dptr(psf), P, nnum, Nz, H, W, _dptr(r), _dptr(out),
                         nthreads or default_threads())
    return out


def forward_at(psf, nnum: int, v, pix, nthreads: int | None = None) -> np.ndarray:
    """Hv at the pixels pix[q] = (i, j) only."""
    psf = _f64(psf)
    v = _f64(v)
    Nz, P = _geom(psf, nnum)
    H, W = v.shape[1:]
    pix = np.ascontiguousarray(pix, dtype=np.int32).reshape(-1, 2)
    out = np.zeros(len(pix), np.float64)
    _load().orc_forward_at(_dptr(psf), P, nnum, Nz, H, W, _dptr(v), len(pix),
                           pix.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                           _dptr(out), nthreads or default_threads())
    return out


def backward_at(psf, nnum: int, r, vox, nthreads: int | None = None) -> np.ndarray:
    """H^T r at the voxels vox[q] = (z, i', j') only."""
    psf = _f64(psf)
    r = _f64(r)
    Nz, P = _geom(psf, nnum)
    H, W = r.shape
    vox = np.ascontiguousarray(vox, dtype=np.int32).reshape(-1, 3)
    out = np.zeros(len(vox), np.float64)
    _load().orc_backward_at(_dptr(psf), P, nnum, Nz, H, W, _dptr(r), len(vox),
                            vox.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                            _dptr(out), nthreads or default_threads())
    return out


def backward_block(psf, nnum: int, r, z0: int, z1: int, i0: int, i1: int, j0: int, j1: int,
                   nthreads: int | None = None) -> np.ndarray:
    """H^T r at every voxel of the block [z0, z1) x [i0, i1) x [j0, j1), as an
    array [z1-z0][i1-i0][j1-j0]; the same sums as ``backward_at`` (bit for bit),
    several neighbouring voxels computed side by side."""
    psf = _f64(psf)
    r = _f64(r)
    Nz, P = _geom(psf, nnum)
    H, W = r.shape
    if not (0 <= z0 < z1 <= Nz and 0 <= i0 < i1 <= H and 0 <= j0 < j1 <= W):
        raise ValueError("block outside the volume")
    out = np.zeros((z1 - z0, i1 - i0, j1 - j0), np.float64)
    _load().orc_backward_block(_dptr(psf), P, nnum, Nz, H, W, _dptr(r), z0, z1, i0, i1, j0, j1,
                               _dptr(out), nthreads or default_threads())
    return out


def forward_crop(psf, nnum: int, v, i0: int, i1: int, j0: int, j1: int,
                 nthreads: int | None = None) -> np.ndarray:
    """Hv on the pixels [i0, i1) x [j0, j1) of the sensor, by ``forward`` over
    a window of the volume. A pixel (i, j) sums the voxels with |i - i'| <= c
    and |j - j'| <= c (c = (P-1)/2) only, so the window is the crop widened by
    c on every side (inside the sensor), with its origin moved down to a
    multiple of Nnum so that every voxel keeps its lenslet phase (i' mod Nnum,
    j' mod Nnum). Inside the crop the window's forward adds the same terms in
    the same order as the full frame's: the values are equal bit for bit."""
    psf = _f64(psf)
    Nz, P = _geom(psf, nnum)
    H, W = v.shape[1:]
    if not (0 <= i0 < i1 <= H and 0 <= j0 < j1 <= W):
        raise ValueError("crop outside the sensor")
    c = (P - 1) // 2
    wy0 = max(0, i0 - c) // nnum * nnum
    wx0 = max(0, j0 - c) // nnum * nnum
    wy1, wx1 = min(H, i1 + c), min(W, j1 + c)
    win = forward(psf, nnum, np.asarray(v)[:, wy0:wy1, wx0:wx1], nthreads)
    return win[i0 - wy0:i1 - wy0, j0 - wx0:j1 - wx0]


def macs_per_projection(P: int, Nz: int, H: int, W: int) -> float:
    """Multiply-adds of one projection with zero-padded taps excluded."""
    return _load().orc_macs(P, Nz, H, W)
