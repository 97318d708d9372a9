"""C-ABI checks that need no GPU: the library loads, exports every function
that include/lfd.h declares, validates shapes before touching CUDA, and its
host-only helpers agree with the oracle."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import metric
from paper_2208_11422_gb300 import lfd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2208_11422_gb300 import build
    build.build()
    return lfd.load()


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(lfd_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "lfd_create" in names and "lfd_rl_iterate" in names
    for n in names:
        assert hasattr(lib, n), n
    # and the binding covers the same set
    assert set(names) <= set(lfd.exported_names())


@pytest.mark.parametrize("args", [
    (25, 4, 5, 75, 75),    # even Nnum
    (24, 5, 5, 75, 75),    # even P
    (27, 5, 5, 75, 75),    # P not a multiple of Nnum
    (25, 5, 0, 75, 75),    # no depths
    (25, 5, 5, 74, 75),    # H not a multiple of Nnum
    (25, 5, 5, 75, 0),     # empty sensor
    (25, 5, 5, -5, 75),
])
def test_create_rejects_bad_shapes_before_any_cuda_call(lib, args):
    P, N, Nz, H, W = args
    psf = np.zeros(16, np.float32)
    out = ctypes.c_void_p(123)
    st = lib.lfd_create(psf.ctypes.data, P, N, Nz, H, W, None, None, ctypes.byref(out))
    assert st == lfd.LFD_EINVAL
    assert out.value is None


def test_create_rejects_null_psf_and_bad_options(lib):
    out = ctypes.c_void_p()
    assert lib.lfd_create(None, 25, 5, 5, 75, 75, None, None, ctypes.byref(out)) == lfd.LFD_EINVAL
    psf = np.zeros(16, np.float32)
    o = lfd.lfd_default_options()
    o.precision = 9
    assert lib.lfd_create(psf.ctypes.data, 25, 5, 5, 75, 75, ctypes.byref(o), None,
                          ctypes.byref(out)) == lfd.LFD_EINVAL
    o = lfd.lfd_default_options(XS=100, YS=4)   # region wider than the image
    assert lib.lfd_create(psf.ctypes.data, 25, 5, 5, 75, 75, ctypes.byref(o), None,
                          ctypes.byref(out)) == lfd.LFD_EINVAL
    assert lib.lfd_create(psf.ctypes.data, 25, 5, 5, 75, 75, None, None, None) == lfd.LFD_EINVAL
    o = lfd.lfd_default_options(variant="fft", contraction_cols=48)   # 16, 32 or 64
    assert lib.lfd_create(psf.ctypes.data, 25, 5, 5, 75, 75, ctypes.byref(o), None,
                          ctypes.byref(out)) == lfd.LFD_EINVAL
    o = lfd.lfd_default_options(precision="tf32", variant="fft")   # TF32 is a direct-GEMM mode
    assert lib.lfd_create(psf.ctypes.data, 25, 5, 5, 75, 75, ctypes.byref(o), None,
                          ctypes.byref(out)) == lfd.LFD_EUNSUPPORTED
    assert out.value is None


def test_null_context_calls(lib):
    assert lib.lfd_rl_load(None, None, None) == lfd.LFD_EINVAL
    assert lib.lfd_rl_step(None, None, 1, None, None, None) == lfd.LFD_EINVAL
    assert lib.lfd_rl_store(None, None, None) == lfd.LFD_EINVAL
    assert lib.lfd_forward(None, None, None, None) == lfd.LFD_EINVAL
    assert lib.lfd_backward(None, None, None, None) == lfd.LFD_EINVAL
    assert lib.lfd_rl_iterate(None, None, None, 1, 0, None, None, None, None, None) == lfd.LFD_EINVAL
    assert lib.lfd_get_exact_plan(None, None, None, None, None) == lfd.LFD_EINVAL
    lib.lfd_destroy(None)
    assert lfd.lfd_status_string(lfd.LFD_EINVAL) == "LFD_EINVAL"


def test_defaults():
    o = lfd.lfd_default_options()
    assert o.precision == lfd.LFD_FP32 and abs(o.eps - 1e-6) < 1e-12
    assert (o.dML_um, o.Q, o.NA, o.lambda_um) == (150.0, 40.0, 0.95, 0.525)
    assert o.l2_over_region == 1
    assert o.spectra_lo_tau == 2.0 ** -8


@pytest.mark.parametrize("N,H,W", [(5, 75, 75), (15, 615, 615), (15, 2025, 2025),
                                   (15, 615, 2025), (11, 363, 1331), (13, 13, 13), (1, 7, 3),
                                   (3, 900, 30)])
def test_region_size_matches_oracle(N, H, W):
    assert lfd.lfd_region_size(N, H, W) == metric.region_size(N, H, W)


def test_region_size_rejects_bad_optics(lib):
    xs, ys = ctypes.c_int(), ctypes.c_int()
    assert lib.lfd_region_size(5, 75, 75, 0.0, 40.0, 0.95, 0.5, ctypes.byref(xs), ctypes.byref(ys)) \
        == lfd.LFD_EINVAL


def test_predict_stop_matches_oracle():
    rng = np.random.default_rng(0)
    for trial in range(200):
        n = int(rng.integers(1, 12))
        E = rng.integers(0, 4, n).astype(float).tolist()   # many ties on purpose
        assert lfd.lfd_predict_stop(E) == metric.predicted_iteration(E), E
    assert lfd.lfd_predict_stop([]) == 0


STRUCTS = {
    "lfd_options": ["precision", "eps", "dML_um", "XS", "l2_over_region", "fft_size", "spectra_lo_tau",
                    "contraction_cols"],
    "lfd_server_options": ["opt", "arena_bytes", "max_frames_per_set", "max_iter"],
    "lfd_request": ["set_id", "H", "y", "v_out", "max_iter", "entropy_hist"],
    "lfd_result": ["status", "predicted", "queue_us", "latency_us"],
    "lfd_server_stats": ["submitted", "columns", "resident_bytes", "queued", "in_flight"],
}


def test_binding_structs_match_the_header(tmp_path):
    """sizeof / offsetof of every ABI struct, from a C program compiled against
    include/lfd.h, equal the ctypes layouts."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "lfd.h"', "int main(void) {"]
    for s, fields in STRUCTS.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (s, s))
        for f in fields:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (s, f, s, f))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                 check=True).stdout.splitlines())
    for s, fields in STRUCTS.items():
        cls = getattr(lfd, s)
        assert int(out[s]) == ctypes.sizeof(cls), s
        for f in fields:
            assert int(out["%s.%s" % (s, f)]) == getattr(cls, f).offset, (s, f)


def test_server_rejects_bad_options_before_cuda(lib):
    for kw in ({"max_cols": 8}, {"max_cols": 100}, {"max_frames_per_set": 0}, {"max_iter": 0},
               {"max_queue": 0}, {"opt_fft_size": 48}):
        o = lfd.lfd_server_default_options(**kw)
        srv = ctypes.c_void_p()
        assert lib.lfd_server_create(ctypes.byref(o), ctypes.byref(srv)) == lfd.LFD_EINVAL, kw
        assert not srv.value
    o = lfd.lfd_server_default_options()
    o.opt.precision = lfd.LFD_TF32   # the server runs the FFT variant: split BF16, BF16 or FP32
    srv = ctypes.c_void_p()
    assert lib.lfd_server_create(ctypes.byref(o), ctypes.byref(srv)) == lfd.LFD_EINVAL


def test_server_calls_reject_null_handles(lib):
    r = lfd.lfd_request()
    t = ctypes.c_uint64(0)
    assert lib.lfd_submit(None, ctypes.byref(r), ctypes.byref(t)) == lfd.LFD_EINVAL
    assert lib.lfd_poll(None, 1, 0, None) == lfd.LFD_EINVAL
    assert lib.lfd_cancel(None, 1) == lfd.LFD_EINVAL
    assert lib.lfd_server_add_psf(None, None, 3, 1, 1, 3, 3, None) == lfd.LFD_EINVAL
    lib.lfd_server_destroy(None)


def test_bounded_wait_selftest_rejects_limits_before_cuda(lib):
    code = ctypes.c_int(5)
    assert lib.lfd_selftest_bounded_wait(10, ctypes.byref(code)) == lfd.LFD_EINVAL
    assert lib.lfd_selftest_bounded_wait(5_000_000_000, ctypes.byref(code)) == lfd.LFD_EINVAL
    assert lib.lfd_selftest_bounded_wait(20_000_000, None) == lfd.LFD_EINVAL
    lib.lfd_debug_fail_allocs(0)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_serving_arena_free_list(lib, seed):
    """The serving arena's first-fit free list against a byte-map model."""
    assert lib.lfd_selftest_freelist(seed, 400) == lfd.LFD_OK
    assert lib.lfd_selftest_freelist(seed, 0) == lfd.LFD_EINVAL


@pytest.mark.parametrize("seed,N,Nz,k,L", [(1, 5, 3, 5, 15), (2, 15, 4, 11, 41), (3, 3, 2, 23, 20),
                                           (4, 15, 2, 23, 90), (5, 7, 5, 31, 30)])
def test_exact_runs_plan(lib, seed, N, Nz, k, L):
    """The plan of runs for the exact low-sensitivity sums covers every listed
    voxel once, along lenslet rows / columns of one channel, within limits
    (k = 31 with N = 7 gives PSF rows of 217 taps; k = 23 with N = 15 345)."""
    assert lib.lfd_selftest_exact_runs(seed, N, Nz, k, L) == lfd.LFD_OK


def test_exact_runs_plan_rejects_bad_shapes(lib):
    assert lib.lfd_selftest_exact_runs(1, 4, 2, 5, 10) == lfd.LFD_EINVAL   # even Nnum
    assert lib.lfd_selftest_exact_runs(1, 5, 2, 4, 10) == lfd.LFD_EINVAL   # even k
    assert lib.lfd_selftest_exact_runs(1, 5, 0, 5, 10) == lfd.LFD_EINVAL


@pytest.mark.parametrize("seed,n,grid", [(1, 190080, 152), (2, 1000, 152), (3, 152, 152), (4, 5, 1),
                                         (5, 7000, 300)])
def test_adjoint_balanced_ranges(lib, seed, n, grid):
    assert lib.lfd_selftest_balanced_ranges(seed, n, grid) == lfd.LFD_OK


def test_adjoint_balanced_ranges_rejects_bad_sizes(lib):
    assert lib.lfd_selftest_balanced_ranges(1, 10, 11) == lfd.LFD_EINVAL
    assert lib.lfd_selftest_balanced_ranges(1, 0, 1) == lfd.LFD_EINVAL
