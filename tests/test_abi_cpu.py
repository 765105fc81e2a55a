"""The C-ABI library builds for sm_103a, loads without a GPU, exports every function
include/psf.h declares, and rejects bad arguments on the host before any CUDA call."""
import ctypes
import os
import re

import numpy as np
import pytest

import obsgen
from paper_2009_07010_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return _lib.lib()


def _declared():
    src = open(os.path.join(ROOT, "include", "psf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(psf_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(L):
    names = _declared()
    assert set(names) == set(_lib.EXPORTS)
    for n in names:
        assert hasattr(L, n), n


def test_strerror(L):
    for code in [0, -1, -2, -3, -4, -5]:
        assert L.psf_strerror(code)
    assert L.psf_strerror(0) == b"ok"
    assert L.psf_strerror(-5) == b"device-side wait timed out"
    assert L.psf_strerror(12345) == b"unknown status"


def test_null_handles(L):
    assert L.psf_plan_nvis(None) == -1
    L.psf_plan_destroy(None)
    b = _lib.BatchT(0, None, None, 0, 1e-5, None)
    for fn in (L.psf_exact, L.psf_approx_uv, L.psf_approx_img, L.psf_approx_img_grid):
        assert fn(None, ctypes.byref(b), None, None) == _lib.PSF_EINVAL
    assert L.psf_img_grid_table(None, 64, 1e-5, None, None) == _lib.PSF_EINVAL
    cfg = _lib.CleanT(64, 64, 1e-5, 0.0, 0.0, 16, 3, 0.1, 0.0, 10, 0)
    assert L.psf_clean(None, ctypes.byref(cfg), None, None, None, None, None, None) == _lib.PSF_EINVAL
    assert ctypes.sizeof(_lib.CleanT) == 56
    assert L.psf_fwhm(None, ctypes.byref(b), None, None, None) == _lib.PSF_EINVAL
    assert L.psf_plan_set_windows(None, None, None) == _lib.PSF_EINVAL
    assert L.psf_approx_uv_img(None, ctypes.byref(b), None, None, None) == _lib.PSF_EINVAL
    assert L.psf_adjoint(None, 0, ctypes.byref(b), None, None, None, None) == _lib.PSF_EINVAL
    assert L.psf_sync_status(None, None) == _lib.PSF_EINVAL
    assert L.psf_plan(None, None, None) == _lib.PSF_EINVAL


def _obs_struct(o, keep):
    arrs = [np.ascontiguousarray(o.uvw_m), np.ascontiguousarray(o.time_s), np.ascontiguousarray(o.freq_hz),
            np.ascontiguousarray(o.chan_width_hz), np.ascontiguousarray(o.tavg, np.int32)]
    keep.extend(arrs)
    return _lib.ObsT(o.uvw_m.shape[0], o.uvw_m.shape[1], o.freq_hz.shape[0], *[a.ctypes.data for a in arrs[:4]],
                     arrs[4].ctypes.data, int(o.favg), None)


@pytest.mark.parametrize("mutate", ["favg_not_divisor", "zero_tavg", "neg_width", "uneven_time",
                                    "bad_prec", "bad_flags", "no_bins"])
def test_plan_rejects_bad_observations_on_host(L, mutate):
    o = obsgen.tiny_obs()
    opts = _lib.OptsT(0, 0, 0, 0)
    if mutate == "favg_not_divisor":
        o.favg = 3
    elif mutate == "zero_tavg":
        o.tavg[1] = 0
    elif mutate == "neg_width":
        o.chan_width_hz = -o.chan_width_hz
    elif mutate == "uneven_time":
        o.time_s = o.time_s.copy()
        o.time_s[5] += 0.3
    elif mutate == "bad_prec":
        opts = _lib.OptsT(7, 0, 0, 0)
    elif mutate == "bad_flags":
        opts = _lib.OptsT(0, 1 << 10, 0, 0)
    elif mutate == "no_bins":
        o.tavg[:] = o.ntime + 1
    keep = []
    s = _obs_struct(o, keep)
    h = ctypes.c_void_p()
    assert L.psf_plan(ctypes.byref(s), ctypes.byref(opts), ctypes.byref(h)) == _lib.PSF_EINVAL
    assert not h.value


def test_plan_without_device_reports_cuda_error(L):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    o = obsgen.tiny_obs()
    keep = []
    s = _obs_struct(o, keep)
    h = ctypes.c_void_p()
    assert L.psf_plan(ctypes.byref(s), None, ctypes.byref(h)) == _lib.PSF_ECUDA
    assert not h.value


def test_header_constants_match_binding():
    src = open(os.path.join(ROOT, "include", "psf.h")).read()
    consts = dict(re.findall(r"#define\s+(PSF_[A-Z0-9_]+)\s+(-?\d+)u?", src))
    assert int(consts["PSF_OK"]) == _lib.PSF_OK
    assert int(consts["PSF_ETIMEOUT"]) == _lib.PSF_ETIMEOUT
    assert int(consts["PSF_TC_BF16"]) == _lib.PSF_TC_BF16
    assert int(consts["PSF_WTERM"]) == _lib.PSF_WTERM
    assert int(consts["PSF_IMG_LITERAL_THETA"]) == _lib.PSF_IMG_LITERAL_THETA
    assert int(consts["PSF_DETERMINISTIC"]) == _lib.PSF_DETERMINISTIC
    assert int(consts["PSF_COMPLEX_OUT"]) == _lib.PSF_COMPLEX_OUT
