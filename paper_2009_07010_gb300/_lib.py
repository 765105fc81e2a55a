"""ctypes view of the C ABI declared in include/psf.h (marshalling only).

The shared library must have been built (``paper_2009_07010_gb300.build``); loading
fails loudly otherwise.  There is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

PSF_OK, PSF_EINVAL, PSF_ENOMEM, PSF_ECUDA, PSF_EUNSUPPORTED, PSF_ETIMEOUT = 0, -1, -2, -3, -4, -5
PSF_FP32, PSF_TC_FP16, PSF_TC_BF16, PSF_TC_FP16X3, PSF_TC_BF16X3 = 0, 1, 3, 2, 4
PSF_WTERM, PSF_IMG_LITERAL_THETA, PSF_DETERMINISTIC, PSF_COMPLEX_OUT = 1, 2, 4, 8
PSF_CLEAN_FACET_PSF = 1
PSF_ALGO_AUTO, PSF_ALGO_CUTOUT = 0, 1
EXACT, UV, IMG, IMG_GRID = 0, 1, 2, 3

# every function include/psf.h declares
EXPORTS = ["psf_plan", "psf_plan_set_opts", "psf_plan_set_windows", "psf_plan_set_weights", "psf_plan_nvis", "psf_exact", "psf_approx_uv", "psf_approx_img",
           "psf_approx_uv_img", "psf_approx_img_grid", "psf_img_grid_table", "psf_clean", "psf_fwhm", "psf_adjoint", "psf_sync_status", "psf_profile_enable", "psf_profile_read", "psf_plan_destroy",
           "psf_strerror", "psf_selftest_umma", "psf_selftest_timeout", "psf_exact_noalloc",
           "psf_selftest_fma_rate"]


class CleanT(ctypes.Structure):
    _fields_ = [("nl", ctypes.c_int32), ("nm", ctypes.c_int32), ("cell_rad", ctypes.c_double),
                ("l_c", ctypes.c_double), ("m_c", ctypes.c_double), ("psf_npix", ctypes.c_int32), ("method", ctypes.c_int32), ("gain", ctypes.c_float),
                ("threshold", ctypes.c_float), ("max_iter", ctypes.c_int32), ("options", ctypes.c_int32)]


class PsfError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        msg = lib().psf_strerror(status).decode() if _LIB is not None else str(status)
        super().__init__(f"{what}: {msg} ({status})" if what else f"{msg} ({status})")


class ObsT(ctypes.Structure):
    _fields_ = [("nbl", ctypes.c_int32), ("ntime", ctypes.c_int32), ("nchan", ctypes.c_int32),
                ("uvw_m", ctypes.c_void_p), ("time_s", ctypes.c_void_p), ("freq_hz", ctypes.c_void_p),
                ("chan_width_hz", ctypes.c_void_p), ("tavg", ctypes.c_void_p), ("favg", ctypes.c_int32),
                ("weights", ctypes.c_void_p)]


class OptsT(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int32), ("flags", ctypes.c_uint32), ("algo", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class BatchT(ctypes.Structure):
    _fields_ = [("npos", ctypes.c_int32), ("lm", ctypes.c_void_p), ("npix", ctypes.c_void_p),
                ("npix0", ctypes.c_int32), ("cell_rad", ctypes.c_double), ("out_offset", ctypes.c_void_p)]


_LIB = None
_lock = threading.Lock()


def lib_path() -> str:
    return _build.LIB


def lib(auto_build: bool = False):
    """The loaded library; raises if it has not been built."""
    global _LIB
    with _lock:
        if _LIB is None:
            if not os.path.exists(_build.LIB):
                if not auto_build:
                    raise RuntimeError(f"CUDA library not built: {_build.LIB} (run __graft_entry__.build())")
                _build.build()
            L = ctypes.CDLL(_build.LIB)
            P, I = ctypes.c_void_p, ctypes.c_int
            L.psf_plan.argtypes = [ctypes.POINTER(ObsT), ctypes.POINTER(OptsT), ctypes.POINTER(P)]
            L.psf_plan.restype = I
            L.psf_plan_set_opts.argtypes = [P, ctypes.POINTER(OptsT)]
            L.psf_plan_set_opts.restype = I
            L.psf_plan_set_windows.argtypes = [P, P, P]
            L.psf_plan_set_windows.restype = I
            L.psf_plan_set_weights.argtypes = [P, P, P]
            L.psf_plan_set_weights.restype = I
            L.psf_plan_nvis.argtypes = [P]
            L.psf_plan_nvis.restype = ctypes.c_int64
            for name in ("psf_exact", "psf_approx_uv", "psf_approx_img", "psf_approx_img_grid"):
                f = getattr(L, name)
                f.argtypes = [P, ctypes.POINTER(BatchT), P, P]
                f.restype = I
            L.psf_clean.argtypes = [P, ctypes.POINTER(CleanT), P, P, P, P, ctypes.POINTER(ctypes.c_int32), P]
            L.psf_clean.restype = I
            L.psf_fwhm.argtypes = [P, ctypes.POINTER(BatchT), P, P, P]
            L.psf_fwhm.restype = I
            L.psf_img_grid_table.argtypes = [P, I, ctypes.c_double, P, P]
            L.psf_img_grid_table.restype = I
            L.psf_approx_uv_img.argtypes = [P, ctypes.POINTER(BatchT), P, P, P]
            L.psf_approx_uv_img.restype = I
            L.psf_adjoint.argtypes = [P, I, ctypes.POINTER(BatchT), P, P, P, P]
            L.psf_adjoint.restype = I
            L.psf_sync_status.argtypes = [P, P]
            L.psf_sync_status.restype = I
            L.psf_profile_enable.argtypes = [P, I]
            L.psf_profile_enable.restype = I
            L.psf_profile_read.argtypes = [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64),
                                           ctypes.POINTER(ctypes.c_int64)]
            L.psf_profile_read.restype = I
            L.psf_plan_destroy.argtypes = [P]
            L.psf_plan_destroy.restype = None
            L.psf_strerror.argtypes = [I]
            L.psf_strerror.restype = ctypes.c_char_p
            L.psf_selftest_timeout.argtypes = [I]
            L.psf_selftest_timeout.restype = I
            L.psf_selftest_fma_rate.argtypes = [I, ctypes.POINTER(ctypes.c_double)]
            L.psf_selftest_fma_rate.restype = I
            L.psf_selftest_umma.argtypes = [P, P, P, I]
            L.psf_selftest_umma.restype = I
            _LIB = L
    return _LIB


def check(status: int, what: str = "") -> None:
    if status != PSF_OK:
        raise PsfError(status, what)
