"""GB300 (sm_103a) library for the averaging-distorted, position-dependent PSF of
Atemkeng et al. (2020): exact bin-averaged PSF cutouts, the uv-plane (Method 1)
and image-plane (Method 2) approximations, and the adjoint, behind the C ABI of
include/psf.h.
"""
from ._lib import (EXACT, IMG, PSF_ALGO_AUTO, PSF_ALGO_CUTOUT, PSF_COMPLEX_OUT, PSF_DETERMINISTIC,  # noqa: F401
                   PSF_EINVAL, PSF_EUNSUPPORTED, PSF_IMG_LITERAL_THETA, PSF_OK, PSF_WTERM, UV,
                   PsfError, lib)
from .api import Batch, Plan, SmearedPSF, fma_rate, selftest_umma, smeared_psf  # noqa: F401
from .build import build as build_library  # noqa: F401
