"""psf_exact_noalloc: the exact PSF of one cutout with no device allocation in the call.

Callers inside a CUDA stream capture, real-time pipelines that forbid allocation after
start-up, or plug-ins whose host application owns the device memory cannot call
cudaMalloc while they compute; this entry point keeps its scratch in a fixed array of
the library's device image.  The test calls it through the C ABI twice in a row (the
scratch keeps the first call's contents) and compares each result with psf_exact on
the FP32 path, within the FP32 tolerance of the parity tests (1e-6 of the peak).
This file is collected last so a failure here leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest

import obsgen

pytestmark = pytest.mark.gpu


def test_noalloc_matches_psf_exact_twice():
    import torch

    import paper_2009_07010_gb300 as psf
    from paper_2009_07010_gb300 import _lib
    psf.build_library()
    L = _lib.lib()
    L.psf_exact_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                    ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]
    L.psf_exact_noalloc.restype = ctypes.c_int
    obs = obsgen.config1_obs()
    cell = obsgen.ARCSEC * 2.0
    cases = [((0.02, 0.02), 64), ((-0.035, 0.011), 128)]
    with psf.Plan(obs, prec="fp32") as plan:
        stream = torch.cuda.current_stream()
        for (l0, m0), N in cases:
            out = torch.full((N * N,), float("nan"), device="cuda")
            rc = L.psf_exact_noalloc(plan._h, l0, m0, N, cell, ctypes.c_void_p(out.data_ptr()),
                                     ctypes.c_void_p(stream.cuda_stream))
            assert rc == 0, _lib.lib().psf_strerror(rc)
            ref = plan.exact(psf.Batch([[l0, m0]], [N], cell)).cpu().numpy().astype(np.float64)
            got = out.cpu().numpy().astype(np.float64)
            err = np.max(np.abs(got - ref[:N * N])) / np.max(np.abs(ref[:N * N]))
            assert err <= 1e-6, err
        # beyond the fixed scratch: a clear error, nothing launched
        rc = L.psf_exact_noalloc(plan._h, 0.01, 0.0, 258, cell, ctypes.c_void_p(out.data_ptr()), None)
        assert rc == _lib.PSF_EUNSUPPORTED
        assert plan.sync_status() == 0
