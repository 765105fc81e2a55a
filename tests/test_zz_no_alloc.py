"""psf_exact_noalloc: the exact PSF of one cutout with no device allocation in the call.

Real-time pipelines that forbid allocation once they have started, and plug-ins whose
host application owns the device memory, cannot call cudaMalloc while they compute;
this entry point keeps its scratch in a fixed array of the library's device image.

The tests call it through the C ABI twice in a row (the scratch keeps the first call's
contents) and compare each result with psf_exact on the FP32 path, and compare it with
the FP64 oracle directly: the workload-1 cutout in full, a ragged size (66: a partial
64-pixel edge tile), the largest size the scratch holds (256, sampled pixels) and the
MeerKAT-shaped 128 x 128 cutout (58 M visibilities, sampled pixels), all within the
FP32 tolerance of the parity tests (1e-6 of the peak).  This file is collected last so
that a failure here leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest

import obsgen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import paper_2009_07010_gb300 as psf
    from paper_2009_07010_gb300 import _lib
    psf.build_library()
    L = _lib.lib()
    L.psf_exact_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                    ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]
    L.psf_exact_noalloc.restype = ctypes.c_int
    return psf, _lib, L


def _noalloc(L, _lib, plan, l0, m0, N, cell):
    import torch
    out = torch.full((N * N,), float("nan"), device="cuda")
    rc = L.psf_exact_noalloc(plan._h, l0, m0, N, cell, ctypes.c_void_p(out.data_ptr()),
                             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, _lib.lib().psf_strerror(rc)
    return out.cpu().numpy().astype(np.float64)


def _err(got, ref):
    return np.max(np.abs(got - ref)) / np.max(np.abs(ref))


def test_noalloc_matches_psf_exact_twice(lib):
    psf, _lib, L = lib
    obs = obsgen.config1_obs()
    cell = obsgen.ARCSEC * 2.0
    cases = [((0.02, 0.02), 64), ((-0.035, 0.011), 128)]
    with psf.Plan(obs, prec="fp32") as plan:
        for (l0, m0), N in cases:
            got = _noalloc(L, _lib, plan, l0, m0, N, cell)
            ref = plan.exact(psf.Batch([[l0, m0]], [N], cell)).cpu().numpy().astype(np.float64)
            assert _err(got, ref[:N * N]) <= 1e-6
        # beyond the fixed scratch: a clear error, nothing launched
        rc = L.psf_exact_noalloc(plan._h, 0.01, 0.0, 258, cell, None, None)
        assert rc == _lib.PSF_EINVAL   # NULL output is checked first
        import torch
        out = torch.zeros(4, device="cuda")
        rc = L.psf_exact_noalloc(plan._h, 0.01, 0.0, 258, cell, ctypes.c_void_p(out.data_ptr()), None)
        assert rc == _lib.PSF_EUNSUPPORTED
        assert plan.sync_status() == 0


def test_noalloc_against_oracle(lib):
    """The workload-1 cutout in full, a ragged 66 x 66 cutout in full and a 256 x 256
    one on sampled pixels, against the FP64 oracle."""
    psf, _lib, L = lib
    obs = obsgen.config1_obs()
    cell = obsgen.ARCSEC * 2.0
    with psf.Plan(obs, prec="fp32") as plan:
        for (l0, m0), N, sel in (((0.02, 0.02), 64, None), ((0.013, -0.027), 66, None),
                                 ((-0.031, 0.006), 256, np.array([128 * 256 + 128, 0, 255, 256 * 255, 65535,
                                                                  128 * 256, 128 * 256 + 255, 77, 40000, 12345]))):
            got = _noalloc(L, _lib, plan, l0, m0, N, cell)
            batch = obsgen.Batch(np.array([[l0, m0]]), np.array([N], np.int32), cell)
            ref = oracle.psf(obs, oracle.EXACT, batch, pix_sel=sel)
            if sel is not None:
                got, ref = got[sel], ref[sel]
            assert _err(got, ref) <= 1e-6, (N, _err(got, ref))
        assert plan.sync_status() == 0


def test_noalloc_meerkat_cutout(lib):
    """The MeerKAT-shaped 128 x 128 cutout (58 060 800 visibilities) on sampled pixels."""
    psf, _lib, L = lib
    obs = obsgen.config2_obs()
    batch = obsgen.config2_batch()
    N = int(batch.npix[0])
    sel = np.array([64 * N + 64, 0, N - 1, N * N - 1, 64 * N + 65, 67 * N + 62, 31 * N + 100, 100 * N + 3], np.int64)
    with psf.Plan(obs, prec="fp32") as plan:
        got = _noalloc(L, _lib, plan, float(batch.lm[0, 0]), float(batch.lm[0, 1]), N, batch.cell_rad)
        assert plan.sync_status() == 0
    ref = oracle.psf(obs, oracle.EXACT, batch, pix_sel=sel)
    assert _err(got[sel], ref[sel]) <= 1e-6, _err(got[sel], ref[sel])


def test_noalloc_leaves_device_memory_untouched(lib):
    """After a first call (which looks up the scratch array), further calls change the
    device's free memory by nothing: no allocation by the library, the CUDA runtime or
    the driver on its behalf (an allocation is granular to at least 2 MB, so the free
    byte count would move).  The output buffer is allocated before the measurement."""
    import torch
    psf, _lib, L = lib
    obs = obsgen.config1_obs()
    cell = obsgen.ARCSEC * 2.0
    N = 128
    with psf.Plan(obs, prec="fp32") as plan:
        out = torch.empty(N * N, device="cuda")
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        assert L.psf_exact_noalloc(plan._h, 0.01, -0.02, N, cell, ctypes.c_void_p(out.data_ptr()), stream) == 0
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        for i in range(5):
            l0 = 0.005 * (i + 1)
            assert L.psf_exact_noalloc(plan._h, l0, -l0, N, cell, ctypes.c_void_p(out.data_ptr()), stream) == 0
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0, (free0, free1)
        assert plan.sync_status() == 0
