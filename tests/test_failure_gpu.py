"""Failure detection on the GPU without a fault: a bounded device-side wait that
nothing completes gives up after its wall-clock limit, the kernel returns, the host
reads PSF_ETIMEOUT, and the device stays usable for the next computation."""
import numpy as np
import pytest

import obsgen
import oracle

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives():
    import paper_2009_07010_gb300 as psf
    from paper_2009_07010_gb300 import _lib
    psf.build_library()
    L = _lib.lib()
    assert L.psf_selftest_timeout(0) == _lib.PSF_EINVAL
    assert L.psf_selftest_timeout(50) == _lib.PSF_ETIMEOUT
    obs = obsgen.tiny_obs()
    batch = obsgen.Batch(np.array([[0.02, -0.01]]), np.array([8], np.int32), 4e-5)
    with psf.Plan(obs, prec="tc_fp16") as plan:
        got = plan.exact(psf.Batch.from_obsgen(batch)).cpu().numpy().astype(np.float64)
        assert plan.sync_status() == 0
    ref = oracle.psf(obs, oracle.EXACT, batch)
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) <= 2e-3
