"""Tensor-core weights with tiny decorrelation arguments.

The FP16/BF16 paths evaluate sinc and the channel Dirichlet kernel with the MUFU sine,
whose error bound is absolute; a visibility whose delay is nearly perpendicular to l0
has a tiny argument, where a ratio of two such sines is meaningless (a sinc anywhere
between 0 and 1, a Dirichlet kernel of 0/0).  On the paper's FWHM setting (20 raw
channels of 50 kHz per output channel, 2 h at 1.4 GHz; here 16 of the 64 antennas) the
exact method produced NaN cutouts before the small-argument series were added.  Sampled
pixels of all three methods against the oracle, FP16 tolerance 1e-4 of the peak."""
import math

import numpy as np
import pytest

import obsgen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def psf():
    import paper_2009_07010_gb300 as m
    m.build_library()
    return m


@pytest.mark.parametrize("cf", ["10x20", "20x40"])
def test_tiny_arguments_fp16(psf, cf):
    obs = obsgen.fig3_obs(cf, every=4)
    N, cell = 64, 2.0 * np.pi / 180 / 3600
    lm = []
    for d, phi in ((0.5, 0.39), (2.0, 2.2), (1.0, -1.0)):
        s = math.sin(math.radians(d))
        lm.append((s * math.cos(phi), s * math.sin(phi)))
    lm = np.array(lm)
    bg = obsgen.Batch(lm, np.full(len(lm), N, np.int32), cell)
    rng = np.random.default_rng(9)
    sel = np.unique(np.concatenate([[p * N * N + N // 2 * N + N // 2 for p in range(len(lm))],
                                    rng.choice(len(lm) * N * N, 60, replace=False)])).astype(np.int64)
    with psf.Plan(obs, prec="tc_fp16") as plan:
        for method, mid in (("exact", oracle.EXACT), ("uv", oracle.UV), ("img", oracle.IMG)):
            got = plan.forward(method, psf.Batch(lm, N, cell)).cpu().numpy().astype(np.float64)
            assert not np.any(np.isnan(got)), method
            ref = oracle.psf(obs, mid, bg, pix_sel=sel)
            for p in range(len(lm)):
                m = (sel >= p * N * N) & (sel < (p + 1) * N * N)
                peak = abs(ref[p * N * N + N // 2 * N + N // 2])
                err = np.max(np.abs(got[sel[m]] - ref[sel[m]])) / peak
                assert err <= 1e-4, (method, p, err)
        assert plan.sync_status() == 0
