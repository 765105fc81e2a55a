"""GPU parity of psf_fwhm (PSF size along the radial and tangential directions, Fig. 3)
against the oracle's definition.

The same synthetic cutouts go to both sides (elliptical Gaussians, a profile whose walk
leaves the cutout, caller offsets with gaps), and each side measures its own PSF
cutouts of workload 1.  The device samples the profile in float32 (positions and
values to ~1e-7 relative), so widths agree to 1e-5 relative; on the PSF cutouts the
two sides' PSFs differ by their own tolerance (1e-6 in FP32), 1e-4 relative."""
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


def _gauss(N, sr, st, phi):
    c = N // 2
    y, x = np.mgrid[0:N, 0:N].astype(np.float64)
    dx, dy = x - c, y - c
    r = dx * math.cos(phi) + dy * math.sin(phi)
    t = -dx * math.sin(phi) + dy * math.cos(phi)
    return np.exp(-0.5 * (r / sr) ** 2 - 0.5 * (t / st) ** 2)


def test_fwhm_synthetic_cutouts(psf):
    import torch
    rng = np.random.default_rng(5)
    sizes = [64, 32, 48, 16, 64, 32]
    lm, cuts = [], []
    for k, N in enumerate(sizes):
        phi = rng.uniform(-math.pi, math.pi)
        lm.append((0.03 * math.cos(phi), 0.03 * math.sin(phi)) if k else (0.0, 0.0))
        cuts.append(_gauss(N, rng.uniform(1.5, N / 8), rng.uniform(1.5, N / 8), phi + rng.normal(0, 0.3)))
    flat = np.zeros(1 + 7 * len(sizes) + sum(n * n for n in sizes))
    offs, run = [], 1
    for c in cuts:
        offs.append(run)
        flat[run:run + c.size] = c.ravel()
        run += c.size + 7
    flat[offs[3]:offs[3] + 256] = np.tile(np.maximum(1.0 - np.abs(np.arange(16) - 8) / 40.0, 0), 16)  # never halves
    cell = 1.7e-6
    b = psf.Batch(np.array(lm), np.array(sizes), cell, out_offset=np.array(offs))
    with psf.Plan(obsgen.tiny_obs(), prec="fp32") as plan:
        got = plan.fwhm(b, torch.tensor(flat, dtype=torch.float32, device="cuda")).cpu().numpy()
        assert plan.sync_status() == 0
    for p, N in enumerate(sizes):
        P = flat[offs[p]:offs[p] + N * N].astype(np.float32).astype(np.float64).reshape(N, N)
        ref = oracle.fwhm(P, lm[p][0], lm[p][1], cell)
        for k in range(2):
            if math.isnan(ref[k]):
                assert math.isnan(got[p, k]), (p, k)
            else:
                assert got[p, k] == pytest.approx(ref[k], rel=1e-5), (p, k)
    assert math.isnan(got[3, 0]) and math.isnan(got[3, 1])


def test_fwhm_of_psf_cutouts(psf):
    """Workload 1's exact PSF at positions out to 0.3 rad: each side measures its own."""
    obs = obsgen.config1_obs()
    lm = np.array([(0.0, 0.0), (0.02, 0.02), (0.1, -0.05), (-0.2, 0.15), (0.05, 0.28)])
    N, cell = 64, 2.0 * np.pi / 180 / 3600
    bg = obsgen.Batch(lm, np.full(len(lm), N, np.int32), cell)
    ref_cut = oracle.psf(obs, oracle.EXACT, bg).reshape(len(lm), N, N)
    with psf.Plan(obs, prec="fp32") as plan:
        b = psf.Batch(lm, N, cell)
        cut = plan.exact(b)
        got = plan.fwhm(b, cut).cpu().numpy()
        assert plan.sync_status() == 0
    for p in range(len(lm)):
        ref = oracle.fwhm(ref_cut[p], lm[p, 0], lm[p, 1], cell)
        np.testing.assert_allclose(got[p], ref, rtol=1e-4)
    assert got[-1, 0] > got[0, 0]          # smearing widens the PSF away from the centre


def test_fwhm_grows_with_distance_and_averaging(psf):
    """The paper's FWHM setting (64 antennas, 1.4 GHz, 2 h, 6 MHz): the radial and
    tangential widths grow with distance, and more with 20 s x 2 MHz averaging than with
    10 s x 1 MHz (properties of the full-size result)."""
    bg = obsgen.fig3_batch(radii_deg=(0.0, 1.5, 3.0, 4.5), nang=4)
    res = {}
    for cf in ("10x20", "20x40"):
        with psf.Plan(obsgen.fig3_obs(cf), prec="tc_fp16") as plan:
            b = psf.Batch.from_obsgen(bg)
            res[cf] = plan.fwhm(b, plan.exact(b)).cpu().numpy()
            assert plan.sync_status() == 0
    r = np.degrees(np.arcsin(np.hypot(bg.lm[:, 0], bg.lm[:, 1])))
    for cf in res:
        w = res[cf]
        assert not np.any(np.isnan(w))
        for k in range(2):
            means = [w[np.abs(r - d) < 1e-6, k].mean() for d in (0.0, 1.5, 3.0, 4.5)]
            assert all(b > a for a, b in zip(means, means[1:])), (cf, k, means)
    far = np.abs(r - 4.5) < 1e-6
    assert res["20x40"][far].mean() > res["10x20"][far].mean()
