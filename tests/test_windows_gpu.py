"""GPU parity of the windowed bin average (Sect. 2.3, Eqs. 15-16) against the FP64
oracle: baseline-dependent windows over each bin's raw samples and each output channel's
raw channels (psf_plan_set_windows), for the exact method and for Methods 1 and 2, whose
two sincs become the window's transforms (complex for asymmetric windows).  Tolerances:
1e-6 (FP32) of the cutout peak everywhere, 1e-4 (FP16 tensor cores) on workload 1 and a
few FP16 unit roundoffs (2e-3) on the 592-visibility observation, 2e-5 for the split
precision mode; the adjoint as its own tests (2e-5 on dL/dW, 2e-4 on dL/dl0)."""
import numpy as np
import pytest

import obsgen
import oracle

pytestmark = pytest.mark.gpu
TOL = {"fp32": 1e-6, "tc_fp16": 1e-4}


@pytest.fixture(scope="module")
def psf():
    import paper_2009_07010_gb300 as m
    m.build_library()
    return m


def _windowed(obs, strength):
    tw, cw = obsgen.bd_windows(obs, strength)
    return obsgen.Observation(obs.uvw_m, obs.time_s, obs.freq_hz, obs.chan_width_hz, obs.tavg, obs.favg,
                              obs.weights, obs.enu_m, tw, cw)


def _cases():
    c1 = _windowed(obsgen.config1_obs(), 1.5)
    b1 = obsgen.Batch(np.array([[0.02, 0.02], [-0.05, 0.03]]), np.array([64, 32], np.int32), 2 * obsgen.ARCSEC)
    t = _windowed(obsgen.tiny_obs(nant=6, ntime=48, nchan=8, tavg=[2, 3, 4, 6, 8, 12, 16, 24, 2, 3, 4, 6, 8, 12, 16],
                                  favg=2, weights=True), 2.0)
    bt = obsgen.Batch(np.array([[0.03, -0.02], [-0.01, 0.045]]), np.array([64, 32], np.int32), 3e-5)
    return [("config1", c1, b1), ("bda_favg2", t, bt)]


def _tol(prec, obs):
    if prec == "tc_fp16" and obs.nvis() < 10000:   # few visibilities: per-term bound
        return 2e-3
    return {"fp32": 1e-6, "tc_fp16": 1e-4, "tc_bf16x3": 2e-5}[prec]


def _asymmetric(obs):
    """The cases' windows with an asymmetric factor on the time taper (complex transforms)."""
    tw = (obs.time_window * (1.0 + 0.4 * np.sin(np.arange(obs.time_window.size)))).astype(np.float32)
    return obsgen.Observation(obs.uvw_m, obs.time_s, obs.freq_hz, obs.chan_width_hz, obs.tavg, obs.favg,
                              obs.weights, obs.enu_m, tw, obs.chan_window)


@pytest.mark.parametrize("prec", ["fp32", "tc_fp16"])
def test_windowed_exact(psf, prec):
    for name, obs, bg in _cases():
        tol = _tol(prec, obs)
        ref = oracle.psf(obs, oracle.EXACT, bg)
        plain = oracle.psf(obsgen.Observation(obs.uvw_m, obs.time_s, obs.freq_hz, obs.chan_width_hz, obs.tavg,
                                              obs.favg, obs.weights), oracle.EXACT, bg)
        with psf.Plan(obs, prec=prec) as plan:
            got = plan.exact(psf.Batch.from_obsgen(bg)).cpu().numpy().astype(np.float64)
            assert plan.sync_status() == 0
        offs = obsgen.concat_pixels(bg)
        for p in range(bg.npos):
            n2 = int(bg.npix[p]) ** 2
            g, r = got[offs[p]:offs[p] + n2], ref[offs[p]:offs[p] + n2]
            err = np.max(np.abs(g - r)) / np.max(np.abs(r))
            assert err <= tol, (name, p, err)
        assert np.max(np.abs(ref - plain)) > 10 * TOL[prec] * np.max(np.abs(ref))   # the windows matter


def test_windowed_batched_and_reset(psf):
    """The batched form (>= 32 positions of one size) with windows, and the boxcar restored
    by psf_plan_set_windows(NULL, NULL) reproducing an unwindowed plan bit for bit."""
    _, obs, _ = _cases()[1]
    rng = np.random.default_rng(4)
    lm = rng.uniform(-0.04, 0.04, (40, 2))
    bg = obsgen.Batch(lm, np.full(40, 32, np.int32), 3e-5)
    sel = np.array([k * 1024 + 16 * 32 + 16 for k in (0, 7, 39)] + list(rng.choice(40 * 1024, 30, replace=False)))
    ref = oracle.psf(obs, oracle.EXACT, bg, pix_sel=sel)
    plain_obs = obsgen.Observation(obs.uvw_m, obs.time_s, obs.freq_hz, obs.chan_width_hz, obs.tavg, obs.favg,
                                   obs.weights)
    with psf.Plan(obs, prec="tc_fp16") as plan:
        b = psf.Batch.from_obsgen(bg)
        got = plan.exact(b).cpu().numpy().astype(np.float64)
        peak = np.max(np.abs(ref[sel]))
        assert np.max(np.abs(got[sel] - ref[sel])) / peak <= TOL["tc_fp16"]
        plan.set_windows(None, None)
        back = plan.exact(b).cpu().numpy()
        assert plan.sync_status() == 0
    with psf.Plan(plain_obs, prec="tc_fp16") as plan2:
        fresh = plan2.exact(psf.Batch.from_obsgen(bg)).cpu().numpy()
    assert np.array_equal(back, fresh)


def test_windowed_adjoint(psf):
    import torch
    _, obs, bg = _cases()[1]
    P = oracle.psf(obs, oracle.EXACT, bg)
    rng = np.random.default_rng(3)
    R = 2 * (P - (P * (1 + 0.01 * rng.standard_normal(P.size)) + 0.05 * np.abs(P).max() * rng.standard_normal(P.size)))
    g_lm_ref, g_W_ref = oracle.vjp(obs, oracle.EXACT, bg, R)
    with psf.Plan(obs, prec="fp32") as plan:
        g_lm, g_W = plan.adjoint("exact", psf.Batch.from_obsgen(bg), torch.tensor(R, dtype=torch.float32, device="cuda"))
        assert plan.sync_status() == 0
    g_lm, g_W = g_lm.cpu().numpy(), g_W.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(g_W - g_W_ref)) / np.max(np.abs(g_W_ref)) <= 2e-5
    assert np.max(np.abs(g_lm - g_lm_ref)) / np.max(np.abs(g_lm_ref)) <= 2e-4


def test_window_validation(psf):
    obs = obsgen.tiny_obs()
    with psf.Plan(obs, prec="fp32") as plan:
        n = int(np.sum(obs.tavg))
        for tw in (np.full(n, -1.0, np.float32), np.zeros(n, np.float32), np.full(n, np.nan, np.float32)):
            with pytest.raises(psf.PsfError) as e:
                plan.set_windows(tw, None)
            assert e.value.status == psf.PSF_EINVAL


@pytest.mark.parametrize("prec", ["fp32", "tc_fp16", "tc_bf16x3"])
@pytest.mark.parametrize("method", ["uv", "img"])
def test_windowed_approximations(psf, prec, method):
    """Methods 1 and 2 with asymmetric baseline-dependent windows (complex decorrelation,
    so the per-cutout tensor-core form takes its complex-weight path), whole cutouts."""
    mid = {"uv": oracle.UV, "img": oracle.IMG}[method]
    for name, obs0, bg in _cases():
        obs = _asymmetric(obs0)
        ref = oracle.psf(obs, mid, bg)
        plain = oracle.psf(obsgen.Observation(obs.uvw_m, obs.time_s, obs.freq_hz, obs.chan_width_hz, obs.tavg,
                                              obs.favg, obs.weights), mid, bg)
        with psf.Plan(obs, prec=prec) as plan:
            got = plan.forward(method, psf.Batch.from_obsgen(bg)).cpu().numpy().astype(np.float64)
            assert plan.sync_status() == 0
        offs = obsgen.concat_pixels(bg)
        for p in range(bg.npos):
            n2 = int(bg.npix[p]) ** 2
            g, r = got[offs[p]:offs[p] + n2], ref[offs[p]:offs[p] + n2]
            err = np.max(np.abs(g - r)) / np.max(np.abs(r))
            assert err <= _tol(prec, obs), (name, method, p, err)
        assert np.max(np.abs(ref - plain)) > 1e-3 * np.max(np.abs(ref))   # the windows matter


def test_windowed_approximations_batched_and_fused(psf):
    """40 cutouts of 32^2 (the batched form, complex weights) and the fused call
    psf_approx_uv_img (two separate passes when windowed), FP16 tensor cores."""
    _, obs0, _ = _cases()[1]
    obs = _asymmetric(obs0)
    rng = np.random.default_rng(12)
    lm = rng.uniform(-0.04, 0.04, (40, 2))
    bg = obsgen.Batch(lm, np.full(40, 32, np.int32), 3e-5)
    sel = np.array([k * 1024 + 16 * 32 + 16 for k in (0, 9, 39)] + list(rng.choice(40 * 1024, 30, replace=False)))
    refs = {m: oracle.psf(obs, mid, bg, pix_sel=sel) for m, mid in (("uv", oracle.UV), ("img", oracle.IMG))}
    with psf.Plan(obs, prec="tc_fp16") as plan:
        b = psf.Batch.from_obsgen(bg)
        for m in ("uv", "img"):
            got = plan.forward(m, b).cpu().numpy().astype(np.float64)
            assert np.max(np.abs(got[sel] - refs[m][sel])) / np.max(np.abs(refs[m][sel])) <= 2e-3, m
        b2 = obsgen.Batch(lm[:2], np.full(2, 64, np.int32), 3e-5)
        guv, gimg = plan.approx_uv_img(psf.Batch.from_obsgen(b2))
        assert plan.sync_status() == 0
    for got, mid in ((guv, oracle.UV), (gimg, oracle.IMG)):
        ref = oracle.psf(obs, mid, b2)
        got = got.cpu().numpy().astype(np.float64)
        for p in range(2):
            sl = slice(p * 4096, (p + 1) * 4096)
            assert np.max(np.abs(got[sl] - ref[sl])) / np.max(np.abs(ref[sl])) <= 2e-3


@pytest.mark.parametrize("method", ["uv", "img"])
def test_windowed_adjoint_approximations(psf, method):
    import torch
    mid = {"uv": oracle.UV, "img": oracle.IMG}[method]
    _, obs0, bg = _cases()[1]
    obs = _asymmetric(obs0)
    P = oracle.psf(obs, mid, bg)
    rng = np.random.default_rng(5)
    R = 2 * (P - (P * (1 + 0.01 * rng.standard_normal(P.size)) + 0.05 * np.abs(P).max() * rng.standard_normal(P.size)))
    g_lm_ref, g_W_ref = oracle.vjp(obs, mid, bg, R)
    with psf.Plan(obs, prec="fp32") as plan:
        g_lm, g_W = plan.adjoint(method, psf.Batch.from_obsgen(bg), torch.tensor(R, dtype=torch.float32, device="cuda"))
        assert plan.sync_status() == 0
    g_lm, g_W = g_lm.cpu().numpy(), g_W.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(g_W - g_W_ref)) / np.max(np.abs(g_W_ref)) <= 2e-5
    assert np.max(np.abs(g_lm - g_lm_ref)) / np.max(np.abs(g_lm_ref)) <= 2e-4
