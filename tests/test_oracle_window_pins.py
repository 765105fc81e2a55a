"""Pins of the oracle's windowed bin average (Sect. 2.3, Eqs. 15-16: the normalised boxcar
replaced by a window over the bin's samples and raw channels).

Checked against: the boxcar (a constant window reproduces the unwindowed exact average),
the single-sample fringe (a window on one sample and one raw channel leaves that sample's
phase relative to the bin centre times its channel's sinc, from the raw data), the phase
centre (D = 1 for any window), normalisation (scaling a window changes nothing) and the
Hermitian mirror."""
import numpy as np
import pytest

import obsgen
import oracle

C = 299792458.0


def _with(obs, tw=None, cw=None):
    o = obsgen.Observation(obs.uvw_m, obs.time_s, obs.freq_hz, obs.chan_width_hz, obs.tavg, obs.favg,
                           obs.weights, obs.enu_m, tw, cw)
    return o


def test_w1_constant_window_is_the_boxcar():
    obs = obsgen.tiny_obs(tavg=[2, 3, 4, 6, 8, 12], favg=2, nchan=8, weights=True)
    ref = oracle.decorr(obs, oracle.EXACT, 0.03, -0.02)
    o = _with(obs, np.full(int(np.sum(obs.tavg)), 3.0, np.float32), np.full((obs.nbl, obs.favg), 0.5, np.float32))
    np.testing.assert_allclose(oracle.decorr(o, oracle.EXACT, 0.03, -0.02), ref, rtol=0, atol=1e-13)


def test_w2_single_sample_single_channel():
    obs = obsgen.tiny_obs(tavg=4, favg=2, nchan=4)
    tw = np.zeros(int(np.sum(obs.tavg)), np.float32)
    cw = np.zeros((obs.nbl, obs.favg), np.float32)
    s_star, c_star = 2, 1
    for b in range(obs.nbl):
        tw[b * 4 + s_star] = 1.0
        cw[b, c_star] = 1.0
    o = _with(obs, tw, cw)
    l0, m0 = 0.04, 0.015
    D = oracle.decorr(o, oracle.EXACT, l0, m0)
    vt = oracle.vis_table(obs)
    nout = obs.nchan // obs.favg
    nb = obs.ntime // 4
    k = 0
    for b in range(obs.nbl):
        for tau in range(nb):
            for r in range(nout):
                s = tau * 4 + s_star
                c = r * obs.favg + c_star
                X = obs.uvw_m[b, s, 0] * l0 + obs.uvw_m[b, s, 1] * m0
                Xbar = vt["ubar_m"][k, 0] * l0 + vt["ubar_m"][k, 1] * m0
                ref = np.exp(-2j * np.pi * (obs.freq_hz[c] * X - vt["nu"][k] * Xbar) / C) \
                    * np.sinc(X * obs.chan_width_hz[c] / C)
                assert D[k] == pytest.approx(ref, abs=1e-12)
                k += 1


def test_w3_phase_centre_and_normalisation():
    obs = obsgen.tiny_obs(tavg=[2, 3, 4, 6, 8, 12], favg=2, nchan=8)
    tw, cw = obsgen.bd_windows(obs, 2.0)
    o = _with(obs, tw, cw)
    assert np.max(np.abs(oracle.decorr(o, oracle.EXACT, 0.0, 0.0) - 1.0)) < 1e-14
    o2 = _with(obs, tw * 8.0, cw * 0.25)          # powers of two: exact in float32
    np.testing.assert_allclose(oracle.decorr(o2, oracle.EXACT, 0.05, 0.02), oracle.decorr(o, oracle.EXACT, 0.05, 0.02),
                               rtol=0, atol=1e-13)
    # the taper does change the average
    assert np.max(np.abs(oracle.decorr(o, oracle.EXACT, 0.05, 0.02) - oracle.decorr(obs, oracle.EXACT, 0.05, 0.02))) > 1e-4


def test_w4_hermitian_mirror():
    obs = obsgen.tiny_obs(tavg=3, favg=2, nchan=4)
    tw, cw = obsgen.bd_windows(obs, 1.0)
    o = _with(obs, tw, cw)
    m = _with(obsgen.Observation(-obs.uvw_m, obs.time_s, obs.freq_hz, obs.chan_width_hz, obs.tavg, obs.favg), tw, cw)
    np.testing.assert_allclose(oracle.decorr(m, oracle.EXACT, 0.03, 0.01), np.conj(oracle.decorr(o, oracle.EXACT, 0.03, 0.01)),
                               rtol=0, atol=1e-13)


# ------------------------------------------------------------------ Methods 1 and 2 with windows
# With a window the two sincs of Methods 1 and 2 (Eq. 35 and Eqs. 42-44) become the
# transforms of the window: the time factor T(A) = average over the bin of
# exp(-2 pi i A tau) weighted by the window (raw sample s carrying its weight over its own
# 1/n of the bin), the frequency factor F(B) likewise over the band (raw channel c carrying
# its weight over its own width).  A = dPsi / (2 pi), B = dPhi / (2 pi).

def _AB_method1(obs, l0, m0):
    vt = oracle.vis_table(obs)
    A = (vt["dedge_m"][:, 0] * l0 + vt["dedge_m"][:, 1] * m0) * vt["nu"] / C
    B = (vt["ubar_m"][:, 0] * l0 + vt["ubar_m"][:, 1] * m0) * vt["dnu"] / C
    return A, B


@pytest.mark.parametrize("method", [oracle.UV, oracle.IMG])
def test_w5_constant_window_is_the_boxcar_for_the_approximations(method):
    obs = obsgen.tiny_obs(tavg=[2, 3, 4, 6, 8, 12], favg=2, nchan=8, weights=True)
    ref = oracle.decorr(obs, method, 0.03, -0.02)
    o = _with(obs, np.full(int(np.sum(obs.tavg)), 3.0, np.float32), np.full((obs.nbl, obs.favg), 0.5, np.float32))
    np.testing.assert_allclose(oracle.decorr(o, method, 0.03, -0.02), ref, rtol=0, atol=1e-13)


def test_w6_time_factor_is_the_transform_of_the_window():
    """One raw channel per output channel (no channel window, F = sinc_pi(B)), a
    baseline-dependent time window: D / sinc_pi(B) equals the bin average of
    exp(-2 pi i A tau) under the piecewise-constant window, by midpoint quadrature."""
    obs = obsgen.tiny_obs(tavg=[3, 5, 8, 4, 6, 7], favg=1, nchan=3, ntime=40, dt=20.0)
    tw, _ = obsgen.bd_windows(obs, 2.0)
    tw = tw * (1.0 + 0.3 * np.sin(np.arange(tw.size)))          # asymmetric tapers
    tw = tw.astype(np.float32)
    o = _with(obs, tw, None)
    l0, m0 = 0.08, -0.05
    D = oracle.decorr(o, oracle.UV, l0, m0)
    A, B = _AB_method1(obs, l0, m0)
    vt = oracle.vis_table(obs)
    toff = np.concatenate([[0], np.cumsum(obs.tavg)[:-1]])
    nout = obs.nchan // obs.favg
    k = 0
    M = 4000                                                     # quadrature points per raw sample
    for b in range(obs.nbl):
        n = int(obs.tavg[b])
        x = tw[toff[b]:toff[b] + n].astype(np.float64)
        x /= x.sum()
        tau = (np.arange(n * M) + 0.5) / (n * M) - 0.5          # midpoints over the bin
        dens = np.repeat(x * n, M)                               # window density (integrates to 1)
        for _ in range(obs.ntime // n):
            for _ in range(nout):
                T = np.mean(dens * np.exp(-2j * np.pi * A[k] * tau))
                assert D[k] / np.sinc(B[k]) == pytest.approx(T, abs=2e-8)
                k += 1
    assert k == vt["nu"].size
    assert np.max(np.abs(D.imag)) > 1e-3                          # an asymmetric window: complex D


def test_w7_frequency_factor_is_the_transform_of_the_window():
    """A channel window only (T = sinc_pi(A)), unequal raw channels: D / sinc_pi(A)
    equals the average over the band of exp(-2 pi i B nu~) under the piecewise-constant
    channel window (weight x width per raw channel), nu~ = (nu - nu_r) / Dnu_r."""
    obs = obsgen.tiny_obs(nant=4, ntime=24, nchan=6, tavg=4, favg=3)
    obs.chan_width_hz = np.array([1e6, 3e6, 2e6, 2e6, 2e6, 1e6])
    edges = 1.2e9 + np.concatenate([[0], np.cumsum(obs.chan_width_hz)])
    obs.freq_hz = 0.5 * (edges[:-1] + edges[1:])
    rng = np.random.default_rng(8)
    cw = rng.uniform(0.2, 1.0, (obs.nbl, obs.favg)).astype(np.float32)
    o = _with(obs, None, cw)
    l0, m0 = 0.35, 0.2                                          # strong bandwidth smearing
    D = oracle.decorr(o, oracle.UV, l0, m0)
    A, B = _AB_method1(obs, l0, m0)
    vt = oracle.vis_table(obs)
    nout, nb = obs.nchan // obs.favg, obs.ntime // 4
    M = 20000
    k = 0
    for b in range(obs.nbl):
        for _ in range(nb):
            for r in range(nout):
                c = np.arange(r * 3, r * 3 + 3)
                y = cw[b].astype(np.float64) * obs.chan_width_hz[c]
                y /= y.sum()
                lo = (edges[c] - vt["nu"][k]) / vt["dnu"][k]
                hi = (edges[c + 1] - vt["nu"][k]) / vt["dnu"][k]
                F = 0j
                for q in range(3):                               # density y_q / width_q over channel q
                    nu = lo[q] + (np.arange(M) + 0.5) / M * (hi[q] - lo[q])
                    F += y[q] * np.mean(np.exp(-2j * np.pi * B[k] * nu))
                assert D[k] / np.sinc(A[k]) == pytest.approx(F, abs=2e-8)
                k += 1


def test_w8_windowed_method1_tends_to_the_windowed_exact_average():
    """Linear track u(t) = u0 + a t, one raw channel: the exact windowed average is the
    discrete window mean of the fringe, Method 1 the piecewise-constant one; they differ
    by the sub-interval sinc, so the difference falls as 1/n^2 as the bin is sampled more
    finely at a fixed bin length."""
    l0 = 0.02
    errs = []
    for n in (8, 32):
        T = 64.0
        obs = obsgen.linear_track_obs(3000.0, 0.1, ntime=n, dt=T / n, tavg=n, freq_hz=[1.4e9], width_hz=[1.0],
                                      favg=1)   # phase change across the bin A = 0.6 turns
        s = np.arange(n)
        tw = np.exp(-0.5 * ((s - 0.3 * n) / (0.3 * n)) ** 2).astype(np.float32)
        o = _with(obs, tw, None)
        Dex = oracle.decorr(o, oracle.EXACT, l0, 0.0)[0]
        Duv = oracle.decorr(o, oracle.UV, l0, 0.0)[0]
        errs.append(abs(Dex - Duv))
        assert abs(Duv.imag) > 1e-2                                # asymmetric window: complex
    assert errs[1] < errs[0] / 10 and errs[1] < 2e-3, errs


def test_w9_phase_centre_and_mirror_for_the_approximations():
    obs = obsgen.tiny_obs(tavg=[2, 3, 4, 6, 8, 12], favg=2, nchan=8)
    tw, cw = obsgen.bd_windows(obs, 2.0)
    tw = (tw * (1.0 + 0.3 * np.cos(np.arange(tw.size)))).astype(np.float32)
    o = _with(obs, tw, cw)
    for method in (oracle.UV, oracle.IMG):
        assert np.max(np.abs(oracle.decorr(o, method, 0.0, 0.0) - 1.0)) < 1e-14
    m = _with(obsgen.Observation(-obs.uvw_m, obs.time_s, obs.freq_hz, obs.chan_width_hz, obs.tavg, obs.favg), tw, cw)
    np.testing.assert_allclose(oracle.decorr(m, oracle.UV, 0.03, 0.01), np.conj(oracle.decorr(o, oracle.UV, 0.03, 0.01)),
                               rtol=0, atol=1e-13)


@pytest.mark.parametrize("method", [oracle.UV, oracle.IMG])
def test_w10_windowed_vjp_matches_central_differences(method):
    obs = obsgen.tiny_obs(nant=3, ntime=16, nchan=4, tavg=4, favg=2, weights=True)
    tw, cw = obsgen.bd_windows(obs, 1.5)
    tw = (tw * (1.0 + 0.4 * np.sin(np.arange(tw.size)))).astype(np.float32)
    o = _with(obs, tw, cw)
    rng = np.random.default_rng(6)
    lm = np.array([[0.031, -0.017], [-0.022, 0.041]])
    b = obsgen.Batch(lm, np.array([8, 6], np.int32), 5e-5)
    P = oracle.psf(o, method, b)
    T = P * (1 + 0.01 * rng.standard_normal(P.size)) + 0.05 * abs(P).max() * rng.standard_normal(P.size)
    g_lm, _ = oracle.vjp(o, method, b, 2 * (P - T))

    def loss(lm_):
        return np.sum((oracle.psf(o, method, obsgen.Batch(lm_, b.npix, b.cell_rad)) - T) ** 2)

    h = 1e-7
    for p in range(2):
        for d in range(2):
            lp, lmn = lm.copy(), lm.copy()
            lp[p, d] += h
            lmn[p, d] -= h
            fd = (loss(lp) - loss(lmn)) / (2 * h)
            assert abs(fd - g_lm[p, d]) < 2e-5 * max(abs(g_lm).max(), 1e-30)
