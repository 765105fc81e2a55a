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
