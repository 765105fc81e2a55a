"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: a closed form,
a limit, a symmetry, a library routine (numpy FFT), an undivided extended
precision brute force, or finite differences.  A plausible slip anywhere in the
oracle (dropped term, wrong sign or index, transposed operand, wrong pixel origin,
wrong normalisation) fails at least one of them.
"""
import math

import numpy as np
import pytest

import obsgen
import oracle
from oracle import brute

C = 299792458.0


def _static_obs(uv_lambda, nu, ntime=1, width=1.0):
    """Baselines whose uvw is constant in time, one raw channel at nu."""
    nbl = len(uv_lambda)
    uvw = np.zeros((nbl, ntime, 3))
    for b, (u, v) in enumerate(uv_lambda):
        uvw[b, :, 0] = u * C / nu
        uvw[b, :, 1] = v * C / nu
    t = (np.arange(ntime) + 0.5) * 1.0
    return obsgen.Observation(uvw, t, np.array([nu]), np.array([width]),
                              np.full(nbl, ntime, np.int32), 1)


# ----------------------------------------------------------------- P1
@pytest.mark.parametrize("method", [oracle.EXACT, oracle.UV, oracle.IMG])
def test_p1_phase_centre_no_distortion(method):
    """Eqs. 64-66: at l0 = 0 every decorrelation is exactly 1 and the PSF peak is sum W."""
    obs = obsgen.tiny_obs(weights=True)
    D = oracle.decorr(obs, method, 0.0, 0.0)
    assert np.max(np.abs(D - 1.0)) < 1e-14
    b = obsgen.Batch(np.zeros((1, 2)), np.array([16], np.int32), 2e-5)
    P = oracle.psf(obs, method, b).reshape(16, 16)
    W = obs.weights.astype(np.float64).sum()
    assert abs(P[8, 8] - W) < 1e-12 * W
    assert P[8, 8] == P.max()


def test_p1_effective_psf_equals_inverse_fft():
    """Eq. 8: the effective PSF is the inverse Fourier transform of the weighted
    sampling.  On a uv grid commensurate with the cutout, numpy's ifft2 of the
    gridded weights gives it exactly; this pins the pixel origin, the axis order
    (row = m, column = l), the twiddle and the normalisation."""
    N, cell = 16, 1e-4
    du = 1.0 / (N * cell)
    rng = np.random.default_rng(3)
    a = rng.integers(-7, 8, size=9)
    bb = rng.integers(-7, 8, size=9)
    nu = 1.0e9
    obs = _static_obs(list(zip(a * du, bb * du)), nu)
    obs.weights = rng.uniform(0.5, 2.0, size=9).astype(np.float32)
    P = oracle.psf(obs, oracle.EXACT, obsgen.Batch(np.zeros((1, 2)), np.array([N], np.int32), cell))
    G = np.zeros((N, N), complex)
    for k in range(9):
        G[bb[k] % N, a[k] % N] += obs.weights[k]
    ref = np.fft.fftshift(np.real(np.fft.ifft2(G)) * N * N)
    np.testing.assert_allclose(P.reshape(N, N), ref, rtol=0, atol=1e-10)


# ----------------------------------------------------------------- P2
def test_p2_smearing_limits():
    """Eqs. 17-19: with bins shrinking to a point, the averaged visibility equals the
    instantaneous one, so every decorrelation tends to 1."""
    l0, m0 = 0.03, -0.02
    prev = None
    for scale in [0.01, 0.001, 0.0001]:
        obs = obsgen.tiny_obs(dt=2.0 * scale, df=2e6 * scale)
        errs = [np.max(np.abs(oracle.decorr(obs, m, l0, m0) - 1)) for m in range(3)]
        if prev is not None:
            for e, p in zip(errs, prev):
                assert e < 0.05 * p          # second order: shrinking by 10 gives ~100x
        prev = errs
    assert max(prev) < 1e-7


# ----------------------------------------------------------------- P3
def test_p3_linear_track_dirichlet():
    """Single baseline, u(t) = u0 + a t, one narrow channel: the exact average over n
    instantaneous samples is the Dirichlet kernel sin(n pi x) / (n sin(pi x)) with
    x = nu a dt l0 / c; Method 1 gives sinc_pi(n x) (Eq. 35)."""
    nu, dt, l0 = 1.4e9, 1.0, 0.05
    for n, a in [(4, 3.0), (10, 1.7), (25, 0.9)]:
        obs = obsgen.linear_track_obs(2000.0, a, ntime=3 * n, dt=dt, tavg=n,
                                      freq_hz=[nu], width_hz=1e-3, favg=1)
        x = nu * a * dt * l0 / C
        dirichlet = math.sin(n * math.pi * x) / (n * math.sin(math.pi * x))
        D = oracle.decorr(obs, oracle.EXACT, l0, 0.0)
        np.testing.assert_allclose(D.real, dirichlet, rtol=0, atol=1e-11)
        np.testing.assert_allclose(D.imag, 0.0, atol=1e-11)
        Duv = oracle.decorr(obs, oracle.UV, l0, 0.0)
        sinc_n = math.sin(n * math.pi * x) / (n * math.pi * x)
        np.testing.assert_allclose(Duv.real, sinc_n, rtol=0, atol=1e-11)


def test_p3_dirichlet_tends_to_sinc():
    """With the bin length n dt fixed and n growing, the discrete mean tends to the
    continuous boxcar average, i.e. the exact decorrelation tends to Method 1."""
    nu, l0, T = 1.4e9, 0.05, 40.0
    gaps = []
    for n in [4, 16, 64]:
        obs = obsgen.linear_track_obs(5000.0, 0.1, ntime=n, dt=T / n, tavg=n,
                                      freq_hz=[nu], width_hz=1e-3, favg=1)
        gaps.append(abs(oracle.decorr(obs, 0, l0, 0)[0] - oracle.decorr(obs, 1, l0, 0)[0]))
    assert gaps[1] < gaps[0] / 10 and gaps[2] < gaps[1] / 10


def test_p3_contiguous_channels_integrate_the_band():
    """A static baseline observed in F contiguous equal channels: the channel-averaged
    fringe is the continuous band average sinc_pi(X Dnu / c) (boxcar, Eq. 14)."""
    for F, width in [(1, 5e6), (4, 2e6), (7, 0.5e6)]:
        f0 = 1.0e9
        freq = f0 + (np.arange(F) + 0.5) * width
        obs = obsgen.linear_track_obs(3000.0, 0.0, ntime=1, dt=1.0, tavg=1,
                                      freq_hz=freq, width_hz=width, favg=F)
        for l0 in [0.01, 0.07]:
            X = 3000.0 * l0
            D = oracle.decorr(obs, oracle.EXACT, l0, 0.0)[0]
            y = X * F * width / C
            np.testing.assert_allclose(D.real, math.sin(math.pi * y) / (math.pi * y), atol=1e-12)
            np.testing.assert_allclose(D.imag, 0.0, atol=1e-12)


# ----------------------------------------------------------------- P4
def test_p4_hermitian_mirror():
    """Eq. 1 with real skies: the mirrored baseline -uvw measures the conjugate, so
    D(-uvw) = conj D(uvw), and the real PSF of the mirrored array is unchanged."""
    obs = obsgen.tiny_obs()
    mir = obsgen.Observation(-obs.uvw_m, obs.time_s, obs.freq_hz, obs.chan_width_hz,
                             obs.tavg, obs.favg)
    for method in range(3):
        D = oracle.decorr(obs, method, 0.04, 0.01)
        Dm = oracle.decorr(mir, method, 0.04, 0.01)
        np.testing.assert_allclose(Dm, np.conj(D), atol=1e-14)
    b = obsgen.Batch(np.array([[0.04, 0.01]]), np.array([12], np.int32), 3e-5)
    np.testing.assert_allclose(oracle.psf(mir, 0, b), oracle.psf(obs, 0, b), rtol=0, atol=1e-10)


@pytest.mark.parametrize("method", [oracle.UV, oracle.IMG])
def test_p4_real_decorrelation_gives_centrosymmetric_cutout(method):
    """For real D (Methods 1 and 2) each term is W D cos(phase), even in the offset."""
    obs = obsgen.tiny_obs()
    N = 12
    P = oracle.psf(obs, method, obsgen.Batch(np.array([[0.05, -0.03]]), np.array([N], np.int32),
                                             4e-5)).reshape(N, N)
    inner = P[1:, 1:]
    np.testing.assert_allclose(inner, inner[::-1, ::-1], rtol=0, atol=1e-10 * abs(P).max())


def test_p4_imaginary_part_flips_under_mirroring():
    """The imaginary part of the complex sum (PSF_COMPLEX_OUT): the mirrored array
    measures conjugate visibilities, so its imaginary cutout is the negative of the
    original for every method (D(-uvw) = conj D(uvw), conj twiddles)."""
    obs = obsgen.tiny_obs()
    mir = obsgen.Observation(-obs.uvw_m, obs.time_s, obs.freq_hz, obs.chan_width_hz,
                             obs.tavg, obs.favg)
    b = obsgen.Batch(np.array([[0.04, 0.01]]), np.array([12], np.int32), 3e-5)
    for method in range(3):
        im = oracle.psf(obs, method, b, imag=True)
        im_m = oracle.psf(mir, method, b, imag=True)
        assert np.max(np.abs(im)) > 1e-3 * np.max(np.abs(oracle.psf(obs, method, b)))
        np.testing.assert_allclose(im_m, -im, rtol=0, atol=1e-10 * np.max(np.abs(im)))


def test_p1_imaginary_part_at_zero_smearing():
    """With D = 1 (phase centre) the imaginary part is sum_k W_k sin(2 pi (u_k dl + v_k dm)):
    on a uv grid commensurate with the cutout it is the imaginary part of numpy's
    ifft2 of the gridded weights."""
    N, cell = 16, 1e-4
    du = 1.0 / (N * cell)
    rng = np.random.default_rng(5)
    a = rng.integers(-7, 8, size=9)
    bb = rng.integers(-7, 8, size=9)
    obs = _static_obs(list(zip(a * du, bb * du)), 1.0e9)
    obs.weights = rng.uniform(0.5, 2.0, size=9).astype(np.float32)
    P = oracle.psf(obs, oracle.EXACT, obsgen.Batch(np.zeros((1, 2)), np.array([N], np.int32), cell), imag=True)
    G = np.zeros((N, N), complex)
    for k in range(9):
        G[bb[k] % N, a[k] % N] += obs.weights[k]
    ref = np.fft.fftshift(np.imag(np.fft.ifft2(G)) * N * N)
    np.testing.assert_allclose(P.reshape(N, N), ref, rtol=0, atol=1e-10)


# ----------------------------------------------------------------- P5
def test_p5_linear_in_weights():
    obs1 = obsgen.tiny_obs(weights=True)
    obs2 = obsgen.tiny_obs(seed=7, weights=True)
    obs2.weights = np.random.default_rng(9).uniform(0, 1, obs1.nvis()).astype(np.float32)
    obs12 = obsgen.tiny_obs(weights=True)
    obs12.weights = (obs1.weights.astype(np.float64) + obs2.weights).astype(np.float32)
    b = obsgen.Batch(np.array([[0.02, 0.03]]), np.array([8], np.int32), 5e-5)
    for method in range(3):
        p12 = oracle.psf(obs12, method, b)
        p1 = oracle.psf(obs1, method, b)
        p2 = oracle.psf(obs2, method, b)
        np.testing.assert_allclose(p12, p1 + p2, rtol=1e-6, atol=1e-6 * abs(p12).max())


# ----------------------------------------------------------------- P6
@pytest.mark.parametrize("wterm", [False, True])
def test_p6_bruteforce_undivided(wterm):
    """The factored oracle (absolute phase cancelled analytically, closed-form
    channel integral) equals the undivided extended-precision sum with quadrature."""
    obs = obsgen.tiny_obs(nant=3, ntime=12, nchan=4, tavg=[3, 4, 6], favg=2, weights=True)
    for (l0, m0) in [(0.03, -0.02), (-0.06, 0.045)]:
        N, cell = 8, 6e-5
        ref = brute.psf_exact(obs, l0, m0, N, cell, wterm=wterm).astype(np.float64)
        got = oracle.psf(obs, oracle.EXACT, obsgen.Batch(np.array([[l0, m0]]), np.array([N], np.int32),
                                                         cell), flags=oracle.WTERM if wterm else 0)
        np.testing.assert_allclose(got.reshape(N, N), ref, rtol=0, atol=1e-11 * abs(ref).max())
        # the imaginary part along the same undivided route
        ref_i = brute.psf_exact(obs, l0, m0, N, cell, wterm=wterm, imag=True).astype(np.float64)
        got_i = oracle.psf(obs, oracle.EXACT, obsgen.Batch(np.array([[l0, m0]]), np.array([N], np.int32), cell),
                           flags=oracle.WTERM if wterm else 0, imag=True)
        np.testing.assert_allclose(got_i.reshape(N, N), ref_i, rtol=0, atol=1e-11 * abs(ref).max())


# ----------------------------------------------------------------- P7
def test_p7_approximation_order_and_growth():
    """Sect. 4: the uv-plane approximation is closer to the exact PSF than the
    image-plane one, and both errors grow with distance from the phase centre."""
    obs = obsgen.tiny_obs(nant=6, ntime=40, nchan=8, tavg=10, favg=4, dt=2.0, df=2e6,
                          radius_m=6000.0)
    N, cell = 16, 4e-5
    errs = []
    for r in [0.005, 0.02, 0.05]:
        b = obsgen.Batch(np.array([[r * 0.6, r * 0.8]]), np.array([N], np.int32), cell)
        ex = oracle.psf(obs, oracle.EXACT, b)
        peak = abs(ex).max()
        e_uv = abs(oracle.psf(obs, oracle.UV, b) - ex).max() / peak
        e_img = abs(oracle.psf(obs, oracle.IMG, b) - ex).max() / peak
        assert e_uv <= e_img
        errs.append((e_uv, e_img))
    assert errs[0][0] < errs[1][0] < errs[2][0]
    assert errs[0][1] < errs[1][1] < errs[2][1]


def test_p7_circular_track_model_matches_method1():
    """Eqs. 38-41 model E-W baselines tracing circles; a pure E-W baseline seen at the
    celestial pole does exactly that, and with negligible bandwidth the model's time
    decorrelation equals Method 1's edge-difference one up to O((omega dt)^2)."""
    enu = np.array([[0.0, 0, 0], [4000.0, 0, 0]])
    t = -3 * 3600.0 + (np.arange(10800) + 0.5) * 2.0           # 6 h at 2 s
    uvw = obsgen.uvw_tracks(enu, -90 * obsgen.DEG, -90 * obsgen.DEG, t)
    obs = obsgen.Observation(uvw, t, np.array([1.4e9]), np.array([1.0]), np.array([11], np.int32), 1)
    worst = 0.0
    for (l0, m0) in [(0.01, 0.0), (0.0, 0.01), (0.006, -0.008)]:
        Duv = oracle.decorr(obs, oracle.UV, l0, m0).real
        Dimg = oracle.decorr(obs, oracle.IMG, l0, m0).real
        worst = max(worst, np.max(np.abs(1 - Duv)))
        np.testing.assert_allclose(Dimg, Duv, rtol=0, atol=2e-5)
    assert worst > 0.05                                       # the case is not trivial


# ----------------------------------------------------------------- P8
@pytest.mark.parametrize("method", [oracle.EXACT, oracle.UV, oracle.IMG])
def test_p8_vjp_matches_central_differences(method):
    obs = obsgen.tiny_obs(nant=3, ntime=16, nchan=4, tavg=4, favg=2, weights=True)
    rng = np.random.default_rng(5)
    lm = np.array([[0.031, -0.017], [-0.022, 0.041]])
    b = obsgen.Batch(lm, np.array([8, 6], np.int32), 5e-5)
    P = oracle.psf(obs, method, b)
    T = P * (1 + 0.01 * rng.standard_normal(P.size)) + 0.05 * abs(P).max() * rng.standard_normal(P.size)
    R = 2 * (P - T)
    g_lm, g_W = oracle.vjp(obs, method, b, R)

    def loss(lm_, W_=None):
        o = obs
        if W_ is not None:
            o = obsgen.Observation(obs.uvw_m, obs.time_s, obs.freq_hz, obs.chan_width_hz,
                                   obs.tavg, obs.favg, W_.astype(np.float32))
        return np.sum((oracle.psf(o, method, obsgen.Batch(lm_, b.npix, b.cell_rad)) - T) ** 2)

    h = 1e-7
    for p in range(2):
        for d in range(2):
            lp, lmn = lm.copy(), lm.copy()
            lp[p, d] += h
            lmn[p, d] -= h
            fd = (loss(lp) - loss(lmn)) / (2 * h)
            assert abs(fd - g_lm[p, d]) < 2e-5 * max(abs(g_lm).max(), 1e-30)
    # W enters linearly, L quadratically: central differences are exact up to rounding.
    W = obs.weights.astype(np.float64)
    for k in rng.choice(W.size, 5, replace=False):
        hw = 1e-3 * W[k]
        Wp, Wm = W.copy(), W.copy()
        Wp[k] += hw
        Wm[k] -= hw
        # weights are float32 in the interface: use exactly representable steps
        Wp = Wp.astype(np.float32).astype(np.float64)
        Wm = Wm.astype(np.float32).astype(np.float64)
        fd = (loss(lm, Wp) - loss(lm, Wm)) / (Wp[k] - Wm[k])
        assert abs(fd - g_W[k]) < 1e-6 * max(abs(g_W).max(), 1e-30)


def test_vis_table_bins_and_edges():
    """Eqs. 12 and 33 on a hand-checkable track: 3 baselines, unequal averaging."""
    obs = obsgen.tiny_obs(nant=3, ntime=12, nchan=4, tavg=[3, 4, 5], favg=2)
    tab = oracle.vis_table(obs)
    # bins: 12//3 + 12//4 + 12//5 = 4 + 3 + 2 = 9 time bins, 2 output channels
    assert tab["W"].shape[0] == 9 * 2
    np.testing.assert_array_equal(tab["W"], np.repeat([6, 6, 6, 6, 8, 8, 8, 10, 10], 2))
    # first bin of baseline 0: mean of samples 0..2; edge delta spans 3 sample intervals
    u = obs.uvw_m[0]
    np.testing.assert_allclose(tab["ubar_m"][0], u[0:3].mean(0), rtol=1e-15)
    np.testing.assert_allclose(tab["dedge_m"][0], (u[2] - u[0]) * 3 / 2, rtol=1e-13)
    # channel centres and widths of the 2:1 averaged band
    np.testing.assert_allclose(tab["nu"][:2], [obs.freq_hz[:2].mean(), obs.freq_hz[2:].mean()])
    np.testing.assert_allclose(tab["dnu"][:2], [4e6, 4e6])
    np.testing.assert_allclose(tab["dt"][0], 3 * 2.0)
    np.testing.assert_allclose(tab["uvw_lambda"][0], u[0:3].mean(0) * tab["nu"][0] / C, rtol=1e-15)


def test_p3_unequal_contiguous_channels():
    """Eq. 13 weights each raw channel by its width: channels of unequal widths that
    tile a band average to the band integral, whose closed form is
    exp(-2 pi i (nu_mid - nu_r) X / c) sinc_pi(X Dnu / c) after removing the
    centre-visibility phase (nu_r is the mean of the channel centres)."""
    widths = np.array([1e6, 3e6, 2e6])
    edges = 1.2e9 + np.concatenate([[0], np.cumsum(widths)])
    freq = 0.5 * (edges[:-1] + edges[1:])
    obs = obsgen.linear_track_obs(2500.0, 0.0, ntime=1, dt=1.0, tavg=1,
                                  freq_hz=freq, width_hz=widths, favg=3)
    nu_r, nu_mid, dnu = freq.mean(), 0.5 * (edges[0] + edges[-1]), widths.sum()
    for l0 in [0.004, 0.03]:
        X = 2500.0 * l0
        ref = np.exp(-2j * np.pi * (nu_mid - nu_r) * X / C) * np.sinc(X * dnu / C)
        D = oracle.decorr(obs, oracle.EXACT, l0, 0.0)[0]
        assert abs(D - ref) < 1e-12


# ----------------------------------------------------------------- Algorithm 1, printed theta
def _dsinc(y):
    return 0.0 if y == 0 else (math.cos(math.pi * y) - np.sinc(y)) / y


@pytest.mark.parametrize("uv", [(0.0, 3000.0), (0.0, -2500.0), (4000.0, 0.0), (-1800.0, 0.0)])
def test_literal_theta_closed_forms(uv):
    """Algorithm 1's printed theta = arctan(u/v) (Sect. 3.2), pinned on baselines along the
    axes, where the arctangent is fixed: u = 0 gives theta = 0 and (du/dt, dv/dt) =
    omega_E |uv| (-sin theta, cos theta) = omega_E (0, |v|), so dPsi/(2 pi) =
    omega_E Dt |v| m0; v = 0 gives theta = +-pi/2 and dPsi/(2 pi) = -+omega_E Dt |u| l0.
    D = sinc_pi(dPsi / 2 pi) sinc_pi((Dnu/nu) |uv| rho) and its l0, m0 derivatives in
    closed form.  The default reading theta = atan2(v, u) pairs the other way (u = 0:
    dPsi/(2 pi) = -omega_E Dt v l0), so a swapped sine and cosine in either branch fails."""
    u, v = uv
    nu, width, ntime = 1.4e9, 2e6, 100
    dt = float(ntime)                                 # one bin of 100 samples of 1 s
    l0, m0 = 0.031, -0.017
    rho = math.hypot(l0, m0)
    obs = _static_obs([(u, v)], nu, ntime=ntime, width=width)
    uvlen = math.hypot(u, v)
    w = obsgen.OMEGA_E * dt
    if u == 0.0:
        A, Al, Am = w * abs(v) * m0, 0.0, w * abs(v)
        A_def = -w * v * l0
    else:
        A, Al, Am = -w * u * l0, -w * u, 0.0
        A_def = w * u * m0
    B = width / nu * uvlen * rho
    Bl, Bm = width / nu * uvlen * l0 / rho, width / nu * uvlen * m0 / rho
    D, g = oracle.decorr(obs, oracle.IMG, l0, m0, flags=oracle.LITERAL_THETA, grad=True)
    assert abs(D[0] - np.sinc(A) * np.sinc(B)) < 1e-13
    assert abs(D[0].imag) == 0.0
    assert abs(g[0, 0] - (_dsinc(A) * Al * np.sinc(B) + np.sinc(A) * _dsinc(B) * Bl)) < 1e-11
    assert abs(g[0, 2] - (_dsinc(A) * Am * np.sinc(B) + np.sinc(A) * _dsinc(B) * Bm)) < 1e-11
    D_def = oracle.decorr(obs, oracle.IMG, l0, m0)
    assert abs(D_def[0] - np.sinc(A_def) * np.sinc(B)) < 1e-13
    assert abs(D_def[0] - D[0]) > 1e-3   # the two readings differ on these baselines
