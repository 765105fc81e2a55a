"""Pins of the oracle's FWHM along the radial and tangential directions (Fig. 3).

Checked against analytic shapes: elliptical Gaussians whose axes are the radial and
tangential directions of the cutout's position (the half-maximum widths are
2 sqrt(2 ln 2) sigma), rotation of a circular Gaussian, and a separable profile whose
piecewise-linear crossing is known exactly."""
import math

import numpy as np
import pytest

import oracle

K = 2.0 * math.sqrt(2.0 * math.log(2.0))


def _gauss(N, sr, st, phi):
    c = N // 2
    y, x = np.mgrid[0:N, 0:N].astype(np.float64)
    dx, dy = x - c, y - c
    r = dx * math.cos(phi) + dy * math.sin(phi)
    t = -dx * math.sin(phi) + dy * math.cos(phi)
    return np.exp(-0.5 * (r / sr) ** 2 - 0.5 * (t / st) ** 2)


@pytest.mark.parametrize("phi", [0.0, 0.3, 1.1, 2.5, -2.0])
def test_f1_elliptical_gaussian_axes(phi):
    """sigma of 8 and 5 pixels: bilinear interpolation moves the crossing by < 0.3 %."""
    N, cell = 96, 2e-6
    sr, st = 8.0, 5.0
    P = _gauss(N, sr, st, phi)
    rho = 0.02
    fr, ft = oracle.fwhm(P, rho * math.cos(phi), rho * math.sin(phi), cell)
    assert fr == pytest.approx(K * sr * cell, rel=4e-3)
    assert ft == pytest.approx(K * st * cell, rel=4e-3)


def test_f2_circular_gaussian_any_direction():
    P = _gauss(64, 6.0, 6.0, 0.0)
    w = [oracle.fwhm(P, math.cos(a), math.sin(a), 1.0) for a in np.linspace(0, 3, 7)]
    for fr, ft in w:
        assert fr == pytest.approx(ft, rel=3e-3)
        assert fr == pytest.approx(K * 6.0, rel=4e-3)


def test_f3_piecewise_linear_crossing_exact():
    """A cutout that is linear along l near the centre (1 - |dx| / 8, constant in m):
    bilinear interpolation reproduces it and the linear crossing lands exactly on
    |dx| = 4 on both sides, so the radial FWHM at a position on the l axis is 8 cells
    and the tangential one (along m, constant profile) leaves the cutout: NaN."""
    N = 32
    x = np.arange(N) - N // 2
    P = np.tile(np.maximum(1.0 - np.abs(x) / 8.0, -1.0), (N, 1))
    fr, ft = oracle.fwhm(P, 0.01, 0.0, 1.0)
    assert fr == pytest.approx(8.0, abs=1e-12)
    assert math.isnan(ft)


def _linear_crossing(f):
    """Where the linear interpolant of samples f[0], f[1], ... first falls to f[0] / 2."""
    h = 0.5 * f[0]
    for k in range(1, len(f)):
        if f[k] <= h:
            return k - 1 + (f[k - 1] - h) / (f[k - 1] - f[k])
    return math.nan


def test_f4_centre_position_uses_the_axes():
    """At l0 = 0 the radial and tangential directions are the l and m axes; along an axis
    bilinear interpolation is linear between pixels, so the widths are exactly the
    crossings of the pixel samples' linear interpolant (both sides)."""
    N = 48
    P = _gauss(N, 2.0, 5.0, 0.0)           # narrow along l, wide along m
    P[N // 2, N // 2 + 3] *= 0.97           # break the left-right symmetry a little
    c = N // 2
    fr, ft = oracle.fwhm(P, 0.0, 0.0, 1.0)
    er = _linear_crossing(P[c, c:]) + _linear_crossing(P[c, c::-1])
    et = _linear_crossing(P[c:, c]) + _linear_crossing(P[c::-1, c])
    assert fr == pytest.approx(er, abs=1e-12) and ft == pytest.approx(et, abs=1e-12)
