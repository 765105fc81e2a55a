"""Pins of the gridded image-plane oracle (Eq. 45 with Algorithm 1 on uv cells).

Each test checks ``oracle.grid_tables`` / ``oracle.psf_img_grid`` against something
other than their own code: numpy's FFT, the visibility-level Method 2 oracle
(already pinned against closed forms) on inputs where the two forms must agree
exactly, a brute-force gridding in numpy, and symmetries.  A wrong cell spacing,
index origin, transform sign or axis, a missing mirror cell, a wrong wrap or a
wrong cell mean fails at least one of them.
"""
import numpy as np
import pytest

import obsgen
import oracle

C = 299792458.0


def _obs(uv_cells, du, nu=1.0e9, ntime=64, dt=1.0, width=5.0e7, tavg=None, weights=None):
    """Baselines whose uvw is constant in time at (a du, b du) wavelengths, one channel."""
    nbl = len(uv_cells)
    uvw = np.zeros((nbl, ntime, 3))
    for k, (a, b) in enumerate(uv_cells):
        uvw[k, :, 0] = a * du * C / nu
        uvw[k, :, 1] = b * du * C / nu
    t = (np.arange(ntime) + 0.5) * dt
    tavg = np.full(nbl, ntime, np.int32) if tavg is None else np.asarray(tavg, np.int32)
    o = obsgen.Observation(uvw, t, np.array([nu]), np.array([width]), tavg, 1)
    if weights is not None:
        o.weights = np.asarray(weights, np.float32)
    return o


def _dft_limit(obs, lm, N, cell, flags=0):
    lm = np.asarray(lm, np.float64).reshape(-1, 2)
    b = obsgen.Batch(lm, np.full(len(lm), N, np.int32), cell)
    return oracle.psf(obs, oracle.IMG, b, flags=flags).reshape(len(lm), N, N)


def test_g1_transform_is_the_shifted_dft():
    """S = F{P} on the cutout's uv grid is numpy's FFT of the centred cutout, and P is
    the undistorted cutout at the phase centre (Eqs. 21-22 with D = 1)."""
    obs = obsgen.tiny_obs(weights=True)
    N, cell = 32, 2e-5
    g = oracle.grid_tables(obs, N, cell)
    b = obsgen.Batch(np.zeros((1, 2)), np.array([N], np.int32), cell)
    P0 = oracle.psf(obs, oracle.EXACT, b).reshape(N, N)
    np.testing.assert_allclose(g["P"], P0, rtol=0, atol=1e-10 * np.abs(P0).max())
    ref = np.fft.fftshift(np.fft.fft2(np.fft.ifftshift(g["P"])))
    np.testing.assert_allclose(g["S"], ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    # P real -> S Hermitian about the centre cell (N/2, N/2)
    mir = np.roll(np.flip(g["S"], (0, 1)), 1, (0, 1))
    np.testing.assert_allclose(mir, np.conj(g["S"]), rtol=0, atol=1e-12 * np.abs(ref).max())


def test_g2_phase_centre_gives_the_effective_psf():
    """Algorithm 1 at l0 = 0 gives D = 1 on every cell, so F^-1 F P = P."""
    obs = obsgen.tiny_obs(weights=True)
    N, cell = 32, 2e-5
    g = oracle.grid_tables(obs, N, cell)
    out = oracle.psf_img_grid(obs, [[0.0, 0.0]], N, cell)[0]
    np.testing.assert_allclose(out, g["P"], rtol=0, atol=1e-12 * np.abs(g["P"]).max())


@pytest.mark.parametrize("flags", [0, oracle.LITERAL_THETA])
def test_g3_visibilities_on_cell_centres_match_the_visibility_form(flags):
    """With every uv point on a cell centre and one dt and dnu/nu, the gridded form is
    the visibility-level Method 2 cutout exactly (both are sum_k W_k D(u_k) cos(...))."""
    N, cell = 16, 1e-4
    du = 1.0 / (N * cell)
    rng = np.random.default_rng(11)
    cells = [(int(a), int(b)) for a, b in zip(rng.integers(-7, 8, 7), rng.integers(-7, 8, 7))]
    cells.append((3, -5))
    cells.append((3, -5))                  # two visibilities in one cell
    obs = _obs(cells, du, weights=rng.uniform(0.5, 2.0, len(cells)))
    lm = [[0.05, -0.03], [-0.2, 0.1], [0.0, 0.3], [0.12, 0.12]]
    got = oracle.psf_img_grid(obs, lm, N, cell, flags=flags)
    ref = _dft_limit(obs, lm, N, cell, flags=flags)
    peak = float(obs.weights.astype(np.float64).sum())
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-10 * peak)
    # the distortion is far from negligible on these positions
    und = _dft_limit(obs, [[0.0, 0.0]], N, cell)[0]
    assert np.abs(ref - und[None]).max() > 0.2 * peak


def test_g4_points_outside_the_grid_wrap_modulo_n():
    """A uv point at (a + N) du is indistinguishable from a du on the pixel grid; the
    gridded form puts it in cell a and evaluates Algorithm 1 at that cell centre."""
    N, cell = 16, 1e-4
    du = 1.0 / (N * cell)
    inside = [(3, -2), (-5, 6)]
    outside = [(3 + N, -2), (-5, 6 - 2 * N)]
    w = [1.3, 0.7]
    lm = [[0.05, -0.08], [0.1, 0.02]]
    got = oracle.psf_img_grid(_obs(outside, du, width=5e6, weights=w), lm, N, cell)
    ref = _dft_limit(_obs(inside, du, width=5e6, weights=w), lm, N, cell)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-9 * sum(w))
    # the visibility form of the outside points differs: the wrap is a real effect
    far = _dft_limit(_obs(outside, du, width=5e6, weights=w), lm, N, cell)
    assert np.abs(far - ref).max() > 0.05 * sum(w)


def test_g5_cell_takes_the_weighted_mean_interval():
    """Baseline-dependent averaging: visibilities of dt and 2 dt (weights 1, 1, 2) in
    one cell act as weight 4 at the W-weighted mean interval 1.5 dt."""
    N, cell = 16, 1e-4
    du = 1.0 / (N * cell)
    dt = 40.0
    a = _obs([(4, 3), (4, 3)], du, ntime=2, dt=dt, tavg=[1, 2])      # bins: W 1, 1 (dt) and 2 (2 dt)
    b = _obs([(4, 3)], du, ntime=2, dt=1.5 * dt, tavg=[1], weights=[2.0, 2.0])
    lm = [[0.3, -0.25], [-0.4, 0.1]]
    got = oracle.psf_img_grid(a, lm, N, cell)
    ref = _dft_limit(b, lm, N, cell)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-10 * 4)
    g = oracle.grid_tables(a, N, cell)
    c = (3 + N // 2, 4 + N // 2)
    assert g["dt"][c] == pytest.approx(1.5 * dt, rel=1e-14)
    assert g["wsum"][c] == pytest.approx(4.0, rel=1e-14)


def test_g6_cell_tables_equal_brute_force_gridding():
    """Per-cell sums and means against a plain numpy gridding of the visibility table:
    nearest cell and its mirror, modulo N; empty cells hold the global means."""
    obs = obsgen.tiny_obs(weights=True)
    N, cell = 16, 3e-5
    g = oracle.grid_tables(obs, N, cell)
    vt = oracle.vis_table(obs)
    u, v = vt["uvw_lambda"][:, 0], vt["uvw_lambda"][:, 1]
    W, dt, r = vt["W"], vt["dt"], vt["dnu"] / vt["nu"]
    ia = np.floor(u * (N * cell) + 0.5).astype(np.int64)
    ib = np.floor(v * (N * cell) + 0.5).astype(np.int64)
    sw = np.zeros((N, N))
    sdt = np.zeros((N, N))
    sr = np.zeros((N, N))
    for sgn in (1, -1):
        bi = (sgn * ib + N // 2) % N
        ai = (sgn * ia + N // 2) % N
        np.add.at(sw, (bi, ai), W)
        np.add.at(sdt, (bi, ai), W * dt)
        np.add.at(sr, (bi, ai), W * r)
    full = sw > 0
    assert full.sum() > 10 and (~full).sum() > 10
    np.testing.assert_allclose(g["wsum"], sw, rtol=1e-12, atol=0)
    np.testing.assert_allclose(g["dt"][full], sdt[full] / sw[full], rtol=1e-12)
    np.testing.assert_allclose(g["r"][full], sr[full] / sw[full], rtol=1e-12)
    np.testing.assert_allclose(g["dt"][~full], (W * dt).sum() / W.sum(), rtol=1e-12)
    np.testing.assert_allclose(g["r"][~full], (W * r).sum() / W.sum(), rtol=1e-12)
    assert g["wsum"].sum() == pytest.approx(2 * W.sum(), rel=1e-12)


def test_g7_point_symmetric_positions_give_the_same_cutout():
    """Algorithm 1's D is even in l0 (sinc is even, the bandwidth term depends on |l0|),
    so positions l0 and -l0 give identical gridded cutouts."""
    obs = obsgen.tiny_obs(weights=True)
    out = oracle.psf_img_grid(obs, [[0.04, -0.07], [-0.04, 0.07]], 16, 3e-5)
    np.testing.assert_allclose(out[0], out[1], rtol=0, atol=1e-12 * np.abs(out[0]).max())
