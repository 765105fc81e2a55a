"""Pins of the FP64 oracle of Hogbom CLEAN with position-dependent PSFs (Algorithm 2).

Each test checks ``oracle.clean`` against a closed form that does not use its code:
an isolated source shaped like the PSF at its pixel decays geometrically by (1 - gain)
per iteration, the do-while runs its first iteration whatever the threshold, gain 1
removes such a source exactly, two isolated sources are taken in the order the two
geometric series predict, and a window clipped at the image edge behaves the same.
"""
import numpy as np
import pytest

import obsgen
import oracle

N, CELL, NL, NM = 16, 3e-5, 64, 48


def _psf_at(obs, method, x, y):
    l0, m0 = (x - NL // 2) * CELL, (y - NM // 2) * CELL
    if method == "img_grid":
        P = oracle.psf_img_grid(obs, [[l0, m0]], N, CELL)[0]
    else:
        b = obsgen.Batch(np.array([[l0, m0]]), np.array([N], np.int32), CELL)
        P = oracle.psf(obs, {"exact": oracle.EXACT, "uv": oracle.UV, "img": oracle.IMG}[method], b).reshape(N, N)
    return P / P[N // 2, N // 2]


def _place(img, P, x, y, c):
    y0, x0 = y - N // 2, x - N // 2
    ya, yb, xa, xb = max(y0, 0), min(y0 + N, img.shape[0]), max(x0, 0), min(x0 + N, img.shape[1])
    img[ya:yb, xa:xb] += c * P[ya - y0:yb - y0, xa - x0:xb - x0]


def _isolated(obs, method, x, y, c):
    P = _psf_at(obs, method, x, y)
    off = P.copy()
    off[N // 2, N // 2] = -np.inf
    assert off.max() < 0.95            # the normalised PSF peaks at its centre pixel
    d = np.zeros((NM, NL))
    _place(d, P, x, y, c)
    return d, P


@pytest.mark.parametrize("method", ["exact", "uv", "img", "img_grid"])
def test_c1_isolated_source_decays_geometrically(method):
    obs = obsgen.tiny_obs(weights=True)
    x, y, c, gain, thr = 40, 20, 2.0, 0.3, 0.05
    d, P = _isolated(obs, method, x, y, c)
    res, model, comps = oracle.clean(obs, method, d, CELL, N, gain, thr, 100)
    K = 1
    while c * (1 - gain) ** K > thr:
        K += 1
    assert len(comps) == K
    for k, (idx, g) in enumerate(comps):
        assert idx == y * NL + x
        assert g == pytest.approx(gain * c * (1 - gain) ** k, rel=1e-12)
    assert model[y, x] == pytest.approx(c * (1 - (1 - gain) ** K), rel=1e-12)
    ref = np.zeros_like(d)
    _place(ref, P, x, y, c * (1 - gain) ** K)
    np.testing.assert_allclose(res, ref, rtol=0, atol=1e-12)


def test_c2_first_iteration_always_runs():
    obs = obsgen.tiny_obs(weights=True)
    d, _ = _isolated(obs, "uv", 30, 25, 1.0)
    res, model, comps = oracle.clean(obs, "uv", d, CELL, N, 0.2, 10.0, 50)
    assert len(comps) == 1 and comps[0][1] == pytest.approx(0.2, rel=1e-12)


def test_c3_unit_gain_removes_the_source():
    obs = obsgen.tiny_obs(weights=True)
    d, _ = _isolated(obs, "img", 22, 30, 1.5)
    res, model, comps = oracle.clean(obs, "img", d, CELL, N, 1.0, 0.0, 50)
    assert len(comps) == 1 and model[30, 22] == pytest.approx(1.5, rel=1e-12)
    assert np.max(np.abs(res)) < 1e-12


def test_c4_two_sources_follow_the_geometric_series():
    """Windows that do not overlap: every iteration takes the larger remaining peak (the
    first pixel on ties), which the two series c_s (1 - gain)^k_s predict."""
    obs = obsgen.tiny_obs(weights=True)
    srcs = [(12, 10, 1.0), (45, 33, 0.83)]
    d = np.zeros((NM, NL))
    for x, y, c in srcs:
        _place(d, _psf_at(obs, "uv", x, y), x, y, c)
    gain, thr = 0.25, 0.05
    res, model, comps = oracle.clean(obs, "uv", d, CELL, N, gain, thr, 200)
    cur = [c for _, _, c in srcs]
    seq = []
    while True:
        s = 0 if (cur[0] > cur[1] or (cur[0] == cur[1] and srcs[0][1] * NL + srcs[0][0] < srcs[1][1] * NL + srcs[1][0])) \
            else 1
        if seq and not cur[s] > thr:
            break
        seq.append((srcs[s][1] * NL + srcs[s][0], gain * cur[s]))
        cur[s] *= 1 - gain
    assert [i for i, _ in comps] == [i for i, _ in seq]
    np.testing.assert_allclose([g for _, g in comps], [g for _, g in seq], rtol=1e-12)
    assert len({i for i, _ in comps}) == 2


def test_c5_window_clipped_at_the_image_edge():
    obs = obsgen.tiny_obs(weights=True)
    x, y, c, gain = 3, NM - 4, 1.0, 0.5
    d, P = _isolated(obs, "uv", x, y, c)
    res, model, comps = oracle.clean(obs, "uv", d, CELL, N, gain, 0.2, 100)
    assert [i for i, _ in comps] == [y * NL + x] * 3            # 0.5, 0.25, 0.125 <= 0.2
    ref = np.zeros_like(d)
    _place(ref, P, x, y, c * 0.125)
    np.testing.assert_allclose(res, ref, rtol=0, atol=1e-12)


def test_c6_facet_psf_closed_form():
    """One PSF at the image centre for every component (faceting, Eqs. 57-58): a source at
    the centre pixel is cleaned exactly as with position-dependent PSFs; an off-centre
    source, taken at its own pixel every time, leaves c P_src - c (1 - (1-gain)^K) P_centre
    (the centre PSF, not its own, is subtracted)."""
    obs = obsgen.tiny_obs(weights=True)
    centre = (0.01, 0.005)          # the normalised PSF peaks at its centre pixel here
    gain, thr = 0.3, 0.1
    xc, yc = NL // 2, NM // 2
    def psf_at(x, y):
        l0, m0 = centre[0] + (x - NL // 2) * CELL, centre[1] + (y - NM // 2) * CELL
        b = obsgen.Batch(np.array([[l0, m0]]), np.array([N], np.int32), CELL)
        P = oracle.psf(obs, oracle.UV, b).reshape(N, N)
        return P / P[N // 2, N // 2]
    Pc = psf_at(xc, yc)
    d = np.zeros((NM, NL))
    _place(d, Pc, xc, yc, 1.0)
    a = oracle.clean(obs, "uv", d, CELL, N, gain, thr, 100, centre=centre)
    b = oracle.clean(obs, "uv", d, CELL, N, gain, thr, 100, centre=centre, facet_psf=True)
    np.testing.assert_allclose(a[0], b[0], rtol=0, atol=1e-12)
    assert [i for i, _ in a[2]] == [i for i, _ in b[2]]
    x, y = xc + 9, yc - 6
    Ps = psf_at(x, y)
    d = np.zeros((NM, NL))
    _place(d, Ps, x, y, 1.0)
    res, model, comps = oracle.clean(obs, "uv", d, CELL, N, gain, thr, 100, centre=centre, facet_psf=True)
    K = len(comps)
    assert all(i == y * NL + x for i, _ in comps)
    np.testing.assert_allclose([g for _, g in comps], gain * (1 - gain) ** np.arange(K), rtol=1e-12)
    ref = np.zeros_like(d)
    _place(ref, Ps, x, y, 1.0)
    _place(ref, Pc, x, y, -(1 - (1 - gain) ** K))
    np.testing.assert_allclose(res, ref, rtol=0, atol=1e-12)
    assert np.max(np.abs(Ps - Pc)) > 1e-3          # the two PSFs do differ
