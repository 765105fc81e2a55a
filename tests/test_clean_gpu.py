"""GPU parity of psf_clean (Hogbom CLEAN with position-dependent PSFs, Algorithm 2)
against the FP64 oracle.

CLEAN's argmax decides the rest of the run, and on broad PSF main lobes the residual
often has near-ties (pixels within 1e-6 of the peak), where float32 and float64 may
pick different pixels and both be correct.  So each side builds its dirty image from
its own PSFs (same seeded source list), the device runs the loop, and the oracle then
replays the device's choices (``oracle.clean(..., follow=...)``): every choice must be
an argmax of the oracle's residual within the tolerance, every flux and the final
residual and model must match, and the stopping decision must agree within the
tolerance.  Tolerance 2e-5 of the brightest source: the FP32 PSFs are within 1e-6 of
the oracle's (1e-5 for the gridded form), and float32 subtraction over a few hundred
iterations adds ~1e-6."""
import numpy as np
import pytest

import obsgen
import oracle

pytestmark = pytest.mark.gpu
ARC = np.pi / 180 / 3600
TOL = 2e-5


@pytest.fixture(scope="module")
def psf():
    import paper_2009_07010_gb300 as m
    m.build_library()
    return m


def _place(img, P, x, y, c):
    N = P.shape[0]
    y0, x0 = y - N // 2, x - N // 2
    ya, yb, xa, xb = max(y0, 0), min(y0 + N, img.shape[0]), max(x0, 0), min(x0 + N, img.shape[1])
    img[ya:yb, xa:xb] += c * P[ya - y0:yb - y0, xa - x0:xb - x0]


def _oracle_psf(obs, method, l0, m0, N, cell):
    if method == "img_grid":
        P = oracle.psf_img_grid(obs, [[l0, m0]], N, cell)[0]
    else:
        b = obsgen.Batch(np.array([[l0, m0]]), np.array([N], np.int32), cell)
        P = oracle.psf(obs, {"exact": oracle.EXACT, "uv": oracle.UV, "img": oracle.IMG}[method], b).reshape(N, N)
    return P / P[N // 2, N // 2]


def _device_psf(psf, plan, method, l0, m0, N, cell):
    b = psf.Batch(np.array([[l0, m0]]), N, cell)
    out = plan.approx_img_grid(b) if method == "img_grid" else plan.forward(method, b)
    P = out[:N * N].cpu().numpy().astype(np.float64).reshape(N, N)
    return P / P[N // 2, N // 2]


def _run(psf, obs, plan, method, nl, nm, cell, centre, N, srcs, gain, thr, maxit, facet_psf=False):
    import torch
    dg, do = np.zeros((nm, nl)), np.zeros((nm, nl))
    for x, y, c in srcs:
        l0, m0 = centre[0] + (x - nl // 2) * cell, centre[1] + (y - nm // 2) * cell
        _place(dg, _device_psf(psf, plan, method, l0, m0, N, cell), x, y, c)
        _place(do, _oracle_psf(obs, method, l0, m0, N, cell), x, y, c)
    dirty = torch.tensor(dg, dtype=torch.float32, device="cuda")
    res, model, cpix, cflux = plan.clean(dirty, cell, N, method=method, gain=gain, threshold=thr, max_iter=maxit,
                                         centre=centre, facet_psf=facet_psf)
    assert plan.sync_status() == 0
    cpix, cflux = cpix.cpu().numpy(), cflux.cpu().numpy().astype(np.float64)
    res, model = res.cpu().numpy().astype(np.float64), model.cpu().numpy().astype(np.float64)
    ro, mo, comps, trace = oracle.clean(obs, method, do, cell, N, gain, thr, maxit, centre=centre, follow=cpix,
                                        facet_psf=facet_psf)
    scale = max(c for _, _, c in srcs)
    for k, (mx, val) in enumerate(trace):
        assert mx - val <= TOL * scale, (k, mx, val)
        if k > 0:
            assert val > thr - TOL * scale
    if len(cpix) < maxit:
        assert np.max(ro) <= thr + TOL * scale
    np.testing.assert_allclose(cflux, [g for _, g in comps], rtol=0, atol=TOL * scale)
    np.testing.assert_allclose(res, ro, rtol=0, atol=TOL * scale)
    np.testing.assert_allclose(model, mo, rtol=0, atol=TOL * scale)
    return len(cpix)


@pytest.mark.parametrize("method", ["exact", "uv", "img", "img_grid"])
def test_clean_overlapping_sources(psf, method):
    """Workload 1 (16 antennas, 1 km), a 96 x 96 image at 2" centred on (0.02, 0.02), three
    sources whose 32 x 32 PSF windows overlap, gain 0.25, threshold 0.15."""
    obs = obsgen.config1_obs()
    with psf.Plan(obs, prec="fp32") as plan:
        n = _run(psf, obs, plan, method, 96, 96, 2 * ARC, (0.02, 0.02), 32,
                 [(40, 50, 1.0), (52, 44, 0.8), (30, 35, 0.65)], 0.25, 0.15, 60)
    assert n > 10


@pytest.mark.parametrize("method", ["exact", "img_grid"])
def test_clean_facet_psf(psf, method):
    """One PSF at the image centre for every component (faceting): the same sources as
    above, so the subtracted shape differs from each source's own PSF."""
    obs = obsgen.config1_obs()
    with psf.Plan(obs, prec="fp32") as plan:
        n = _run(psf, obs, plan, method, 96, 96, 2 * ARC, (0.02, 0.02), 32,
                 [(40, 50, 1.0), (52, 44, 0.8), (30, 35, 0.65)], 0.25, 0.15, 60, facet_psf=True)
    assert n > 10


def test_clean_gridded_long_run(psf):
    """Workload 1, a 128 x 96 image at 2" centred on (0.02, 0.02), six sources, gain 0.1,
    no threshold, capped at 400 iterations: the device-resident loop of the gridded PSF
    runs several queued chunks of 64 and stops at the cap."""
    obs = obsgen.config1_obs()
    srcs = [(20, 20, 1.0), (60, 24, 0.87), (100, 18, 0.76), (28, 68, 0.69), (72, 76, 0.58), (110, 60, 0.51)]
    with psf.Plan(obs, prec="fp32") as plan:
        n = _run(psf, obs, plan, "img_grid", 128, 96, 2 * ARC, (0.02, 0.02), 32, srcs, 0.1, 0.0, 400)
    assert n == 400


def test_clean_threshold_stop_and_caps(psf):
    """The gridded loop stops on the threshold inside a chunk; max_iter caps the count;
    max_iter = 0 leaves the image untouched."""
    import torch
    obs = obsgen.config1_obs()
    srcs = [(20, 20, 1.0), (60, 40, 0.7)]
    with psf.Plan(obs, prec="fp32") as plan:
        n = _run(psf, obs, plan, "img_grid", 128, 96, 2 * ARC, (0.02, 0.02), 32, srcs, 0.3, 0.05, 500)
        assert 1 < n < 64
        d = torch.zeros((48, 64), dtype=torch.float32, device="cuda")
        d[20, 20] = 1.0
        r, m, cp, cf = plan.clean(d.clone(), 3e-5, 16, method="uv", gain=0.5, threshold=0.0, max_iter=3)
        assert len(cp) == 3
        d2 = d.clone()
        r, m, cp, cf = plan.clean(d2, 3e-5, 16, method="img_grid", gain=0.5, max_iter=0)
        assert len(cp) == 0 and torch.equal(r, d) and float(m.abs().max()) == 0.0


def test_clean_errors(psf):
    import torch
    obs = obsgen.tiny_obs()
    d = torch.zeros((48, 64), dtype=torch.float32, device="cuda")
    with psf.Plan(obs, prec="fp32") as plan:
        for kw, st in ((dict(gain=0.0), psf.PSF_EINVAL), (dict(gain=1.5), psf.PSF_EINVAL),
                       (dict(npix=15), psf.PSF_EINVAL), (dict(npix=48, method="img_grid"), psf.PSF_EUNSUPPORTED)):
            args = dict(cell=3e-5, npix=16, method="uv", gain=0.1, max_iter=5)
            args.update(kw)
            with pytest.raises(psf.PsfError) as e:
                plan.clean(d, args["cell"], args["npix"], method=args["method"], gain=args["gain"],
                           max_iter=args["max_iter"])
            assert e.value.status == st
        with pytest.raises(psf.PsfError) as e:
            plan.clean(torch.zeros((48, 63), dtype=torch.float32, device="cuda"), 3e-5, 16)
        assert e.value.status == psf.PSF_EINVAL


def test_clean_meerkat_full_size_isolated_source(psf):
    """MeerKAT-shaped observation (58 060 800 visibilities), a 1024 x 1024 image at 1.5"
    centred on (0.03, 0.03), one source shaped like the device's own 128 x 128 PSF at its
    pixel: every method's loop removes gain (1 - gain)^k of it per iteration (closed form),
    the gridded one until the threshold, the visibility-level ones for three iterations."""
    import torch
    obs = obsgen.config2_obs()
    nl = nm = 1024
    cell, centre, N, x, y = 1.5 * ARC, (0.03, 0.03), 128, 600, 400
    l0, m0 = centre[0] + (x - nl // 2) * cell, centre[1] + (y - nm // 2) * cell
    with psf.Plan(obs, prec="tc_fp16") as plan:
        for method, gain, thr, maxit in (("img_grid", 0.2, 0.01, 100), ("exact", 0.3, 0.0, 3), ("uv", 0.3, 0.0, 3),
                                         ("img", 0.3, 0.0, 3)):
            P = _device_psf(psf, plan, method, l0, m0, N, cell)
            off = P.copy()
            off[N // 2, N // 2] = -np.inf
            assert off.max() < 1.0
            d = np.zeros((nm, nl))
            _place(d, P, x, y, 1.0)
            dirty = torch.tensor(d, dtype=torch.float32, device="cuda")
            r, m, cp, cf = plan.clean(dirty, cell, N, method=method, gain=gain, threshold=thr, max_iter=maxit,
                                      centre=centre)
            assert plan.sync_status() == 0
            K = len(cp)
            if method == "img_grid":
                assert K == int(np.ceil(np.log(thr) / np.log(1 - gain)))
            else:
                assert K == maxit
            assert np.all(cp.cpu().numpy() == y * nl + x)
            np.testing.assert_allclose(cf.cpu().numpy(), gain * (1 - gain) ** np.arange(K), rtol=0, atol=1e-5)
            ref = np.zeros((nm, nl))
            _place(ref, P, x, y, (1 - gain) ** K)
            assert np.max(np.abs(r.cpu().numpy() - ref)) < 1e-5
