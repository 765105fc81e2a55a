"""GPU parity of psf_approx_uv_img (Methods 1 and 2 of one batch in one call) against
the FP64 oracle, and equality with the separate calls where it falls back to them.

The fused pass puts the real weights of both methods on the row twiddles and
computes both cutouts with one tensor-core contraction; its tolerances are those of
the separate tensor-core calls (FP16 operands: 1e-4 of each cutout's peak on the
workload-1 and MeerKAT-shaped observations; BF16: 1e-3)."""
import numpy as np
import pytest

import obsgen
import oracle

pytestmark = pytest.mark.gpu
TOL = {"tc_fp16": 1e-4, "tc_bf16": 1e-3}


@pytest.fixture(scope="module")
def psf():
    import paper_2009_07010_gb300 as m
    m.build_library()
    return m


def _err(got, ref, batch, offs, sel=None):
    errs = []
    for p in range(batch.npos):
        n2 = int(batch.npix[p]) ** 2
        if sel is None:
            g, r = got[offs[p]:offs[p] + n2], ref[offs[p]:offs[p] + n2]
        else:
            m = (sel >= offs[p]) & (sel < offs[p] + n2)
            g, r = got[sel[m]], ref[sel[m]]
        errs.append(np.max(np.abs(g - r)) / np.max(np.abs(r)))
    return np.array(errs)


@pytest.mark.parametrize("prec", ["tc_fp16", "tc_bf16"])
def test_fused_config1_full(psf, prec):
    """Workload 1 (64 x 64 cutout): every pixel of both outputs against the oracle."""
    obs, batch = obsgen.config1_obs(), obsgen.config1_batch()
    offs = obsgen.concat_pixels(batch)
    with psf.Plan(obs, prec=prec) as plan:
        uv, img = plan.approx_uv_img(psf.Batch.from_obsgen(batch))
        assert plan.sync_status() == 0
    for got, mid in ((uv, oracle.UV), (img, oracle.IMG)):
        ref = oracle.psf(obs, mid, batch)
        e = _err(got.cpu().numpy().astype(np.float64), ref, batch, offs)
        assert e.max() <= TOL[prec], (mid, e)


def test_fused_config2_sampled(psf):
    """MeerKAT-shaped 128 x 128 cutout (58 060 800 visibilities): sampled pixels."""
    obs, batch = obsgen.config2_obs(), obsgen.config2_batch()
    N = int(batch.npix[0])
    rng = np.random.default_rng(12)
    sel = np.array(sorted({N // 2 * N + N // 2, 0, N - 1, N * N - 1, N // 2 * N + 1,
                           *[int(x) for x in rng.choice(N * N, 10, replace=False)]}), np.int64)
    offs = obsgen.concat_pixels(batch)
    with psf.Plan(obs, prec="tc_fp16") as plan:
        uv, img = plan.approx_uv_img(psf.Batch.from_obsgen(batch))
        assert plan.sync_status() == 0
    for got, mid in ((uv, oracle.UV), (img, oracle.IMG)):
        ref = oracle.psf(obs, mid, batch, pix_sel=sel)
        e = _err(got.cpu().numpy().astype(np.float64), ref, batch, offs, sel)
        assert e.max() <= 1e-4, (mid, e)


def test_fused_mixed_sizes_offsets_gaps(psf):
    """64- and 128-pixel cutouts in one call with caller-given offsets and gaps: both
    outputs against the oracle at sampled pixels; the gaps keep their contents."""
    import torch
    obs = obsgen.config1_obs()
    rng = np.random.default_rng(4)
    npix = np.array([64, 128, 64, 128, 64], np.int32)
    lm = rng.uniform(-0.03, 0.03, size=(len(npix), 2))
    batch = obsgen.Batch(lm, npix, 2 * obsgen.ARCSEC)
    offs = np.zeros(len(npix), np.int64)
    pos = 5
    for i, n in enumerate(npix):
        offs[i] = pos
        pos += int(n) * int(n) + 3
    total = pos + 2
    sel = []
    for i, n in enumerate(npix):
        n = int(n)
        pix = {n // 2 * n + n // 2, 0, n * n - 1, *[int(x) for x in rng.choice(n * n, 6, replace=False)]}
        sel += [int(offs[i]) + x for x in sorted(pix)]
    sel = np.array(sel, np.int64)
    with psf.Plan(obs, prec="tc_fp16") as plan:
        outs = [torch.full((total,), 2.5, device="cuda") for _ in range(2)]
        plan.approx_uv_img(psf.Batch(lm, npix, batch.cell_rad, out_offset=offs), out_uv=outs[0], out_img=outs[1])
        assert plan.sync_status() == 0
    mask = np.ones(total, bool)
    for i, n in enumerate(npix):
        mask[offs[i]:offs[i] + int(n) ** 2] = False
    for got, mid in zip(outs, (oracle.UV, oracle.IMG)):
        g = got.cpu().numpy().astype(np.float64)
        assert np.all(g[mask] == 2.5)
        ref = oracle.psf(obs, mid, batch, pix_sel=sel, offsets=offs)
        assert _err(g, ref, batch, offs, sel).max() <= 1e-4, mid


@pytest.mark.parametrize("prec,npix", [("fp32", 64), ("tc_fp16", 96)])
def test_fallback_equals_separate_calls(psf, prec, npix):
    """FP32 precision and sizes other than 64/128 take the two separate calls:
    the outputs are bitwise those of psf_approx_uv and psf_approx_img."""
    obs = obsgen.config1_obs()
    batch = obsgen.Batch(np.array([[0.01, -0.02]]), np.array([npix], np.int32), 2 * obsgen.ARCSEC)
    with psf.Plan(obs, prec=prec) as plan:
        b = psf.Batch.from_obsgen(batch)
        uv, img = plan.approx_uv_img(b)
        uv1 = plan.approx_uv(b)
        img1 = plan.approx_img(b)
        assert plan.sync_status() == 0
    assert torch_equal(uv, uv1) and torch_equal(img, img1)


def torch_equal(a, b):
    import torch
    return bool(torch.equal(a, b))


def test_fused_rejects_null_outputs(psf):
    import ctypes
    from paper_2009_07010_gb300 import _lib
    obs = obsgen.config1_obs()
    with psf.Plan(obs, prec="tc_fp16") as plan:
        bs = psf.Batch.from_obsgen(obsgen.config1_batch()).struct()
        assert _lib.lib().psf_approx_uv_img(plan._h, ctypes.byref(bs), None, None, None) == _lib.PSF_EINVAL
