"""GPU tests of the option flags PSF_COMPLEX_OUT and PSF_DETERMINISTIC.

Complex cutouts hold the N^2 real parts and then the N^2 imaginary parts of the sum
of Eqs. 21-22; both halves are compared with the FP64 oracle (imaginary part:
oracle.psf(..., imag=True)), peak-normalised by the real cutout's peak, with the
tolerances of the tensor-core path (FP16 1e-4, BF16 1e-3 on the workload-1 and
MeerKAT-shaped observations)."""
import numpy as np
import pytest

import obsgen
import oracle

pytestmark = pytest.mark.gpu
METHODS = [("exact", oracle.EXACT), ("uv", oracle.UV), ("img", oracle.IMG)]
TOL = {"tc_fp16": 1e-4, "tc_bf16": 1e-3}


@pytest.fixture(scope="module")
def psf():
    import paper_2009_07010_gb300 as m
    m.build_library()
    return m


def _cplx_err(got, ref_re, ref_im, N, off, goff, sel=None):
    """Errors of the real and imaginary halves of one complex cutout at got[goff:]."""
    n2 = N * N
    re, im = got[goff:goff + n2], got[goff + n2:goff + 2 * n2]
    rr, ri = ref_re[off:off + n2], ref_im[off:off + n2]
    if sel is not None:
        re, im, rr, ri = re[sel], im[sel], rr[sel], ri[sel]
    peak = np.max(np.abs(rr))
    return np.max(np.abs(re - rr)) / peak, np.max(np.abs(im - ri)) / peak


@pytest.mark.parametrize("prec", ["tc_fp16", "tc_bf16"])
def test_complex_config1_full(psf, prec):
    """Workload 1 (64 x 64): every pixel of both halves for the three methods; the
    imaginary part is not small (half of a Hermitian pair), so both halves are tested."""
    obs, batch = obsgen.config1_obs(), obsgen.config1_batch()
    with psf.Plan(obs, prec=prec, flags=psf.PSF_COMPLEX_OUT) as plan:
        b = psf.Batch.from_obsgen(batch)
        for name, mid in METHODS:
            got = plan.forward(name, b).cpu().numpy().astype(np.float64)
            assert got.size >= 2 * 64 * 64
            ref_re = oracle.psf(obs, mid, batch)
            ref_im = oracle.psf(obs, mid, batch, imag=True)
            assert np.max(np.abs(ref_im)) > 1e-2 * np.max(np.abs(ref_re))
            e_re, e_im = _cplx_err(got, ref_re, ref_im, 64, 0, 0)
            assert e_re <= TOL[prec] and e_im <= TOL[prec], (name, e_re, e_im)
        assert plan.sync_status() == 0


def test_complex_config2_sampled(psf):
    """MeerKAT-shaped 128 x 128 cutout (the 256-row doubled B operand), sampled pixels."""
    obs, batch = obsgen.config2_obs(), obsgen.config2_batch()
    N = 128
    rng = np.random.default_rng(21)
    sel = np.array(sorted({N // 2 * N + N // 2, 0, N - 1, N * N - 1,
                           *[int(x) for x in rng.choice(N * N, 8, replace=False)]}), np.int64)
    with psf.Plan(obs, prec="tc_fp16", flags=psf.PSF_COMPLEX_OUT) as plan:
        got = plan.exact(psf.Batch.from_obsgen(batch)).cpu().numpy().astype(np.float64)
        assert plan.sync_status() == 0
    ref_re = oracle.psf(obs, oracle.EXACT, batch, pix_sel=sel)
    ref_im = oracle.psf(obs, oracle.EXACT, batch, pix_sel=sel, imag=True)
    e_re, e_im = _cplx_err(got, ref_re, ref_im, N, 0, 0, sel)
    assert e_re <= 1e-4 and e_im <= 1e-4, (e_re, e_im)


def test_complex_ragged_sizes_offsets_and_gaps(psf):
    """Cutouts of 2, 66 and 128 pixels with caller-given offsets and gaps (2 N^2 floats
    each): both halves against the oracle, gaps untouched, the real half equal to the
    plain call's output within the tolerance."""
    import torch
    obs = obsgen.config1_obs()
    npix = np.array([66, 2, 128], np.int32)
    lm = np.array([[0.01, 0.02], [-0.03, 0.01], [0.02, -0.015]])
    cell = 2 * obsgen.ARCSEC
    offs = np.array([3, 3 + 2 * 66 * 66 + 5, 3 + 2 * 66 * 66 + 5 + 8 + 7], np.int64)
    total = int(offs[-1] + 2 * 128 * 128 + 4)
    batch = obsgen.Batch(lm, npix, cell)
    with psf.Plan(obs, prec="tc_fp16", flags=psf.PSF_COMPLEX_OUT) as plan:
        out = torch.full((total,), 7.0, device="cuda")
        plan.exact(psf.Batch(lm, npix, cell, out_offset=offs), out=out)
        plan.set_opts(flags=0)
        plain = plan.exact(psf.Batch.from_obsgen(batch)).cpu().numpy().astype(np.float64)
        assert plan.sync_status() == 0
    got = out.cpu().numpy().astype(np.float64)
    mask = np.ones(total, bool)
    for o, n in zip(offs, npix):
        mask[o:o + 2 * int(n) ** 2] = False
    assert np.all(got[mask] == 7.0)
    ref_re = oracle.psf(obs, oracle.EXACT, batch)
    ref_im = oracle.psf(obs, oracle.EXACT, batch, imag=True)
    poff = obsgen.concat_pixels(batch)
    for p, n in enumerate(npix):
        n = int(n)
        e_re, e_im = _cplx_err(got, ref_re, ref_im, n, int(poff[p]), int(offs[p]))
        tol = 1e-4 if n > 2 else 2e-3   # a 2 x 2 cutout holds few pixels near the peak
        assert e_re <= tol and e_im <= tol, (n, e_re, e_im)
        re = got[offs[p]:offs[p] + n * n]
        pl = plain[poff[p]:poff[p] + n * n]
        assert np.max(np.abs(re - pl)) <= 1e-4 * np.max(np.abs(pl))


def test_complex_unsupported_requests(psf):
    obs = obsgen.config1_obs()
    b = psf.Batch(np.array([[0.01, 0.01]]), np.array([256], np.int32), 2 * obsgen.ARCSEC)
    with psf.Plan(obs, prec="tc_fp16", flags=psf.PSF_COMPLEX_OUT) as plan:
        with pytest.raises(psf.PsfError) as ei:          # tensor-core complex cutouts stop at 128
            plan.exact(b)
        assert ei.value.status == -4
        plan.set_opts(prec="fp32")
        with pytest.raises(psf.PsfError) as ei:          # no FP32 complex form
            plan.exact(psf.Batch.from_obsgen(obsgen.config1_batch()))
        assert ei.value.status == -4


def test_complex_fused_call_falls_back_to_complex_calls(psf):
    """psf_approx_uv_img with PSF_COMPLEX_OUT: the two separate complex calls."""
    import torch
    obs = obsgen.config1_obs()
    with psf.Plan(obs, prec="tc_fp16", flags=psf.PSF_COMPLEX_OUT) as plan:
        b = psf.Batch.from_obsgen(obsgen.config1_batch())
        uv, img = plan.approx_uv_img(b)
        uv1, img1 = plan.approx_uv(b), plan.approx_img(b)
        assert plan.sync_status() == 0
    assert torch.equal(uv, uv1) and torch.equal(img, img1)


def test_deterministic_flag(psf):
    """PSF_DETERMINISTIC: a group of 40 cutouts of 32^2 (large enough for the batched
    form, whose atomics add the visibility splits in arrival order) takes the
    per-cutout form; two calls are bitwise identical and within 1e-4 of the oracle."""
    import torch
    obs = obsgen.config1_obs()
    rng = np.random.default_rng(8)
    npix = np.full(40, 32, np.int32)
    lm = rng.uniform(-0.03, 0.03, size=(40, 2))
    batch = obsgen.Batch(lm, npix, 2 * obsgen.ARCSEC)
    offs = obsgen.concat_pixels(batch)
    sel = np.array(sorted({int(o) + 16 * 32 + 16 for o in offs} |
                          {int(x) for x in rng.choice(int(offs[-1]) + 1024, 60, replace=False)}), np.int64)
    with psf.Plan(obs, prec="tc_fp16", flags=psf.PSF_DETERMINISTIC) as plan:
        b = psf.Batch.from_obsgen(batch)
        for name, mid in METHODS:
            a1 = plan.forward(name, b).clone()
            a2 = plan.forward(name, b)
            assert torch.equal(a1, a2), name
            got = a2.cpu().numpy().astype(np.float64)
            ref = oracle.psf(obs, mid, batch, pix_sel=sel)
            for p in range(batch.npos):
                m = (sel >= offs[p]) & (sel < offs[p] + 1024)
                e = np.max(np.abs(got[sel[m]] - ref[sel[m]])) / np.max(np.abs(ref[sel[m]]))
                assert e <= 1e-4, (name, p, e)
        assert plan.sync_status() == 0
