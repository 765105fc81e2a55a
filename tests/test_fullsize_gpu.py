"""GPU parity of the kernel paths the configuration workloads take at full size, against
the FP64 oracle on sampled pixels (the oracle evaluates each selected pixel over every
visibility).

* the batched (Khatri-Rao) kernel on groups of 32^2, 64^2, 128^2 and 256^2 cutouts (32
  positions each) on the baseline-dependent-averaging observation of the batched-positions
  workload (13.7 M visibilities), and all four sizes in one persistent launch;
* one 256 x 256 cutout through the per-cutout tensor-core kernel (two 128-row tiles of 256
  columns each);
* the benchmark's fused call (Methods 1 and 2 in one pass, psf_approx_uv_img) on the
  MeerKAT 128 x 128 cutout (58 M visibilities): one full row and one full column.

Tolerance: err_max <= 1e-4 of each cutout's sampled peak (FP16 operands, FP32
accumulation); the centre pixel (the peak) is always sampled.
"""
import numpy as np
import pytest

import obsgen
import oracle

pytestmark = pytest.mark.gpu
METHODS = [("exact", oracle.EXACT), ("uv", oracle.UV), ("img", oracle.IMG)]


@pytest.fixture(scope="module")
def psf():
    import paper_2009_07010_gb300 as m
    m.build_library()
    return m


def _pixels(N, nrand, seed):
    """Centre pixel, the centre row and column ends, and random pixels (row-major)."""
    rng = np.random.default_rng(seed)
    c = N // 2
    pix = {c * N + c, c * N, c * N + N - 1, c, (N - 1) * N + c, 0, N * N - 1}
    pix.update(int(x) for x in rng.choice(N * N, nrand, replace=False))
    return np.array(sorted(pix), np.int64)


@pytest.mark.parametrize("N", [32, 64, 128, 256])
def test_batched_group_c3_observation(psf, N):
    """32 positions of one size within 1 degree: one 128-position tile of the batched
    kernel with N^2 / 256 pixel tiles each.  Eight of the positions are checked."""
    obs = obsgen.config3_obs()
    rng = np.random.default_rng(obsgen.SEED_BASE + 30 + N)
    s = np.sin(np.radians(1.0))
    lm = rng.uniform(-s, s, size=(32, 2))
    cell = 1.5 * obsgen.ARCSEC
    batch = obsgen.Batch(lm, np.full(32, N, np.int32), cell)
    check = np.array([0, 5, 11, 17, 23, 26, 30, 31])
    pix = _pixels(N, 6, N)
    sub = obsgen.Batch(lm[check], np.full(len(check), N, np.int32), cell)
    sub_sel = np.concatenate([q * N * N + pix for q in range(len(check))])
    with psf.Plan(obs, prec="tc_fp16") as plan:
        b = psf.Batch.from_obsgen(batch)
        for name, mid in METHODS:
            got = plan.forward(name, b).cpu().numpy().astype(np.float64).reshape(32, N * N)
            ref = oracle.psf(obs, mid, sub, pix_sel=sub_sel).reshape(len(check), N * N)
            for q, p in enumerate(check):
                g, r = got[p, pix], ref[q, pix]
                e = np.max(np.abs(g - r)) / np.max(np.abs(r))
                assert e <= 1e-4, (name, N, p, e)
        assert plan.sync_status() == 0


@pytest.mark.parametrize("prec,tol", [("tc_fp16", 1e-4), ("tc_bf16", 1e-3)])
def test_per_cutout_256px(psf, prec, tol):
    """One 256 x 256 cutout on the per-cutout tensor-core kernel (workload-1 observation,
    172 800 visibilities), all three methods: the centre row and column in full plus
    random pixels."""
    obs = obsgen.config1_obs()
    N = 256
    batch = obsgen.Batch(np.array([[-0.021, 0.017]]), np.array([N], np.int32), 2 * obsgen.ARCSEC)
    c = N // 2
    pix = np.array(sorted(set(list(c * N + np.arange(N)) + list(np.arange(N) * N + c))
                          | set(int(x) for x in _pixels(N, 64, 3))), np.int64)
    with psf.Plan(obs, prec=prec, algo=psf.PSF_ALGO_CUTOUT) as plan:
        b = psf.Batch.from_obsgen(batch)
        for name, mid in METHODS:
            got = plan.forward(name, b).cpu().numpy().astype(np.float64)
            ref = oracle.psf(obs, mid, batch, pix_sel=pix)
            e = np.max(np.abs(got[pix] - ref[pix])) / np.max(np.abs(ref[pix]))
            assert e <= tol, (name, e)
        assert plan.sync_status() == 0


def test_config2_fused_uv_img_row_and_column(psf):
    """The benchmark step's psf_approx_uv_img on the MeerKAT-shaped 128 x 128 cutout:
    the centre row and the centre column of both outputs (255 pixels each)."""
    obs = obsgen.config2_obs()
    batch = obsgen.config2_batch()
    N = int(batch.npix[0])
    c = N // 2
    pix = np.array(sorted(set(list(c * N + np.arange(N)) + list(np.arange(N) * N + c))), np.int64)
    with psf.Plan(obs, prec="tc_fp16") as plan:
        guv, gimg = plan.approx_uv_img(psf.Batch.from_obsgen(batch))
        guv = guv.cpu().numpy().astype(np.float64)
        gimg = gimg.cpu().numpy().astype(np.float64)
        assert plan.sync_status() == 0
    for got, mid in ((guv, oracle.UV), (gimg, oracle.IMG)):
        ref = oracle.psf(obs, mid, batch, pix_sel=pix)
        e = np.max(np.abs(got[pix] - ref[pix])) / np.max(np.abs(ref[pix]))
        assert e <= 1e-4, (mid, e)


def test_batched_all_sizes_one_launch(psf):
    """The batched-positions workload's mix: 40 positions of each size 32..256 in one call
    (one persistent launch per visibility chunk pulls the items of every size group);
    three positions per size checked on sampled pixels, all three methods."""
    obs = obsgen.config3_obs()
    rng = np.random.default_rng(obsgen.SEED_BASE + 77)
    s = np.sin(np.radians(1.0))
    npix = np.repeat(np.array([32, 64, 128, 256], np.int32), 40)
    rng.shuffle(npix)
    lm = rng.uniform(-s, s, size=(npix.size, 2))
    cell = 1.5 * obsgen.ARCSEC
    batch = obsgen.Batch(lm, npix, cell)
    check = np.concatenate([np.nonzero(npix == N)[0][:3] for N in (32, 64, 128, 256)])
    sub = obsgen.Batch(lm[check], npix[check], cell)
    offs = obsgen.concat_pixels(batch)
    soffs = obsgen.concat_pixels(sub)
    pix = {int(p): _pixels(int(npix[p]), 5, int(p)) for p in check}
    sub_sel = np.concatenate([soffs[q] + pix[int(p)] for q, p in enumerate(check)])
    with psf.Plan(obs, prec="tc_fp16") as plan:
        b = psf.Batch.from_obsgen(batch)
        for name, mid in METHODS:
            got = plan.forward(name, b).cpu().numpy().astype(np.float64)
            ref = oracle.psf(obs, mid, sub, pix_sel=sub_sel)
            for q, p in enumerate(check):
                g, r = got[offs[p] + pix[int(p)]], ref[soffs[q] + pix[int(p)]]
                e = np.max(np.abs(g - r)) / np.max(np.abs(r))
                assert e <= 1e-4, (name, int(npix[p]), int(p), e)
        assert plan.sync_status() == 0
