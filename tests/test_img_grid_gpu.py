"""GPU parity of psf_approx_img_grid (Method 2 in the gridded form of Eq. 45 with
Algorithm 1 on the cutout's uv grid) against the FP64 oracle.

Tolerances (max error over a cutout / its peak): the effective PSF comes from the
visibility-level path of the plan's precision (1e-6 of the peak in FP32, 1e-4 with FP16
tensor-core operands), and the per-position transform adds an FP32 inverse FFT
(2 log2 N^2 rounding steps of ~6e-8 on values bounded by sum |X| ~ the peak) and FP32
sinc arguments.  The taper is a convolution whose kernel has an l1 norm of a few, so the
bounds are 1e-5 (FP32 path) and 3e-4 (FP16 tensor-core path)."""
import functools

import numpy as np
import pytest

import obsgen
import oracle

pytestmark = pytest.mark.gpu
TOL = {"fp32": 1e-5, "tc_fp16": 3e-4}
ARCSEC = np.pi / 180 / 3600
OMEGA_E = 7.2921150e-5


@pytest.fixture(scope="module")
def psf():
    import paper_2009_07010_gb300 as m
    m.build_library()
    return m


def _rel(got, ref):
    return float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))


C1_LM = ((0.02, 0.02), (0.0, 0.0), (-0.05, 0.03), (0.1, -0.08), (0.2, 0.15))


@functools.lru_cache(maxsize=None)
def _c1_ref(flags):
    obs = obsgen.config1_obs()
    return oracle.psf_img_grid(obs, C1_LM, 64, 2.0 * ARCSEC, flags=flags)


@pytest.mark.parametrize("prec", ["fp32", "tc_fp16"])
@pytest.mark.parametrize("literal", [False, True])
def test_grid_config1_every_pixel(psf, prec, literal):
    """Workload 1 (16 antennas, 64 x 64 at 2"): five positions, every pixel against the
    oracle, both readings of theta."""
    flags = psf.PSF_IMG_LITERAL_THETA if literal else 0
    obs = obsgen.config1_obs()
    ref = _c1_ref(flags)
    with psf.Plan(obs, prec=prec, flags=flags) as plan:
        got = plan.approx_img_grid(psf.Batch(np.array(C1_LM), 64, 2.0 * ARCSEC))
        assert plan.sync_status() == 0
    got = got.cpu().numpy().astype(np.float64).reshape(len(C1_LM), 64, 64)
    errs = [_rel(got[p], ref[p]) for p in range(len(C1_LM))]
    assert max(errs) <= TOL[prec], errs


def test_grid_sizes_offsets_and_gaps(psf):
    """Cutouts of 16, 32, 64 and 128 pixels mixed in one batch, written at caller offsets
    with gaps between them (the gaps stay untouched)."""
    obs = obsgen.tiny_obs(weights=True)
    cell = 3e-5
    sizes = [32, 128, 16, 64, 32, 16, 128]
    lm = np.array([(0.03, -0.02), (0.05, 0.04), (-0.1, 0.02), (0.0, 0.07), (0.2, -0.1), (0.01, 0.0), (-0.04, -0.06)])
    offs, run = [], 7
    for n in sizes:
        offs.append(run)
        run += n * n + 13
    with psf.Plan(obs, prec="fp32") as plan:
        import torch
        out = torch.full((run,), float("nan"), dtype=torch.float32, device="cuda")
        plan.approx_img_grid(psf.Batch(lm, np.array(sizes), cell, out_offset=np.array(offs)), out=out)
        assert plan.sync_status() == 0
    got = out.cpu().numpy().astype(np.float64)
    written = np.zeros(run, bool)
    for p, n in enumerate(sizes):
        ref = oracle.psf_img_grid(obs, lm[p:p + 1], n, cell)[0].ravel()
        seg = got[offs[p]:offs[p] + n * n]
        assert _rel(seg, ref) <= TOL["fp32"], (p, n, _rel(seg, ref))
        written[offs[p]:offs[p] + n * n] = True
    assert np.all(np.isnan(got[~written]))


def test_grid_unsupported_and_empty(psf):
    obs = obsgen.tiny_obs()
    import torch
    out = torch.zeros(256 * 256, dtype=torch.float32, device="cuda")
    with psf.Plan(obs, prec="fp32") as plan:
        for n in (48, 256, 8):
            with pytest.raises(psf.PsfError) as e:
                plan.approx_img_grid(psf.Batch(np.zeros((1, 2)), n, 1e-5), out=out)
            assert e.value.status == psf.PSF_EUNSUPPORTED
        plan.approx_img_grid(psf.Batch(np.zeros((0, 2)), 64, 1e-5), out=out)
        assert plan.sync_status() == 0
        plan.set_opts(flags=psf.PSF_COMPLEX_OUT)
        with pytest.raises(psf.PsfError) as e:
            plan.approx_img_grid(psf.Batch(np.zeros((1, 2)), 64, 1e-5), out=out)
        assert e.value.status == psf.PSF_EUNSUPPORTED


def test_grid_tables_are_kept_and_rebuilt_per_precision(psf):
    """Repeated calls reuse the table (identical output); a precision change builds a new
    one whose output still meets its tolerance."""
    obs = obsgen.config1_obs()
    b = psf.Batch(np.array(C1_LM[:2]), 64, 2.0 * ARCSEC)
    ref = _c1_ref(0)[:2]
    with psf.Plan(obs, prec="tc_fp16") as plan:
        a1 = plan.approx_img_grid(b).cpu().numpy()
        a2 = plan.approx_img_grid(b).cpu().numpy()
        assert np.array_equal(a1, a2)
        plan.set_opts(prec="fp32")
        a3 = plan.approx_img_grid(b).cpu().numpy().astype(np.float64).reshape(2, 64, 64)
        assert plan.sync_status() == 0
    assert max(_rel(a3[p], ref[p]) for p in range(2)) <= TOL["fp32"]


def test_grid_cell_table_bda_full_size(psf):
    """Baseline-dependent averaging (64 antennas, 2 h, 8 channels, 2..30 s bins, 13.7 M
    visibilities): the device's per-cell mean interval and fractional bandwidth equal the
    oracle's on every cell; both take the nearest-cell decisions in FP64 in the same order,
    and a visibility put in another cell would move a cell mean far beyond FP32 rounding."""
    obs = obsgen.config3_obs()
    N, cell = 64, 1.5 * ARCSEC
    ref = oracle.grid_tables(obs, N, cell, cells_only=True)
    with psf.Plan(obs, prec="tc_fp16") as plan:
        t = plan.img_grid_table(N, cell).cpu().numpy().astype(np.float64)   # [b][a][4]
        assert plan.sync_status() == 0
    du = 1.0 / (N * cell)
    dt = t[:, :, 2] / (OMEGA_E * du)
    a = (np.arange(N) - N // 2) * du
    uabs = np.hypot(a[None, :], a[:, None])
    r = np.where(uabs > 0, t[:, :, 3] / np.where(uabs > 0, uabs, 1), ref["r"])
    assert (ref["wsum"] > 0).sum() > N * N // 4
    np.testing.assert_allclose(dt, ref["dt"], rtol=2e-6)
    np.testing.assert_allclose(r, ref["r"], rtol=2e-6)
    assert np.ptp(ref["dt"][ref["wsum"] > 0]) > 1.0                         # the means do vary


def test_grid_transform_of_effective_psf(psf):
    """The table's S is F{P} / N^2 of the device's own effective PSF (the Method 2 cutout
    at the phase centre): numpy's FFT of that cutout reproduces it."""
    obs = obsgen.config1_obs()
    N, cell = 64, 2.0 * ARCSEC
    with psf.Plan(obs, prec="fp32") as plan:
        P = plan.approx_img(psf.Batch(np.zeros((1, 2)), N, cell)).cpu().numpy().astype(np.float64).reshape(N, N)
        t = plan.img_grid_table(N, cell).cpu().numpy().astype(np.float64)
    S = t[:, :, 0] + 1j * t[:, :, 1]
    ref = np.fft.fftshift(np.fft.fft2(np.fft.ifftshift(P))) / N ** 2
    assert np.max(np.abs(S - ref)) <= 1e-6 * np.max(np.abs(ref))


def test_grid_meerkat_full_size_properties(psf):
    """MeerKAT-shaped 128 x 128 cutout at 1.5" (58 060 800 visibilities): at the phase
    centre the gridded form returns the effective PSF (the visibility-level Method 2 cutout
    there), and point-symmetric positions give the same cutout (Algorithm 1's D is even in
    l0).  The gap to the visibility-level Method 2 is the gridding error of Eq. 45."""
    obs = obsgen.config2_obs()
    N, cell = 128, 1.5 * ARCSEC
    lm = np.array([(0.0, 0.0), (0.03, 0.03), (-0.03, -0.03), (0.05, -0.02)])
    with psf.Plan(obs, prec="tc_fp16") as plan:
        g = plan.approx_img_grid(psf.Batch(lm, N, cell)).cpu().numpy().astype(np.float64).reshape(4, N, N)
        v = plan.approx_img(psf.Batch(lm, N, cell)).cpu().numpy().astype(np.float64).reshape(4, N, N)
        assert plan.sync_status() == 0
    assert _rel(g[0], v[0]) <= 1e-5
    assert _rel(g[1], g[2]) <= 1e-5
    gap = [_rel(g[p], v[p]) for p in (1, 3)]
    print("gridded vs visibility-level Method 2 (max err / peak):", gap)
    assert max(gap) < 0.2
