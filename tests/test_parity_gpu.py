"""GPU parity: the CUDA library against the FP64 oracle, element by element.

Error metric: err_max = max |P - P_ref| / max |P_ref| per cutout (peak-normalised;
pointwise relative error is undefined at PSF nulls).  Tolerances:
  * the FP32 path: 1e-6 everywhere, including few-visibility edge cases (its pixel
    phases are formed in float-float from the float64 bin centres, so a term carries
    ~1e-7 of error however large its phase);
  * tensor-core path: 1e-4 on the configuration workloads with FP16 operands; BF16
    single-pass operands 1e-3 (2^-8 unit roundoff averaged over the sum); the split
    precision modes (hi + lo operands, three MMA passes) 2e-5 everywhere;
  * tensor-core few-visibility edge cases (tens of terms): the sum has too few terms
    for rounding errors to average out, so the bound is the per-term error: a few
    FP16 (BF16) unit roundoffs, 2^-11 (2^-8) -> 2e-3 (1.6e-2).
"""
import numpy as np
import pytest

import obsgen
import oracle

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-6, "tc_fp16": 1e-4, "tc_bf16": 1e-3, "tc_fp16x3": 2e-5, "tc_bf16x3": 2e-5}
TOL_SMALL = {"fp32": 1e-6, "tc_fp16": 2e-3, "tc_bf16": 1.6e-2, "tc_fp16x3": 2e-5, "tc_bf16x3": 2e-5}
METHODS = [("exact", oracle.EXACT), ("uv", oracle.UV), ("img", oracle.IMG)]


@pytest.fixture(scope="module")
def psf():
    import paper_2009_07010_gb300 as m
    m.build_library()
    return m


def small_tol(prec, obs, batch):
    return TOL_SMALL[prec]


def err_per_cutout(got, ref, batch):
    errs = []
    offs = obsgen.concat_pixels(batch)
    for p in range(batch.npos):
        n2 = int(batch.npix[p]) ** 2
        g, r = got[offs[p]:offs[p] + n2], ref[offs[p]:offs[p] + n2]
        errs.append(np.max(np.abs(g - r)) / np.max(np.abs(r)))
    return np.array(errs)


# ------------------------------------------------------------------ tcgen05 layout
@pytest.mark.parametrize("n", [16, 64, 128, 256])
def test_umma_selftest_matches_matmul(psf, n):
    import torch
    g = torch.Generator(device="cpu").manual_seed(n)
    a = torch.randn(128, 64, generator=g).half().cuda()
    b = torch.randn(n, 64, generator=g).half().cuda()
    d = psf.selftest_umma(a, b)
    ref = a.float() @ b.float().T
    torch.testing.assert_close(d, ref, rtol=1e-5, atol=1e-4)


def test_fma_rate_probe_is_physical(psf):
    """The FP32 roofline's denominator: positive and below the lane count x 2 flops x a
    2.5 GHz clock (x2 for packed pairs, which may issue two FMAs per lane)."""
    import torch
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    bound = nsm * 128 * 2 * 2.5e9
    s, p = psf.fma_rate(False), psf.fma_rate(True)
    assert 0.25 * bound < s < bound, s
    assert 0.25 * bound < p < 2 * bound, p


# ------------------------------------------------------------------ workload 1 (full)
@pytest.fixture(scope="module")
def c1():
    obs = obsgen.config1_obs()
    batch = obsgen.config1_batch()
    refs = {name: oracle.psf(obs, mid, batch) for name, mid in METHODS}
    return obs, batch, refs


@pytest.mark.parametrize("prec", ["fp32", "tc_fp16", "tc_bf16", "tc_fp16x3", "tc_bf16x3"])
@pytest.mark.parametrize("method", ["exact", "uv", "img"])
def test_config1_full_parity(psf, c1, prec, method):
    obs, batch, refs = c1
    with psf.Plan(obs, prec=prec) as plan:
        b = psf.Batch.from_obsgen(batch)
        got = plan.forward(method, b).cpu().numpy().astype(np.float64)
        assert plan.sync_status() == 0
    e = err_per_cutout(got, refs[method], batch)
    assert e.max() <= TOL[prec], e


# ------------------------------------------------------------------ edge cases
def _edge_obs(kind):
    if kind == "bda_uniform_channels":
        return obsgen.tiny_obs(nant=5, ntime=40, nchan=8, tavg=[1, 2, 3, 5, 7, 8, 10, 13, 20, 40], favg=4,
                               weights=True)
    if kind == "unequal_channels":
        o = obsgen.tiny_obs(nant=4, ntime=30, nchan=6, tavg=6, favg=3)
        o.chan_width_hz = np.array([1e6, 3e6, 2e6, 2e6, 2e6, 1e6])
        edges = 1.2e9 + np.concatenate([[0], np.cumsum(o.chan_width_hz)])
        o.freq_hz = 0.5 * (edges[:-1] + edges[1:])
        return o
    if kind == "single_sample_bins":
        return obsgen.tiny_obs(nant=4, ntime=9, nchan=2, tavg=1, favg=1)
    raise KeyError(kind)


@pytest.mark.parametrize("prec", ["fp32", "tc_fp16", "tc_bf16x3"])
@pytest.mark.parametrize("kind", ["bda_uniform_channels", "unequal_channels", "single_sample_bins"])
@pytest.mark.parametrize("flags", [0, oracle.WTERM])
def test_edge_observations(psf, prec, kind, flags):
    obs = _edge_obs(kind)
    batch = obsgen.Batch(np.array([[0.031, -0.022], [-0.05, 0.04], [0.0, 0.0]]), np.array([8, 20, 6], np.int32),
                         4e-5)
    with psf.Plan(obs, prec=prec, flags=flags) as plan:
        b = psf.Batch.from_obsgen(batch)
        for name, mid in METHODS:
            ref = oracle.psf(obs, mid, batch, flags=flags)
            got = plan.forward(name, b).cpu().numpy().astype(np.float64)
            e = err_per_cutout(got, ref, batch)
            assert e.max() <= small_tol(prec, obs, batch), (name, e)


@pytest.mark.parametrize("prec", ["fp32", "tc_fp16"])
def test_literal_theta_reading(psf, prec):
    obs = obsgen.tiny_obs(nant=5, ntime=40, nchan=4, tavg=8, favg=2)
    batch = obsgen.Batch(np.array([[0.04, 0.03]]), np.array([16], np.int32), 4e-5)
    with psf.Plan(obs, prec=prec, flags=oracle.LITERAL_THETA) as plan:
        got = plan.approx_img(psf.Batch.from_obsgen(batch)).cpu().numpy().astype(np.float64)
    ref = oracle.psf(obs, oracle.IMG, batch, flags=oracle.LITERAL_THETA)
    assert err_per_cutout(got, ref, batch).max() <= small_tol(prec, obs, batch)


@pytest.mark.parametrize("prec", ["fp32", "tc_fp16"])
def test_sizes_offsets_and_ragged_tiles(psf, prec):
    """Sizes that leave ragged tiles (2, 6, 66, 130 with 64/128/256-wide tiles) and
    caller-given non-packed offsets: gaps between cutouts stay untouched."""
    import torch
    obs = obsgen.tiny_obs(nant=6, ntime=24, nchan=4, tavg=4, favg=2, weights=True)
    npix = np.array([2, 6, 66, 130, 64], np.int32)
    lm = np.array([[0.01, 0.02], [-0.03, 0.01], [0.02, -0.04], [0.05, 0.05], [0.0, -0.02]])
    offs = np.cumsum(np.concatenate([[7], (npix[:-1].astype(np.int64) ** 2) + 5]))
    total = int(offs[-1] + npix[-1] ** 2 + 3)
    cell = 3e-5
    with psf.Plan(obs, prec=prec) as plan:
        b = psf.Batch(lm, npix, cell, out_offset=offs)
        out = torch.full((total,), -7.0, device="cuda")
        plan.exact(b, out=out)
        got = out.cpu().numpy().astype(np.float64)
    ref = oracle.psf(obs, oracle.EXACT, obsgen.Batch(lm, npix, cell), offsets=offs)
    gaps = np.concatenate([np.isnan(ref), np.ones(total - ref.size, bool)])
    assert np.all(got[gaps] == -7.0)
    for p in range(len(npix)):
        sl = slice(offs[p], offs[p] + npix[p] ** 2)
        e = np.max(np.abs(got[sl] - ref[sl])) / np.max(np.abs(ref[sl]))
        assert e <= small_tol(prec, obs, obsgen.Batch(lm, npix, cell)), (p, e)


def test_empty_batch_and_bad_requests(psf):
    import torch
    obs = obsgen.tiny_obs()
    with psf.Plan(obs, prec="tc_fp16") as plan:
        out = torch.zeros(4, device="cuda")
        plan.exact(psf.Batch(np.zeros((0, 2)), np.zeros(0, np.int32), 1e-5), out=out)
        assert torch.all(out == 0)
        with pytest.raises(psf.PsfError) as ei:          # odd size
            plan.exact(psf.Batch([[0.01, 0.0]], [7], 1e-5))
        assert ei.value.status == -1
        with pytest.raises(psf.PsfError) as ei:          # tensor cores stop at 256
            plan.exact(psf.Batch([[0.01, 0.0]], [258], 1e-5))
        assert ei.value.status == -4
        with pytest.raises(psf.PsfError):                 # overlapping cutouts
            plan.exact(psf.Batch([[0.01, 0.0], [0.0, 0.01]], [8, 8], 1e-5, out_offset=[0, 10]),
                       out=torch.zeros(200, device="cuda"))
        with pytest.raises(psf.PsfError):                 # |l0| >= 1
            plan.exact(psf.Batch([[1.0, 0.5]], [8], 1e-5))
    with psf.Plan(obs, prec="fp32") as plan:           # the FP32 path takes large cutouts
        out = plan.exact(psf.Batch([[0.01, 0.0]], [258], 1e-5))
        assert torch.isfinite(out).all()
    with psf.Plan(obs, prec="tc_bf16x3", flags=psf.PSF_COMPLEX_OUT) as plan:   # split precision: real parts only
        with pytest.raises(psf.PsfError) as ei:
            plan.exact(psf.Batch([[0.01, 0.0]], [16], 1e-5))
        assert ei.value.status == -4


# ------------------------------------------------------------------ workload 2 (sampled, full size)
@pytest.fixture(scope="module")
def c2():
    obs = obsgen.config2_obs()
    batch = obsgen.config2_batch()
    N = int(batch.npix[0])
    rng = np.random.default_rng(11)
    sel = [N // 2 * N + N // 2, 0, N - 1, N * N - 1, (N // 2) * N + N // 2 + 1, (N // 2 + 3) * N + N // 2 - 2]
    sel += list(rng.choice(N * N, 10, replace=False))
    sel = np.array(sorted(set(int(x) for x in sel)), np.int64)
    refs = {name: oracle.psf(obs, mid, batch, pix_sel=sel)[sel] for name, mid in METHODS}
    return obs, batch, sel, refs


@pytest.mark.parametrize("prec", ["tc_fp16", "fp32", "tc_bf16x3"])
def test_config2_sampled_pixels(psf, c2, prec):
    """MeerKAT-shaped single 128 x 128 cutout at full size, in the launch
    configuration the benchmark times; the oracle evaluates sampled pixels one by one."""
    obs, batch, sel, refs = c2
    with psf.Plan(obs, prec=prec) as plan:
        b = psf.Batch.from_obsgen(batch)
        for name, _ in METHODS:
            got = plan.forward(name, b).cpu().numpy().astype(np.float64)
            ref = refs[name]
            e = np.max(np.abs(got[sel] - ref)) / np.max(np.abs(ref))   # the centre pixel is sampled
            assert e <= TOL[prec], (name, e)
        assert plan.sync_status() == 0
