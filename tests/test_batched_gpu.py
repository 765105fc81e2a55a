"""GPU parity of the batched (Khatri-Rao) tensor-core form against the FP64 oracle.

Groups of at least 32 positions with one cutout size N (a multiple of 32, <= 256) go
to the batched kernel; other positions of the same call go to the per-cutout kernel.
The oracle evaluates sampled pixels of every cutout (the centre pixel and random
ones).  Tolerance: err_max <= 1e-4 of each cutout's sampled peak on workloads with
many visibilities (FP16 operands, FP32 accumulation).
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


def _sample(batch, offsets, per_pos, seed):
    rng = np.random.default_rng(seed)
    sel = []
    for p in range(batch.npos):
        N = int(batch.npix[p])
        pix = {(N // 2) * N + N // 2}
        pix.update(int(x) for x in rng.choice(N * N, per_pos, replace=False))
        sel.extend(int(offsets[p]) + x for x in sorted(pix))
    return np.array(sel, np.int64)


def _errors(got, ref, sel, batch, offsets):
    errs = []
    for p in range(batch.npos):
        n2 = int(batch.npix[p]) ** 2
        m = (sel >= offsets[p]) & (sel < offsets[p] + n2)
        g, r = got[sel[m]], ref[sel[m]]
        errs.append(np.max(np.abs(g - r)) / np.max(np.abs(r)))
    return np.array(errs)


def _mixed_batch(seed, counts, radius, cell):
    rng = np.random.default_rng(seed)
    npix = np.concatenate([np.full(c, n, np.int32) for n, c in counts])
    rng.shuffle(npix)
    lm = rng.uniform(-radius, radius, size=(len(npix), 2))
    return obsgen.Batch(lm, npix, cell)


@pytest.mark.parametrize("prec,tol", [("tc_fp16", 1e-4), ("tc_bf16", 1e-3), ("tc_fp16x3", 2e-5)])
def test_batched_mixed_sizes_config1(psf, prec, tol):
    """Workload-1 observation; 40 x 32^2 and 36 x 64^2 cutouts (batched) plus a few
    96^2 and 128^2 ones (per-cutout), in one call.  The split precision modes take the
    per-cutout form for every position."""
    obs = obsgen.config1_obs()
    batch = _mixed_batch(5, [(32, 40), (64, 36), (96, 3), (128, 2)], 0.03, 2 * obsgen.ARCSEC)
    offs = obsgen.concat_pixels(batch)
    sel = _sample(batch, offs, 4, 9)
    with psf.Plan(obs, prec=prec) as plan:
        b = psf.Batch.from_obsgen(batch)
        for name, mid in METHODS:
            got = plan.forward(name, b).cpu().numpy().astype(np.float64)
            ref = oracle.psf(obs, mid, batch, pix_sel=sel)
            e = _errors(got, ref, sel, batch, offs)
            assert e.max() <= tol, (name, e.max(), int(np.argmax(e)))
        assert plan.sync_status() == 0


def test_batched_gaps_untouched(psf):
    """Caller-given offsets with gaps: the batched path zeroes and fills only cutouts."""
    import torch
    obs = obsgen.config1_obs()
    n = 33
    npix = np.full(n, 32, np.int32)
    lm = np.random.default_rng(2).uniform(-0.02, 0.02, size=(n, 2))
    offs = 11 + np.arange(n, dtype=np.int64) * (32 * 32 + 7)
    total = int(offs[-1] + 32 * 32 + 5)
    cell = 2 * obsgen.ARCSEC
    batch = obsgen.Batch(lm, npix, cell)
    sel = _sample(batch, offs, 3, 4)
    with psf.Plan(obs, prec="tc_fp16") as plan:
        out = torch.full((total,), 3.5, device="cuda")
        plan.exact(psf.Batch(lm, npix, cell, out_offset=offs), out=out)
        got = out.cpu().numpy().astype(np.float64)
    mask = np.ones(total, bool)
    for o in offs:
        mask[o:o + 32 * 32] = False
    assert np.all(got[mask] == 3.5)
    ref = oracle.psf(obs, oracle.EXACT, batch, pix_sel=sel, offsets=offs)
    assert _errors(got, ref, sel, batch, offs).max() <= 1e-4


def test_batched_config4_subset(psf):
    """Baseline-dependent averaging (workload 3/4 observation, 2016 baselines, ~1.45e7
    visibilities), 32 positions of 64^2 within 1 degree: the differentiation
    workload's shape at full visibility count, sampled pixels."""
    obs = obsgen.config3_obs()
    batch = obsgen.config4_batch(npos=32)
    offs = obsgen.concat_pixels(batch)
    sel = _sample(batch, offs, 3, 17)
    with psf.Plan(obs, prec="tc_fp16") as plan:
        b = psf.Batch.from_obsgen(batch)
        for name, mid in METHODS:
            got = plan.forward(name, b).cpu().numpy().astype(np.float64)
            ref = oracle.psf(obs, mid, batch, pix_sel=sel)
            e = _errors(got, ref, sel, batch, offs)
            assert e.max() <= 1e-4, (name, e.max())
        assert plan.sync_status() == 0


def test_batched_exact_channel_recurrence_favg2(psf):
    """Eight equally spaced output channels of two raw channels each: the exact
    weights take the per-bin channel recurrence with the Dirichlet factor.  Few
    visibilities (3 584), so the bound is a few FP16 unit roundoffs (2e-3)."""
    obs = obsgen.tiny_obs(seed=11, nant=8, ntime=64, nchan=16, tavg=4, favg=2, dt=4.0, df=1.5e6,
                          radius_m=4000.0)
    batch = _mixed_batch(8, [(32, 34)], 0.04, 3e-5)
    offs = obsgen.concat_pixels(batch)
    sel = _sample(batch, offs, 4, 21)
    with psf.Plan(obs, prec="tc_fp16") as plan:
        got = plan.exact(psf.Batch.from_obsgen(batch)).cpu().numpy().astype(np.float64)
        assert plan.sync_status() == 0
    ref = oracle.psf(obs, oracle.EXACT, batch, pix_sel=sel)
    assert _errors(got, ref, sel, batch, offs).max() <= 2e-3
