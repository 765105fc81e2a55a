"""GPU adjoint (psf_adjoint) against the oracle's float64 vector-Jacobian product,
which test_oracle_pins.py::test_p8 pins to float64 central differences.

Tolerances are relative to the size of the gradient vector.  FP32 CUDA-core adjoint:
2e-5 of max |dL/dW| and 2e-4 of max |dL/dl0|, |dL/dm0| (the position gradient is a sum
of signed terms much larger than their total).  Tensor-core adjoint (single-pass
FP16/BF16 plans): H = sum over pixels of dL/dP times the twiddles is formed from
16-bit operands, so each H carries about one unit roundoff of its terms' size: 1e-3
(FP16, 2^-11 = 4.9e-4 x 2) and 1e-2 (BF16) of the largest component, for both gradients;
on few visibilities (thousands), where the roundings average out less, 2e-3 (FP16).
"""
import numpy as np
import pytest

import obsgen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def psf():
    import paper_2009_07010_gb300 as m
    m.build_library()
    return m


def _cotangent(P, seed):
    rng = np.random.default_rng(seed)
    T = P * (1 + 0.01 * rng.standard_normal(P.size)) + 0.05 * np.abs(P).max() * rng.standard_normal(P.size)
    return 2 * (P - T)


TOL = {"fp32": (2e-5, 2e-4), "tc_fp16": (1e-3, 1e-3), "tc_bf16": (1e-2, 1e-2)}


def _check(psf, obs, batch, method, flags=0, prec="fp32", tol=None):
    import torch
    mid = {"exact": oracle.EXACT, "uv": oracle.UV, "img": oracle.IMG}[method]
    P = oracle.psf(obs, mid, batch, flags=flags)
    R = _cotangent(P, 3)
    g_lm_ref, g_W_ref = oracle.vjp(obs, mid, batch, R, flags=flags)
    with psf.Plan(obs, prec=prec, flags=flags) as plan:
        b = psf.Batch.from_obsgen(batch)
        g_lm, g_W = plan.adjoint(method, b, torch.tensor(R, dtype=torch.float32, device="cuda"))
        assert plan.sync_status() == 0
        g_lm, g_W = g_lm.cpu().numpy(), g_W.cpu().numpy().astype(np.float64)
    e_w = np.max(np.abs(g_W - g_W_ref)) / np.max(np.abs(g_W_ref))
    e_l = np.max(np.abs(g_lm - g_lm_ref)) / np.max(np.abs(g_lm_ref))
    tw, tl = tol or TOL[prec]
    assert e_w <= tw, (method, prec, e_w)
    assert e_l <= tl, (method, prec, e_l, g_lm, g_lm_ref)


@pytest.mark.parametrize("method", ["exact", "uv", "img"])
def test_adjoint_config1(psf, method):
    obs = obsgen.config1_obs()
    batch = obsgen.Batch(np.array([[0.02, 0.02], [-0.013, 0.031], [0.04, -0.005]]), np.array([64, 32, 64], np.int32),
                         2 * obsgen.ARCSEC)
    _check(psf, obs, batch, method)


@pytest.mark.parametrize("method", ["exact", "uv", "img"])
@pytest.mark.parametrize("flags", [0, oracle.WTERM])
def test_adjoint_edge_cases(psf, method, flags):
    obs = obsgen.tiny_obs(nant=5, ntime=40, nchan=8, tavg=[1, 2, 3, 5, 7, 8, 10, 13, 20, 40], favg=4, weights=True)
    batch = obsgen.Batch(np.array([[0.031, -0.022], [-0.05, 0.04], [0.002, 0.001]]), np.array([8, 34, 2], np.int32),
                         4e-5)
    _check(psf, obs, batch, method, flags)


def test_autograd_positions(psf):
    """torch.autograd through SmearedPSF: d/d(l0,m0) of sum (P - T)^2."""
    import torch
    obs = obsgen.config1_obs()
    lm0 = np.array([[0.02, 0.02], [-0.013, 0.031]])
    cell = 2 * obsgen.ARCSEC
    npix = np.array([32, 32], np.int32)
    T = oracle.psf(obs, oracle.EXACT, obsgen.Batch(lm0 + 1e-5, npix, cell))
    with psf.Plan(obs, prec="fp32") as plan:
        lm = torch.tensor(lm0, dtype=torch.float64, requires_grad=True)
        P = psf.smeared_psf(plan, "exact", lm, npix, cell)
        loss = ((P.double() - torch.tensor(T, device="cuda")) ** 2).sum()
        loss.backward()
        g = lm.grad.numpy()
        R = 2 * (P.detach().cpu().numpy().astype(np.float64) - T)
    g_ref, _ = oracle.vjp(obs, oracle.EXACT, obsgen.Batch(lm0, npix, cell), R)
    assert np.max(np.abs(g - g_ref)) <= 2e-4 * np.max(np.abs(g_ref))


def test_adjoint_rejects_bad_input(psf):
    import torch
    obs = obsgen.tiny_obs()
    with psf.Plan(obs, prec="fp32") as plan:
        R = torch.zeros(600 * 600, device="cuda")
        with pytest.raises(psf.PsfError) as ei:
            plan.adjoint("exact", psf.Batch([[0.01, 0.0]], [600], 1e-5), R)
        assert ei.value.status == -4
        g_lm, g_W = plan.adjoint("exact", psf.Batch(np.zeros((0, 2)), np.zeros(0, np.int32), 1e-5), R)
        assert torch.all(g_W == 0)


# ------------------------------------------------------------------ tensor-core adjoint
@pytest.mark.parametrize("prec", ["tc_fp16", "tc_bf16"])
@pytest.mark.parametrize("method", ["exact", "uv", "img"])
def test_adjoint_tensor_cores_config1(psf, method, prec):
    """Cutouts of 64 and 32 pixels (multiples of 32): H on the tensor cores."""
    obs = obsgen.config1_obs()
    batch = obsgen.Batch(np.array([[0.02, 0.02], [-0.013, 0.031], [0.04, -0.005]]), np.array([64, 32, 64], np.int32),
                         2 * obsgen.ARCSEC)
    _check(psf, obs, batch, method, prec=prec)


@pytest.mark.parametrize("method", ["exact", "uv", "img"])
@pytest.mark.parametrize("flags", [0, oracle.WTERM])
def test_adjoint_tensor_cores_channel_groups(psf, method, flags):
    """Eight equally spaced output channels of two raw channels (the exact method's fold
    then runs the per-bin channel recurrence), baseline-dependent averaging, weights."""
    obs = obsgen.tiny_obs(seed=9, nant=6, ntime=48, nchan=16, tavg=[2, 3, 4, 6, 8, 12, 16, 24, 2, 3, 4, 6, 8, 12, 16],
                          favg=2, df=1.5e6, weights=True)
    batch = obsgen.Batch(np.array([[0.031, -0.022], [-0.05, 0.04], [0.004, 0.001]]), np.array([32, 64, 32], np.int32),
                         3e-5)
    _check(psf, obs, batch, method, flags, prec="tc_fp16", tol=(2e-3, 2e-3))


def test_adjoint_tensor_cores_differentiation_scale(psf):
    """The differentiation workload's observation (baseline-dependent averaging, 13.7 M
    visibilities) with 32 of its 64 x 64 positions; the loss of the workload with targets
    at positions offset by 1e-5 rad (the targets from the FP32 forward, which the parity
    tests tie to the oracle): the tensor-core adjoint against the FP32 adjoint."""
    import torch
    obs = obsgen.config3_obs()
    bg = obsgen.config4_batch(npos=32)
    b = psf.Batch.from_obsgen(bg)
    bt = psf.Batch(bg.lm + 1e-5, bg.npix, bg.cell_rad)
    with psf.Plan(obs, prec="fp32") as plan:
        R = 2 * (plan.exact(b) - plan.exact(bt))
        g32 = [x.cpu().numpy().astype(np.float64) for x in plan.adjoint("exact", b, R)]
        plan.set_opts(prec="tc_fp16")
        gtc = [x.cpu().numpy().astype(np.float64) for x in plan.adjoint("exact", b, R)]
        assert plan.sync_status() == 0
    for a, r in zip(gtc, g32):
        assert np.max(np.abs(a - r)) / np.max(np.abs(r)) <= 1e-3
    # the offset targets pull every position towards them: dL/dl0, dL/dm0 < 0
    assert np.mean(g32[0] < 0) > 0.9


def test_autograd_weights_and_positions(psf):
    """torch.autograd through SmearedPSF with the weights as an input: dL/dW and
    dL/d(l0, m0) of sum (P - T)^2 against the oracle's vector-Jacobian product."""
    import torch
    obs = obsgen.tiny_obs(nant=5, ntime=40, nchan=8, tavg=[1, 2, 3, 5, 7, 8, 10, 13, 20, 40], favg=4, weights=True)
    lm0 = np.array([[0.031, -0.022], [-0.015, 0.02]])
    cell, npix = 4e-5, np.array([16, 8], np.int32)
    bg = obsgen.Batch(lm0, npix, cell)
    T = oracle.psf(obs, oracle.EXACT, obsgen.Batch(lm0 + 1e-5, npix, cell))
    W0 = obs.weights.astype(np.float32)
    with psf.Plan(obs, prec="fp32") as plan:
        lm = torch.tensor(lm0, dtype=torch.float64, requires_grad=True)
        W = torch.tensor(W0 * 1.5, device="cuda", requires_grad=True)     # weights other than the plan's
        P = psf.smeared_psf(plan, "exact", lm, npix, cell, W=W)
        loss = ((P.double() - torch.tensor(T, device="cuda")) ** 2).sum()
        loss.backward()
        R = 2 * (P.detach().cpu().numpy().astype(np.float64) - T)
        g_lm, g_W = lm.grad.numpy(), W.grad.cpu().numpy().astype(np.float64)
    o2 = obsgen.Observation(obs.uvw_m, obs.time_s, obs.freq_hz, obs.chan_width_hz, obs.tavg, obs.favg, W0 * 1.5)
    g_lm_ref, g_W_ref = oracle.vjp(o2, oracle.EXACT, bg, R)
    assert np.max(np.abs(g_lm - g_lm_ref)) <= 2e-4 * np.max(np.abs(g_lm_ref))
    assert np.max(np.abs(g_W - g_W_ref)) <= 2e-5 * np.max(np.abs(g_W_ref))


def test_adjoint_differentiation_scale_vs_oracle(psf):
    """One 64 x 64 position of the differentiation workload (13.7 M visibilities with
    baseline-dependent averaging), loss sum (P - T)^2 with the target at +1e-5 rad: the
    FP32 and tensor-core adjoints against the oracle's vector-Jacobian product for the same
    cotangent (the oracle sums every pixel for every visibility, about a minute)."""
    import torch
    obs = obsgen.config3_obs()
    bg = obsgen.config4_batch(npos=1)
    b = psf.Batch.from_obsgen(bg)
    bt = psf.Batch(bg.lm + 1e-5, bg.npix, bg.cell_rad)
    with psf.Plan(obs, prec="fp32") as plan:
        R = 2 * (plan.exact(b) - plan.exact(bt))
        got = {"fp32": [x.cpu().numpy().astype(np.float64) for x in plan.adjoint("exact", b, R)]}
        plan.set_opts(prec="tc_fp16")
        got["tc_fp16"] = [x.cpu().numpy().astype(np.float64) for x in plan.adjoint("exact", b, R)]
        assert plan.sync_status() == 0
        torch.cuda.synchronize()
    g_lm_ref, g_W_ref = oracle.vjp(obs, oracle.EXACT, bg, R.cpu().numpy().astype(np.float64))
    assert g_lm_ref[0, 0] + g_lm_ref[0, 1] < 0   # pulled towards the target at (+1e-5, +1e-5)
    for prec, (g_lm, g_W) in got.items():
        tw, tl = TOL[prec]
        e_w = np.max(np.abs(g_W - g_W_ref)) / np.max(np.abs(g_W_ref))
        e_l = np.max(np.abs(g_lm - g_lm_ref)) / np.max(np.abs(g_lm_ref))
        assert e_w <= tw, (prec, e_w)
        assert e_l <= tl, (prec, e_l, g_lm, g_lm_ref)
