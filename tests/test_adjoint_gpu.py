"""GPU adjoint (psf_adjoint, FP32) against the oracle's float64 vector-Jacobian
product, which test_oracle_pins.py::test_p8 pins to float64 central differences.

Tolerances: the adjoint sums FP32 products over all visibilities and pixels, so
errors are relative to the size of the gradient vector: 2e-5 of max |dL/dW| and
2e-4 of max |dL/dl0|, |dL/dm0| (the position gradient is a sum of signed terms
much larger than their total).
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


def _check(psf, obs, batch, method, flags=0):
    import torch
    mid = {"exact": oracle.EXACT, "uv": oracle.UV, "img": oracle.IMG}[method]
    P = oracle.psf(obs, mid, batch, flags=flags)
    R = _cotangent(P, 3)
    g_lm_ref, g_W_ref = oracle.vjp(obs, mid, batch, R, flags=flags)
    with psf.Plan(obs, prec="fp32", flags=flags) as plan:
        b = psf.Batch.from_obsgen(batch)
        g_lm, g_W = plan.adjoint(method, b, torch.tensor(R, dtype=torch.float32, device="cuda"))
        assert plan.sync_status() == 0
        g_lm, g_W = g_lm.cpu().numpy(), g_W.cpu().numpy().astype(np.float64)
    e_w = np.max(np.abs(g_W - g_W_ref)) / np.max(np.abs(g_W_ref))
    e_l = np.max(np.abs(g_lm - g_lm_ref)) / np.max(np.abs(g_lm_ref))
    assert e_w <= 2e-5, (method, e_w)
    assert e_l <= 2e-4, (method, e_l, g_lm, g_lm_ref)


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
