"""Undivided brute-force evaluation of the smeared PSF (test infrastructure only).

A second, deliberately different route to the same definition, used to pin the
factored oracle on tiny inputs:

  * the averaged visibility of a unit source at L0 is computed with its full
    absolute phase, exp(-2 pi i uvw_s . L0 nu / c), averaged over the raw samples
    of the bin (Eq. 13, discrete in time) and integrated over each raw channel
    by Gauss-Legendre quadrature instead of the closed-form sinc;
  * each pixel is imaged at its absolute direction l = l0 + dl with the bin-centre
    baseline u_k = ubar_k nu_r / c (Eqs. 21-22), without cancelling u_k . L0
    analytically;
  * everything runs in numpy extended precision (np.longdouble).

Only the exact method is brute-forced: it is the one whose factoring (absolute
phase removal, channel closed form) the oracle relies on.
"""
from __future__ import annotations

import numpy as np

C_LIGHT = np.longdouble(299792458.0)
TWO_PI = 2 * np.longdouble(np.pi)


def _gl_nodes(n: int):
    x, w = np.polynomial.legendre.leggauss(n)
    return x.astype(np.longdouble), w.astype(np.longdouble)


def psf_exact(obs, l0: float, m0: float, npix: int, cell: float, wterm: bool = False,
              nquad: int = 24, imag: bool = False) -> np.ndarray:
    """Cutout [npix, npix] (row j = m offset, column i = l offset) in longdouble: the
    real part of the sum over averaged visibilities, or with imag=True its imaginary
    part."""
    ld = np.longdouble
    uvw = obs.uvw_m.astype(ld)
    freq = obs.freq_hz.astype(ld)
    width = obs.chan_width_hz.astype(ld)
    favg = int(obs.favg)
    nout = obs.nchan // favg
    l0, m0 = ld(l0), ld(m0)
    n0m1 = (np.sqrt(ld(1) - l0 * l0 - m0 * m0) - 1) if wterm else ld(0)
    L0 = np.array([l0, m0, n0m1], dtype=ld)
    xq, wq = _gl_nodes(nquad)
    off = (np.arange(npix) - npix // 2).astype(ld) * ld(cell)
    L = l0 + off[None, :]                     # absolute l for column i
    M = m0 + off[:, None]                     # absolute m for row j
    out = np.zeros((npix, npix), dtype=ld)
    k = 0
    for b in range(obs.nbl):
        n = int(obs.tavg[b])
        for tau in range(obs.ntime // n):
            samp = uvw[b, tau * n:(tau + 1) * n]          # [n, 3]
            ubar = samp.mean(axis=0)
            X = samp @ L0                                  # uvw_s . L0 [m]
            for r in range(nout):
                chans = range(r * favg, (r + 1) * favg)
                dnu = sum(width[c] for c in chans)
                nu_r = sum(freq[c] for c in chans) / favg
                vis = ld(0) + 0j
                vis_re = ld(0)
                vis_im = ld(0)
                for c in chans:
                    # (1/width) * integral over the channel = (1/2) sum_q wq f(nu_c + x_q width/2)
                    nu = freq[c] + xq * width[c] / 2       # [nquad]
                    ph = -TWO_PI * np.outer(X, nu) / C_LIGHT  # [n, nquad]
                    frac = width[c] / dnu / n
                    vis_re += frac * (np.cos(ph) @ wq).sum() / 2
                    vis_im += frac * (np.sin(ph) @ wq).sum() / 2
                u = ubar * nu_r / C_LIGHT
                W = ld(obs.weights[k]) if obs.weights is not None else ld(n * favg)
                ph = TWO_PI * (u[0] * L + u[1] * M + u[2] * n0m1)
                if imag:
                    out += W * (vis_re * np.sin(ph) + vis_im * np.cos(ph))
                else:
                    out += W * (vis_re * np.cos(ph) - vis_im * np.sin(ph))
                k += 1
    return out
