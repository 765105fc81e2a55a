"""Python binding of the smeared-PSF library (argument marshalling only).

Every step of the computation runs in the CUDA library behind the C ABI of
include/psf.h.  PyTorch provides device memory and the current CUDA stream; host
inputs are numpy arrays.  Names follow the paper: l0, m0 positions, W_k weights,
cell = pixel size, N = cutout size.
"""
from __future__ import annotations

import ctypes
from typing import Optional

import numpy as np
import torch

from . import _lib
from ._lib import check

PREC = {"fp32": _lib.PSF_FP32, "tc_fp16": _lib.PSF_TC_FP16, "tc_bf16": _lib.PSF_TC_BF16,
        "tc_fp16x3": _lib.PSF_TC_FP16X3, "tc_bf16x3": _lib.PSF_TC_BF16X3}
METHODS = {"exact": _lib.EXACT, "uv": _lib.UV, "img": _lib.IMG}


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _stream_handle(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Batch:
    """Host-side cutout requests marshalled into psf_batch_t."""

    def __init__(self, lm, npix, cell_rad: float, out_offset=None):
        self.lm = np.ascontiguousarray(np.asarray(lm, np.float64).reshape(-1, 2))
        npos = self.lm.shape[0]
        self.npix = np.ascontiguousarray(np.broadcast_to(np.asarray(npix, np.int32), (npos,)))
        self.cell = float(cell_rad)
        if out_offset is None:
            n2 = self.npix.astype(np.int64) ** 2
            self.offsets = np.concatenate([[0], np.cumsum(n2)[:-1]]).astype(np.int64) if npos else \
                np.zeros(0, np.int64)
            self._given = None
        else:
            self.offsets = np.ascontiguousarray(np.asarray(out_offset, np.int64))
            self._given = self.offsets
        self.npos = npos

    @classmethod
    def from_obsgen(cls, b):
        return cls(b.lm, b.npix, b.cell_rad)

    def total(self, per_px: int = 1) -> int:
        """Output floats needed: per_px = 2 for complex cutouts (PSF_COMPLEX_OUT), whose
        packed default offsets advance by 2 N^2."""
        if self.npos == 0:
            return 0
        n2 = self.npix.astype(np.int64) ** 2
        if self._given is None:
            return int(per_px * n2.sum())
        return int((self.offsets + per_px * n2).max())

    def struct(self) -> _lib.BatchT:
        return _lib.BatchT(self.npos, self.lm.ctypes.data if self.npos else None,
                           self.npix.ctypes.data if self.npos else None, 0, self.cell,
                           None if self._given is None else self._given.ctypes.data)


class Plan:
    """A plan of one observation (psf_plan); owns device arrays until close()."""

    def __init__(self, obs, prec: str = "fp32", flags: int = 0, algo: int = 0):
        L = _lib.lib()
        self._keep = [np.ascontiguousarray(obs.uvw_m, np.float64), np.ascontiguousarray(obs.time_s, np.float64),
                      np.ascontiguousarray(obs.freq_hz, np.float64),
                      np.ascontiguousarray(obs.chan_width_hz, np.float64),
                      np.ascontiguousarray(obs.tavg, np.int32)]
        wt = None if obs.weights is None else np.ascontiguousarray(obs.weights, np.float32)
        uvw, t, f, w, tavg = self._keep
        o = _lib.ObsT(uvw.shape[0], uvw.shape[1], f.shape[0], uvw.ctypes.data, t.ctypes.data, f.ctypes.data,
                      w.ctypes.data, tavg.ctypes.data, int(obs.favg), None if wt is None else wt.ctypes.data)
        opts = _lib.OptsT(PREC[prec], flags, algo, 0)
        h = ctypes.c_void_p()
        check(L.psf_plan(ctypes.byref(o), ctypes.byref(opts), ctypes.byref(h)), "psf_plan")
        self._h = h
        self._keep = None
        self.prec, self.flags, self.algo = prec, flags, algo
        self.nvis = int(L.psf_plan_nvis(h))
        tw, cw = getattr(obs, "time_window", None), getattr(obs, "chan_window", None)
        if tw is not None or cw is not None:
            self.set_windows(tw, cw)

    def set_windows(self, time_window=None, chan_window=None):
        """Windowed averaging (Eqs. 15-16) for the exact method and Methods 1 and 2:
        per-baseline weights over a bin's raw samples (concatenated over baselines) and
        [nbl, favg] over an output channel's raw channels; None for the boxcar."""
        tw = None if time_window is None else np.ascontiguousarray(time_window, np.float32)
        cw = None if chan_window is None else np.ascontiguousarray(chan_window, np.float32)
        check(_lib.lib().psf_plan_set_windows(self._h, None if tw is None else ctypes.c_void_p(tw.ctypes.data),
                                              None if cw is None else ctypes.c_void_p(cw.ctypes.data)),
              "psf_plan_set_windows")

    def set_weights(self, W: Optional[torch.Tensor] = None, stream=None):
        """Visibility weights W_k (device float32 [nvis], plan order) for later calls;
        None restores the natural weights."""
        if W is not None:
            assert W.dtype == torch.float32 and W.is_cuda and W.is_contiguous() and W.numel() == self.nvis
        check(_lib.lib().psf_plan_set_weights(self._h, None if W is None else ctypes.c_void_p(W.data_ptr()),
                                              _stream_handle(stream)), "psf_plan_set_weights")

    def set_opts(self, prec: Optional[str] = None, flags: Optional[int] = None, algo: Optional[int] = None):
        self.prec = prec if prec is not None else self.prec
        self.flags = flags if flags is not None else self.flags
        self.algo = algo if algo is not None else self.algo
        opts = _lib.OptsT(PREC[self.prec], self.flags, self.algo, 0)
        check(_lib.lib().psf_plan_set_opts(self._h, ctypes.byref(opts)), "psf_plan_set_opts")

    def forward(self, method: str, batch: Batch, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        """Cutouts of `method` ('exact' | 'uv' | 'img' | 'img_grid') into a device float32 tensor
        (with PSF_COMPLEX_OUT: N^2 real parts then N^2 imaginary parts per cutout)."""
        per = 2 if (self.flags & _lib.PSF_COMPLEX_OUT) else 1
        if out is None:
            out = torch.empty(max(batch.total(per), 1), dtype=torch.float32, device="cuda")
        assert out.dtype == torch.float32 and out.is_cuda and out.is_contiguous()
        assert out.numel() >= batch.total(per)
        fn = {"exact": "psf_exact", "uv": "psf_approx_uv", "img": "psf_approx_img",
              "img_grid": "psf_approx_img_grid"}[method]
        bs = batch.struct()
        check(getattr(_lib.lib(), fn)(self._h, ctypes.byref(bs), ctypes.c_void_p(out.data_ptr()),
                                      _stream_handle(stream)), fn)
        return out

    def exact(self, batch, out=None, stream=None):
        return self.forward("exact", batch, out, stream)

    def approx_uv(self, batch, out=None, stream=None):
        return self.forward("uv", batch, out, stream)

    def approx_img(self, batch, out=None, stream=None):
        return self.forward("img", batch, out, stream)

    def approx_img_grid(self, batch, out=None, stream=None):
        """Method 2 in the gridded form of Eq. 45 (N in {16, 32, 64, 128})."""
        return self.forward("img_grid", batch, out, stream)

    def img_grid_table(self, npix: int, cell: float, stream=None) -> torch.Tensor:
        """Diagnostic: the gridded form's table [npix(b), npix(a), 4] (Re S, Im S,
        omega_E dt_c du, (dnu/nu)_c |u_c|)."""
        t = torch.empty((npix, npix, 4), dtype=torch.float32, device="cuda")
        check(_lib.lib().psf_img_grid_table(self._h, int(npix), float(cell), ctypes.c_void_p(t.data_ptr()),
                                            _stream_handle(stream)), "psf_img_grid_table")
        return t

    def clean(self, dirty: torch.Tensor, cell: float, npix: int, method: str = "img_grid", gain: float = 0.1,
              threshold: float = 0.0, max_iter: int = 1000, model: Optional[torch.Tensor] = None,
              centre=(0.0, 0.0), facet_psf: bool = False, stream=None):
        """Hogbom CLEAN with position-dependent PSFs (Algorithm 2) on the device.  dirty:
        float32 CUDA tensor [nm, nl], overwritten with the residual; pixel (nl/2, nm/2) looks
        at `centre` (l, m).  facet_psf: one PSF at `centre` for every component (faceting)
        instead of the PSF at each peak.  Returns (residual,
        model, component pixel indices [niter], component fluxes [niter])."""
        assert dirty.dtype == torch.float32 and dirty.is_cuda and dirty.is_contiguous() and dirty.dim() == 2
        nm, nl = dirty.shape
        if model is None:
            model = torch.zeros_like(dirty)
        cpix = torch.empty(max(max_iter, 1), dtype=torch.int32, device=dirty.device)
        cflux = torch.empty(max(max_iter, 1), dtype=torch.float32, device=dirty.device)
        mcode = {"exact": _lib.EXACT, "uv": _lib.UV, "img": _lib.IMG, "img_grid": _lib.IMG_GRID}[method]
        cfg = _lib.CleanT(nl, nm, float(cell), float(centre[0]), float(centre[1]), int(npix), mcode, float(gain),
                          float(threshold), int(max_iter), _lib.PSF_CLEAN_FACET_PSF if facet_psf else 0)
        n = ctypes.c_int32(0)
        check(_lib.lib().psf_clean(self._h, ctypes.byref(cfg), ctypes.c_void_p(dirty.data_ptr()),
                                   ctypes.c_void_p(model.data_ptr()), ctypes.c_void_p(cpix.data_ptr()),
                                   ctypes.c_void_p(cflux.data_ptr()), ctypes.byref(n), _stream_handle(stream)),
              "psf_clean")
        return dirty, model, cpix[:n.value], cflux[:n.value]

    def fwhm(self, batch: Batch, cutouts: torch.Tensor, stream=None) -> torch.Tensor:
        """FWHM (radial, tangential) [npos, 2] float64 of the batch's cutouts (Fig. 3)."""
        assert cutouts.dtype == torch.float32 and cutouts.is_cuda and cutouts.is_contiguous()
        assert cutouts.numel() >= batch.total()
        out = torch.empty((max(batch.npos, 1), 2), dtype=torch.float64, device=cutouts.device)
        bs = batch.struct()
        check(_lib.lib().psf_fwhm(self._h, ctypes.byref(bs), ctypes.c_void_p(cutouts.data_ptr()),
                                  ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)), "psf_fwhm")
        return out[:batch.npos]

    def approx_uv_img(self, batch: Batch, out_uv: Optional[torch.Tensor] = None,
                      out_img: Optional[torch.Tensor] = None, stream=None):
        """Methods 1 and 2 of one batch in one call: (uv cutouts, image-plane cutouts)."""
        outs = []
        per = 2 if (self.flags & _lib.PSF_COMPLEX_OUT) else 1
        for o in (out_uv, out_img):
            if o is None:
                o = torch.empty(max(batch.total(per), 1), dtype=torch.float32, device="cuda")
            assert o.dtype == torch.float32 and o.is_cuda and o.is_contiguous()
            assert o.numel() >= batch.total(per)
            outs.append(o)
        bs = batch.struct()
        check(_lib.lib().psf_approx_uv_img(self._h, ctypes.byref(bs), ctypes.c_void_p(outs[0].data_ptr()),
                                           ctypes.c_void_p(outs[1].data_ptr()), _stream_handle(stream)),
              "psf_approx_uv_img")
        return outs[0], outs[1]

    def adjoint(self, method: str, batch: Batch, dL_dP: torch.Tensor, want_dW: bool = True, stream=None):
        """(dL/d(l0,m0) float64 [npos,2], dL/dW float32 [nvis] or None) on the device."""
        assert dL_dP.dtype == torch.float32 and dL_dP.is_cuda and dL_dP.is_contiguous()
        g_lm = torch.empty((max(batch.npos, 1), 2), dtype=torch.float64, device="cuda")
        g_W = torch.empty(self.nvis, dtype=torch.float32, device="cuda") if want_dW else None
        bs = batch.struct()
        check(_lib.lib().psf_adjoint(self._h, METHODS[method], ctypes.byref(bs), ctypes.c_void_p(dL_dP.data_ptr()),
                                     ctypes.c_void_p(g_lm.data_ptr()),
                                     None if g_W is None else ctypes.c_void_p(g_W.data_ptr()),
                                     _stream_handle(stream)), "psf_adjoint")
        return g_lm[:batch.npos], g_W

    def profile_enable(self, enable: bool = True):
        check(_lib.lib().psf_profile_enable(self._h, 1 if enable else 0), "psf_profile_enable")

    def profile_read(self):
        """(contraction ms, contraction launches, kernel launches) since the last read."""
        ms, nc, nk = ctypes.c_double(), ctypes.c_int64(), ctypes.c_int64()
        check(_lib.lib().psf_profile_read(self._h, ctypes.byref(ms), ctypes.byref(nc), ctypes.byref(nk)),
              "psf_profile_read")
        return ms.value, nc.value, nk.value

    def sync_status(self, stream=None) -> int:
        return int(_lib.lib().psf_sync_status(self._h, _stream_handle(stream)))

    def close(self):
        if getattr(self, "_h", None):
            _lib.lib().psf_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def selftest_umma(a: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
    """D = A B^T through one tcgen05 MMA tile (A [128,64] fp16, B [n,64] fp16)."""
    assert a.shape == (128, 64) and a.dtype == torch.float16 and b.dtype == torch.float16 and b.shape[1] == 64
    a, b = a.contiguous(), b.contiguous()
    d = torch.empty((128, b.shape[0]), dtype=torch.float32, device="cuda")
    check(_lib.lib().psf_selftest_umma(ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                                       ctypes.c_void_p(d.data_ptr()), b.shape[0]), "psf_selftest_umma")
    return d


def fma_rate(packed: bool = False) -> float:
    """Measured FP32 FMA throughput of the current device in flop/s (scalar FMAs, or
    packed FP32 pairs with packed=True)."""
    r = ctypes.c_double(0.0)
    check(_lib.lib().psf_selftest_fma_rate(1 if packed else 0, ctypes.byref(r)), "psf_selftest_fma_rate")
    return r.value


class SmearedPSF(torch.autograd.Function):
    """Cutouts as a differentiable function of the positions (l0, m0) and, optionally,
    of the visibility weights W_k.

    forward(lm, W, ...) evaluates `method` on the plan's observation in the plan's
    precision (with W given, the plan's weights are replaced by W first and stay so);
    backward runs the library's adjoint (psf_adjoint) on the incoming gradient.  The
    backward is the vector-Jacobian product of the exact map of Eqs. 21-22 (the FP64
    definition), not of the rounded forward: FP32 CUDA cores for PSF_FP32 and the split
    precision plans (about 1e-6 of the largest gradient component), the tensor-core
    adjoint (H in FP16/BF16 operands, FP32 accumulation; about 3e-4 / 3e-3) for
    single-pass FP16/BF16 plans whose cutouts are multiples of 32 pixels.  lm is a
    float64 host tensor [npos, 2] (positions are host inputs of the C ABI), its gradient
    is returned on lm's device; W is a device float32 tensor [nvis] or None.
    """

    @staticmethod
    def forward(ctx, lm, W, plan, method, npix, cell):
        batch = Batch(lm.detach().cpu().numpy(), npix, cell)
        if W is not None:
            plan.set_weights(W.detach().contiguous())
        out = plan.forward(method, batch)[:batch.total()]
        ctx.plan, ctx.method, ctx.batch, ctx.lm_device = plan, method, batch, lm.device
        ctx.want_W = W is not None
        return out

    @staticmethod
    def backward(ctx, grad_out):
        g = grad_out.detach().to(torch.float32).contiguous()
        g_lm, g_W = ctx.plan.adjoint(ctx.method, ctx.batch, g, want_dW=ctx.want_W and ctx.needs_input_grad[1])
        return g_lm.to(ctx.lm_device), g_W, None, None, None, None


def smeared_psf(plan: Plan, method: str, lm: torch.Tensor, npix, cell: float,
                W: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Differentiable cutouts of `method` at positions lm, optionally with weights W
    (see SmearedPSF)."""
    return SmearedPSF.apply(lm, W, plan, method, npix, cell)
