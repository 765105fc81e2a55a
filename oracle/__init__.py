"""FP64 CPU oracle for the smeared PSF (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The CUDA
library never imports, links or calls it, and it never calls the library.

The arithmetic lives in ``psf_oracle.c`` (plain loops, double precision,
OpenMP over independent outputs); this module only compiles it with gcc and
marshals numpy arrays through ctypes.  ``brute.py`` holds a second, undivided
evaluation in extended precision used to pin the factored form.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(closed forms, limits, symmetries, brute force, finite differences) and, for the
gridded image-plane form, ``tests/test_oracle_grid_pins.py`` (numpy FFT, exact
agreement with the visibility-level Method 2 on cell-centred uv points, brute-force
gridding, symmetry) and, for Hogbom CLEAN (Algorithm 2, ``clean``),
``tests/test_oracle_clean_pins.py`` (closed-form decay of isolated sources).  The
accuracy levels the paper reads off its MeerKAT figures (Sect. 4, Figs. 4-7)
are *parity unpinned*: they need the paper's array, dataset and imager.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "psf_oracle.c")
_SO = os.path.join(_HERE, "_psf_oracle.so")
_lock = threading.Lock()
_lib = None

EXACT, UV, IMG = 0, 1, 2
WTERM, LITERAL_THETA = 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle shared object (gcc, OpenMP, no fast-math, no FMA contraction:
    the nearest-cell decisions of the gridded form must round as written)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               "-fno-fast-math", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            obs_args = [ctypes.c_int] * 4 + [P] * 8
            lib.or_nvis.restype = ctypes.c_int64
            lib.or_nvis.argtypes = [ctypes.c_int] * 4 + [P]
            lib.or_vis_table.restype = ctypes.c_int
            lib.or_vis_table.argtypes = obs_args + [P]
            lib.or_decorr.restype = ctypes.c_int
            lib.or_decorr.argtypes = obs_args + [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                                 ctypes.c_int, P, P, P]
            lib.or_psf.restype = ctypes.c_int
            lib.or_psf.argtypes = obs_args + [ctypes.c_int, ctypes.c_int, P, P, ctypes.c_double,
                                              ctypes.c_int, P, P, ctypes.c_int64, P]
            lib.or_grid_tables.restype = ctypes.c_int
            lib.or_grid_tables.argtypes = obs_args + [ctypes.c_int, ctypes.c_double, P, P, P, P, P]
            lib.or_psf_img_grid.restype = ctypes.c_int
            lib.or_psf_img_grid.argtypes = obs_args + [ctypes.c_int, P, ctypes.c_int, ctypes.c_double,
                                                       ctypes.c_int, P]
            lib.or_psf_img_grid_tables.restype = ctypes.c_int
            lib.or_psf_img_grid_tables.argtypes = [ctypes.c_int, ctypes.c_double, P, P, P, ctypes.c_int, P,
                                                   ctypes.c_int, P]
            lib.or_vjp.restype = ctypes.c_int
            lib.or_vjp.argtypes = obs_args + [ctypes.c_int, ctypes.c_int, P, P, ctypes.c_double,
                                              ctypes.c_int, P, P, P, P]
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


class _Obs:
    """Contiguous copies of an obsgen.Observation kept alive for a call."""

    def __init__(self, obs):
        self.uvw = np.ascontiguousarray(obs.uvw_m, np.float64)
        self.t = np.ascontiguousarray(obs.time_s, np.float64)
        self.f = np.ascontiguousarray(obs.freq_hz, np.float64)
        self.w = np.ascontiguousarray(obs.chan_width_hz, np.float64)
        self.tavg = np.ascontiguousarray(obs.tavg, np.int32)
        self.wt = None if obs.weights is None else np.ascontiguousarray(obs.weights, np.float32)
        tw, cw = getattr(obs, "time_window", None), getattr(obs, "chan_window", None)
        self.tw = None if tw is None else np.ascontiguousarray(tw, np.float32)
        self.cw = None if cw is None else np.ascontiguousarray(cw, np.float32)
        self.nbl, self.ntime = self.uvw.shape[0], self.uvw.shape[1]
        self.nchan, self.favg = self.f.shape[0], int(obs.favg)

    def args(self):
        return [self.nbl, self.ntime, self.nchan, self.favg, _p(self.uvw), _p(self.t),
                _p(self.f), _p(self.w), _p(self.tavg), _p(self.wt), _p(self.tw), _p(self.cw)]


def nvis(obs) -> int:
    o = _Obs(obs)
    return int(_load().or_nvis(o.nbl, o.ntime, o.nchan, o.favg, _p(o.tavg)))


def vis_table(obs) -> dict:
    """Per averaged visibility: u,v,w [lambda], nu, dnu, dt, W, ubar [m], dedge [m]."""
    o = _Obs(obs)
    n = nvis(obs)
    out = np.empty((n, 13), np.float64)
    if _load().or_vis_table(*o.args(), _p(out)) != 0:
        raise ValueError("invalid observation")
    return dict(uvw_lambda=out[:, 0:3], nu=out[:, 3], dnu=out[:, 4], dt=out[:, 5], W=out[:, 6],
                ubar_m=out[:, 7:10], dedge_m=out[:, 10:13])


def decorr(obs, method: int, l0: float, m0: float, flags: int = 0, grad: bool = False):
    """D_k(l0, m0) as complex128 [nvis]; with grad, also dD [nvis, 4] (re/im d/dl0, d/dm0)."""
    o = _Obs(obs)
    n = nvis(obs)
    dre = np.empty(n)
    dim = np.empty(n)
    dd = np.empty((n, 4)) if grad else None
    if _load().or_decorr(*o.args(), int(method), float(l0), float(m0), int(flags),
                         _p(dre), _p(dim), _p(dd)) != 0:
        raise ValueError("invalid observation")
    D = dre + 1j * dim
    return (D, dd) if grad else D


def _batch_arrays(batch, offsets=None):
    lm = np.ascontiguousarray(batch.lm, np.float64)
    npix = np.ascontiguousarray(batch.npix, np.int32)
    if offsets is None:
        n2 = npix.astype(np.int64) ** 2
        offsets = np.concatenate([[0], np.cumsum(n2)[:-1]]).astype(np.int64)
    offsets = np.ascontiguousarray(offsets, np.int64)
    total = int((offsets + npix.astype(np.int64) ** 2).max()) if len(npix) else 0
    return lm, npix, offsets, total


def psf(obs, method: int, batch, flags: int = 0, pix_sel=None, offsets=None, imag: bool = False) -> np.ndarray:
    """Packed cutouts (float64): the real part of the sum of Eqs. 21-22, or with imag=True
    its imaginary part.  With pix_sel, only those packed indices are filled (rest NaN)."""
    if imag:
        flags = int(flags) | 8
    o = _Obs(obs)
    lm, npix, offs, total = _batch_arrays(batch, offsets)
    out = np.full(total, np.nan)
    sel = None if pix_sel is None else np.ascontiguousarray(pix_sel, np.int64)
    rc = _load().or_psf(*o.args(), int(method), lm.shape[0], _p(lm), _p(npix), float(batch.cell_rad),
                        int(flags), _p(offs), _p(out), 0 if sel is None else sel.size, _p(sel))
    if rc != 0:
        raise ValueError("invalid observation")
    return out


def vjp(obs, method: int, batch, R: np.ndarray, flags: int = 0, offsets=None):
    """(g_lm [npos,2], g_W [nvis]) for cotangent R in the packed output layout."""
    o = _Obs(obs)
    lm, npix, offs, total = _batch_arrays(batch, offsets)
    R = np.ascontiguousarray(R, np.float64)
    assert R.size >= total
    g_lm = np.empty((lm.shape[0], 2))
    g_W = np.empty(nvis(obs))
    rc = _load().or_vjp(*o.args(), int(method), lm.shape[0], _p(lm), _p(npix), float(batch.cell_rad),
                        int(flags), _p(offs), _p(R), _p(g_lm), _p(g_W))
    if rc != 0:
        raise ValueError("invalid observation")
    return g_lm, g_W


def grid_tables(obs, npix: int, cell: float, cells_only: bool = False) -> dict:
    """Position-independent tables of the gridded image-plane form (Eq. 45, Algorithm 1)
    on the npix x npix uv grid of the cutout: S = F{P} (complex [b, a]), per-cell mean
    dt and dnu/nu, per-cell weight sum, and the effective PSF P [j, i].  With
    cells_only, only the per-cell tables (no effective PSF, O(nvis))."""
    o = _Obs(obs)
    N = int(npix)
    S = None if cells_only else np.empty((N, N, 2))
    dt = np.empty((N, N))
    r = np.empty((N, N))
    ws = np.empty((N, N))
    P = None if cells_only else np.empty((N, N))
    if _load().or_grid_tables(*o.args(), N, float(cell), _p(S), _p(dt), _p(r), _p(ws), _p(P)) != 0:
        raise ValueError("invalid observation or grid")
    out = dict(dt=dt, r=r, wsum=ws)
    if not cells_only:
        out.update(S=S[..., 0] + 1j * S[..., 1], P=P)
    return out


def psf_img_grid(obs, lm, npix: int, cell: float, flags: int = 0) -> np.ndarray:
    """Gridded image-plane cutouts [npos, npix, npix] (float64): Re F^-1{F{P} D} with D of
    Algorithm 1 at each uv cell."""
    o = _Obs(obs)
    lm = np.ascontiguousarray(np.asarray(lm, np.float64).reshape(-1, 2))
    N = int(npix)
    out = np.empty((lm.shape[0], N, N))
    if _load().or_psf_img_grid(*o.args(), lm.shape[0], _p(lm), N, float(cell), int(flags), _p(out)) != 0:
        raise ValueError("invalid observation or grid")
    return out


def psf_img_grid_from_tables(tables, lm, npix: int, cell: float, flags: int = 0) -> np.ndarray:
    """psf_img_grid from the tables of grid_tables(obs, npix, cell) (computed once)."""
    N = int(npix)
    lm = np.ascontiguousarray(np.asarray(lm, np.float64).reshape(-1, 2))
    S = np.ascontiguousarray(np.stack([tables["S"].real, tables["S"].imag], axis=-1))
    dt = np.ascontiguousarray(tables["dt"])
    r = np.ascontiguousarray(tables["r"])
    out = np.empty((lm.shape[0], N, N))
    if _load().or_psf_img_grid_tables(N, float(cell), _p(S), _p(dt), _p(r), lm.shape[0], _p(lm), int(flags),
                                      _p(out)) != 0:
        raise ValueError("invalid grid")
    return out


def clean(obs, method, dirty, cell: float, npix: int, gain: float, threshold: float, max_iter: int,
          flags: int = 0, margins: bool = False, centre=(0.0, 0.0), follow=None, facet_psf: bool = False):
    """Hogbom CLEAN with position-dependent PSFs (Algorithm 2), float64.

    dirty [nm, nl]: the dirty image; pixel (x, y) is the direction (l_c + (x - nl/2) cell,
    m_c + (y - nm/2) cell), (l_c, m_c) = centre.  Each iteration takes the peak pixel
    l0 = argmax(I_D) (the first of equal maxima in row-major order), the PSF cutout of
    `method` ('exact' | 'uv' | 'img' | 'img_grid') at l0, normalised to 1 at its centre
    pixel, and subtracts gain * I_D(l0) times it from I_D around l0 (clipped to the image),
    adding gain * I_D(l0) to the model at l0.  As the algorithm's do-while, the first
    iteration always runs and each later one only while the peak exceeds threshold.
    Returns (residual, model, [(pixel index y * nl + x, flux), ...]); with margins, also the
    gap between each iteration's peak and the largest other pixel (how far each argmax
    decision is from a tie).  With follow (a sequence of pixel indices), iteration k takes
    pixel follow[k] instead of the argmax and runs len(follow) iterations without the
    threshold test; the fourth return value is then [(max I_D, I_D at the pixel taken), ...]
    per iteration, so that another implementation's choices can be checked against this
    one's values (where two pixels are within rounding of each other, either is a correct
    argmax).  With facet_psf, the PSF at the image centre `centre` serves every component
    (the faceting approach of Sect. 3.3, Eqs. 57-58) instead of the PSF at each peak."""
    res = np.array(dirty, np.float64, copy=True)
    nm, nl = res.shape
    model = np.zeros_like(res)
    comps, gaps = [], []
    N = int(npix)
    mid = {"exact": EXACT, "uv": UV, "img": IMG}
    tables = grid_tables(obs, N, cell) if method == "img_grid" else None
    Pfix = None
    niter = int(max_iter) if follow is None else len(follow)
    for it in range(niter):
        if follow is None:
            idx = int(np.argmax(res))
        else:
            idx = int(follow[it])
            gaps.append((float(np.max(res)), float(res.flat[idx])))
        y, x = divmod(idx, nl)
        peak = float(res[y, x])
        if follow is None and it > 0 and not peak > threshold:
            break
        if margins and follow is None:
            res[y, x] = -np.inf
            gaps.append(peak - float(np.max(res)))
            res[y, x] = peak
        l0, m0 = centre[0] + (x - nl // 2) * cell, centre[1] + (y - nm // 2) * cell
        if facet_psf:
            l0, m0 = centre
        if facet_psf and Pfix is not None:
            P = Pfix
        else:
            if method == "img_grid":
                P = psf_img_grid_from_tables(tables, [[l0, m0]], N, cell, flags=flags)[0]
            else:
                class _B:
                    pass
                b = _B()
                b.lm = np.array([[l0, m0]])
                b.npix = np.array([N], np.int32)
                b.cell_rad = cell
                P = psf(obs, mid[method], b, flags=flags).reshape(N, N)
            P = P / P[N // 2, N // 2]
            if facet_psf:
                Pfix = P
        g = gain * peak
        y0, x0 = y - N // 2, x - N // 2
        ya, yb = max(y0, 0), min(y0 + N, nm)
        xa, xb = max(x0, 0), min(x0 + N, nl)
        res[ya:yb, xa:xb] -= g * P[ya - y0:yb - y0, xa - x0:xb - x0]
        model[y, x] += g
        comps.append((idx, g))
    return (res, model, comps, gaps) if (margins or follow is not None) else (res, model, comps)


FWHM_STEP = 0.25   # profile sampling step along a direction, in pixels


def _bilinear(P, x, y):
    """P at (column x, row y) by bilinear interpolation; None outside [0, N-1]^2."""
    N = P.shape[0]
    i0, j0 = int(np.floor(x)), int(np.floor(y))
    if i0 < 0 or j0 < 0 or i0 + 1 > N - 1 or j0 + 1 > N - 1:
        if 0 <= x <= N - 1 and 0 <= y <= N - 1 and (x == N - 1 or y == N - 1):
            i0, j0 = min(i0, N - 2), min(j0, N - 2)
        else:
            return None
    fx, fy = x - i0, y - j0
    return ((1 - fx) * (1 - fy) * P[j0, i0] + fx * (1 - fy) * P[j0, i0 + 1]
            + (1 - fx) * fy * P[j0 + 1, i0] + fx * fy * P[j0 + 1, i0 + 1])


def fwhm(P, l0: float, m0: float, cell: float):
    """Full width at half maximum of a cutout along the radial and tangential directions
    of its position (Sect. 2.3, Fig. 3), in direction-cosine units.

    Half maximum h = half the centre pixel P[N/2, N/2] (the PSF at l0).  Along a unit
    direction e (radial (l0, m0)/rho, tangential (-m0, l0)/rho; the l and m axes at
    rho = 0) the profile v(t) = P(centre + t e) is taken by bilinear interpolation at
    t = k FWHM_STEP pixels, k = 1, 2, ..., on each side; the first sample with v <= h
    ends the walk and the crossing is interpolated linearly between it and the previous
    sample.  FWHM = (t+ + t-) cell.  NaN if a walk leaves the cutout first."""
    P = np.asarray(P, np.float64)
    N = P.shape[0]
    c = N // 2
    h = 0.5 * P[c, c]
    rho = float(np.hypot(l0, m0))
    er = (l0 / rho, m0 / rho) if rho > 0 else (1.0, 0.0)
    et = (-er[1], er[0])
    out = []
    for e in (er, et):
        width = 0.0
        for sgn in (1.0, -1.0):
            prev, k, cross = float(P[c, c]), 1, None
            while True:
                t = k * FWHM_STEP
                v = _bilinear(P, c + sgn * t * e[0], c + sgn * t * e[1])
                if v is None:
                    break
                if v <= h:
                    cross = t - FWHM_STEP + FWHM_STEP * (prev - h) / (prev - v)
                    break
                prev, k = v, k + 1
            if cross is None:
                width = np.nan
                break
            width += cross
        out.append(width * cell)
    return tuple(out)
