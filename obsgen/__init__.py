"""Seeded synthetic interferometric observations and PSF position batches.

This module only builds *inputs*: antenna layouts, baseline uvw tracks, channel
tables, averaging intervals and sky positions.  It holds none of the smeared-PSF
arithmetic (no binning, no decorrelation, no Fourier sums); both the FP64
oracle and the CUDA library consume what it returns, and neither shares any
other code.

Geometry follows the textbook local-ENU -> equatorial XYZ -> (u, v, w) chain
(Thompson, Moran & Swenson, the reference the paper cites for Eq. 1), evaluated
in float64.  Baseline vectors are q - p for antenna pairs p < q, in metres;
the paper converts them to wavelengths with u = u_m * nu / c (Sect. 2.1).

The stand-ins for the paper's simulated MeerKAT data (Sect. 4; the real layout
and datasets are not available) are the five workloads defined in ``CONFIGS``:
antennas uniform in a disk (r = R*sqrt(U), phi = 2*pi*U), latitude -30.7 deg,
declination -30 deg, the track centred on transit, raw samples of 1 s.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

OMEGA_E = 7.2921150e-5          # sidereal rotation rate [rad/s]
ARCSEC = math.pi / (180.0 * 3600.0)
DEG = math.pi / 180.0
SEED_BASE = 20200914
ARRAY_SEED = SEED_BASE + 2      # the 64-antenna array shared by workloads 2-5


@dataclasses.dataclass
class Observation:
    """Raw (un-averaged) observation in the C-ABI's layout (``psf_obs_t``)."""
    uvw_m: np.ndarray            # float64 [nbl, ntime, 3], metres
    time_s: np.ndarray           # float64 [ntime], raw sample centres
    freq_hz: np.ndarray          # float64 [nchan], raw channel centres
    chan_width_hz: np.ndarray    # float64 [nchan]
    tavg: np.ndarray             # int32 [nbl], raw samples per averaged time bin
    favg: int                    # raw channels per averaged channel
    weights: Optional[np.ndarray] = None   # float32 [nvis] in plan order, or None
    enu_m: Optional[np.ndarray] = None     # antenna positions (for reference only)
    time_window: Optional[np.ndarray] = None   # float32 [sum(tavg)]: per baseline, over a bin's samples
    chan_window: Optional[np.ndarray] = None   # float32 [nbl, favg]: per baseline, over an output channel's raw channels

    @property
    def nbl(self) -> int:
        return int(self.uvw_m.shape[0])

    @property
    def ntime(self) -> int:
        return int(self.uvw_m.shape[1])

    @property
    def nchan(self) -> int:
        return int(self.freq_hz.shape[0])

    def nvis(self) -> int:
        """Number of averaged visibilities (the interface's counting rule)."""
        nbins = (self.ntime // self.tavg.astype(np.int64)).sum()
        return int(nbins) * (self.nchan // self.favg)


@dataclasses.dataclass
class Batch:
    """Cutout requests: positions, square sizes and the common pixel size."""
    lm: np.ndarray               # float64 [npos, 2] direction cosines
    npix: np.ndarray             # int32 [npos], even sizes
    cell_rad: float              # pixel size (direction cosine units)

    @property
    def npos(self) -> int:
        return int(self.lm.shape[0])

    def total_pixels(self) -> int:
        return int((self.npix.astype(np.int64) ** 2).sum())


def antennas_disk(rng: np.random.Generator, n: int, radius_m: float) -> np.ndarray:
    """n antennas uniform in a disk of the given radius, ENU metres, Up = 0."""
    r = radius_m * np.sqrt(rng.random(n))
    phi = 2.0 * np.pi * rng.random(n)
    return np.stack([r * np.cos(phi), r * np.sin(phi), np.zeros(n)], axis=1)


def baseline_pairs(nant: int) -> np.ndarray:
    p, q = np.triu_indices(nant, k=1)
    return np.stack([p, q], axis=1)


def uvw_tracks(enu: np.ndarray, lat_rad: float, dec_rad: float,
               time_s: np.ndarray) -> np.ndarray:
    """Baseline (q - p) uvw tracks in metres, float64 [nbl, ntime, 3]."""
    pairs = baseline_pairs(enu.shape[0])
    b = enu[pairs[:, 1]] - enu[pairs[:, 0]]                  # [nbl, 3] ENU
    e, n, up = b[:, 0], b[:, 1], b[:, 2]
    sl, cl = math.sin(lat_rad), math.cos(lat_rad)
    X = -sl * n + cl * up
    Y = e
    Z = cl * n + sl * up
    H = OMEGA_E * time_s                                     # hour angle [rad]
    sh, ch = np.sin(H)[None, :], np.cos(H)[None, :]
    sd, cd = math.sin(dec_rad), math.cos(dec_rad)
    X, Y, Z = X[:, None], Y[:, None], Z[:, None]
    u = sh * X + ch * Y
    v = -sd * ch * X + sd * sh * Y + cd * Z
    w = cd * ch * X - cd * sh * Y + sd * Z
    return np.ascontiguousarray(np.stack([u, v, w], axis=2))


def raw_times(duration_s: float, dt_s: float) -> np.ndarray:
    ntime = int(round(duration_s / dt_s))
    return -0.5 * duration_s + (np.arange(ntime) + 0.5) * dt_s


def raw_channels(start_hz: float, width_hz: float, nchan: int):
    freq = start_hz + (np.arange(nchan) + 0.5) * width_hz
    return freq, np.full(nchan, width_hz)


def meerkat_like_array() -> np.ndarray:
    """64 antennas: 32 uniform within 1 km and 32 within 8 km (seeded)."""
    rng = np.random.default_rng(ARRAY_SEED)
    inner = antennas_disk(rng, 32, 1000.0)
    outer = antennas_disk(rng, 32, 8000.0)
    return np.concatenate([inner, outer], axis=0)


def bda_tavg(enu: np.ndarray, dt_ref_s: float, lo: int, hi: int) -> np.ndarray:
    """Baseline-dependent averaging: tavg ~ dt_ref * b_med / |b|, clamped."""
    pairs = baseline_pairs(enu.shape[0])
    b = enu[pairs[:, 1]] - enu[pairs[:, 0]]
    blen = np.hypot(b[:, 0], b[:, 1])
    bmed = float(np.median(blen))
    t = np.rint(dt_ref_s * bmed / np.maximum(blen, 1e-9))
    return np.clip(t, lo, hi).astype(np.int32)


def _obs(enu, duration_s, tavg, f0, df, nchan, favg, unit_weights=False,
         lat=-30.7 * DEG, dec=-30.0 * DEG):
    t = raw_times(duration_s, 1.0)
    uvw = uvw_tracks(enu, lat, dec, t)
    freq, width = raw_channels(f0, df, nchan)
    nbl = uvw.shape[0]
    tavg = np.broadcast_to(np.asarray(tavg, dtype=np.int32), (nbl,)).copy()
    obs = Observation(uvw, t, freq, width, tavg, favg, None, enu)
    if unit_weights:
        obs.weights = np.ones(obs.nvis(), dtype=np.float32)
    return obs


# ---------------------------------------------------------------- workloads
def config1_obs() -> Observation:
    """16 antennas in a 1 km disk, 1 h at 1 s averaged 10:1, 4 x 1 MHz at 1.4 GHz."""
    rng = np.random.default_rng(SEED_BASE + 1)
    enu = antennas_disk(rng, 16, 1000.0)
    return _obs(enu, 3600.0, 10, 1.400e9, 1.0e6, 4, 1, unit_weights=True)


def config1_batch() -> Batch:
    return Batch(np.array([[0.02, 0.02]]), np.array([64], np.int32), 2.0 * ARCSEC)


def config2_obs(hours: float = 4.0) -> Observation:
    """64-antenna array, 4 h at 1 s averaged 8:1, 16 x 0.836 MHz from 856 MHz."""
    return _obs(meerkat_like_array(), hours * 3600.0, 8, 856e6, 0.836e6, 16, 1)


def config2_batch() -> Batch:
    return Batch(np.array([[0.03, 0.03]]), np.array([128], np.int32), 1.5 * ARCSEC)


def config3_obs() -> Observation:
    """64-antenna array, 2 h, 8 channels, baseline-dependent 2..30 s averaging."""
    enu = meerkat_like_array()
    return _obs(enu, 2 * 3600.0, bda_tavg(enu, 8.0, 2, 30), 856e6, 0.836e6, 8, 1)


def config3_batch(npos: int = 4096, seed: int = SEED_BASE + 3) -> Batch:
    rng = np.random.default_rng(seed)
    s = math.sin(1.0 * DEG)
    lm = rng.uniform(-s, s, size=(npos, 2))
    npix = rng.choice(np.array([32, 64, 128, 256], np.int32), size=npos)
    return Batch(lm, npix.astype(np.int32), 1.5 * ARCSEC)


def config4_batch(npos: int = 256, seed: int = SEED_BASE + 4) -> Batch:
    rng = np.random.default_rng(seed)
    s = math.sin(1.0 * DEG)
    lm = rng.uniform(-s, s, size=(npos, 2))
    return Batch(lm, np.full(npos, 64, np.int32), 1.5 * ARCSEC)


def config5_obs() -> Observation:
    """64-antenna array, 4 h at 1 s averaged 8:1, 256 x 3.34375 MHz averaged 4:1."""
    return _obs(meerkat_like_array(), 4 * 3600.0, 8, 856e6, 3.34375e6, 256, 4)


def config5_batch(nrad: int = 128, nang: int = 128) -> Batch:
    a = np.arange(nrad)
    r = 3.0 * DEG * (a + 1) / nrad
    phi = 2.0 * np.pi * np.arange(nang) / nang
    R, PHI = np.meshgrid(r, phi, indexing="ij")
    lm = np.stack([np.sin(R) * np.cos(PHI), np.sin(R) * np.sin(PHI)], axis=-1).reshape(-1, 2)
    return Batch(lm, np.full(lm.shape[0], 64, np.int32), 1.5 * ARCSEC)


# ------------------------------------------------------------ small cases
def fig3_obs(cf: str = "20x40", every: int = 1) -> Observation:
    """The setting of the paper's FWHM figure on the 64-antenna array (every `every`-th
    antenna): 2 h of 1 s samples and 6 MHz of 50 kHz channels centred on 1.4 GHz, averaged
    10 s x 1 MHz ("10x20") or 20 s x 2 MHz ("20x40")."""
    tavg, favg = {"10x20": (10, 20), "20x40": (20, 40)}[cf]
    return _obs(meerkat_like_array()[::every], 2 * 3600.0, tavg, 1.397e9, 50e3, 120, favg)


def fig3_batch(npix: int = 64, cell_arcsec: float = 1.0, radii_deg=(0.0, 0.5, 1.0, 1.5, 2.0, 2.5, 3.0, 3.5, 4.0, 4.5),
               nang: int = 8) -> Batch:
    """Positions at the given distances from the phase centre, nang position angles each
    (one at the centre), as in the FWHM-against-distance figure."""
    lm = []
    for r in radii_deg:
        for k in range(1 if r == 0 else nang):
            phi = 2.0 * np.pi * (k + 0.5) / nang
            s = math.sin(r * DEG)
            lm.append((s * math.cos(phi), s * math.sin(phi)))
    lm = np.array(lm)
    return Batch(lm, np.full(len(lm), npix, np.int32), cell_arcsec * ARCSEC)


def bd_windows(obs: Observation, strength: float = 1.0):
    """Seeded-free example of baseline-dependent windows (input data for the windowed
    average): per baseline a Gaussian taper over the tavg[b] samples of a bin and over the
    favg raw channels of an output channel, narrower on longer baselines (sigma = n /
    (1 + strength |b| / b_median) samples), as baseline-dependent windows are.  Returns
    (time_window [sum(tavg)], chan_window [nbl, favg]) as float32."""
    blen = np.linalg.norm(obs.uvw_m.mean(axis=1), axis=1)
    med = max(float(np.median(blen)), 1e-9)
    tw, cw = [], np.empty((obs.nbl, obs.favg), np.float32)
    for b in range(obs.nbl):
        scale = 1.0 + strength * blen[b] / med
        n = int(obs.tavg[b])
        k = np.arange(n) - 0.5 * (n - 1)
        tw.append(np.exp(-0.5 * (k / (n / scale)) ** 2))
        f = np.arange(obs.favg) - 0.5 * (obs.favg - 1)
        cw[b] = np.exp(-0.5 * (f / (max(obs.favg, 1) / scale)) ** 2)
    return np.concatenate(tw).astype(np.float32), cw


def tiny_obs(seed: int = 7, nant: int = 4, ntime: int = 24, nchan: int = 4,
             tavg=4, favg: int = 2, f0: float = 1.2e9, df: float = 2e6,
             dt: float = 2.0, radius_m: float = 3000.0,
             weights: bool = False) -> Observation:
    """A few baselines and samples, for brute-force and edge-case checks."""
    rng = np.random.default_rng(seed)
    enu = antennas_disk(rng, nant, radius_m)
    t = -0.5 * ntime * dt + (np.arange(ntime) + 0.5) * dt
    uvw = uvw_tracks(enu, -30.7 * DEG, -30.0 * DEG, t)
    freq, width = raw_channels(f0, df, nchan)
    nbl = uvw.shape[0]
    tav = np.broadcast_to(np.asarray(tavg, dtype=np.int32), (nbl,)).copy()
    obs = Observation(uvw, t, freq, width, tav, favg, None, enu)
    if weights:
        obs.weights = rng.uniform(0.5, 2.0, obs.nvis()).astype(np.float32)
    return obs


def random_batch(seed: int, npos: int, sizes=(32, 64), radius: float = 0.03,
                 cell_rad: float = 1.5 * ARCSEC) -> Batch:
    rng = np.random.default_rng(seed)
    lm = rng.uniform(-radius, radius, size=(npos, 2))
    npix = rng.choice(np.asarray(sizes, np.int32), size=npos).astype(np.int32)
    return Batch(lm, npix, cell_rad)


def linear_track_obs(u0_m: float, rate_m_per_s: float, ntime: int, dt: float,
                     tavg: int, freq_hz, width_hz, favg: int) -> Observation:
    """One baseline whose track is u(t) = u0 + rate * t, v = w = 0."""
    t = (np.arange(ntime) + 0.5) * dt
    uvw = np.zeros((1, ntime, 3))
    uvw[0, :, 0] = u0_m + rate_m_per_s * t
    freq = np.asarray(freq_hz, dtype=np.float64)
    width = np.broadcast_to(np.asarray(width_hz, dtype=np.float64), freq.shape).copy()
    return Observation(uvw, t, freq, width, np.array([tavg], np.int32), favg)


def concat_pixels(batch: Batch) -> np.ndarray:
    """Output offsets of the packed layout (prefix sums of N^2)."""
    n2 = batch.npix.astype(np.int64) ** 2
    return np.concatenate([[0], np.cumsum(n2)[:-1]]).astype(np.int64)
