"""Seeded synthetic MWA-shaped cadences.

This module draws random numbers and builds the array geometry.  It holds none
of the calibrate-and-peel arithmetic (no phase, no Jones product, no average,
no solve): visibilities are formed elsewhere from what it returns.

Random numbers
--------------
Every draw is counter-based: the n-th 64-bit word of stream ``s`` under seed
``seed`` is the SplitMix64 output function (Steele, Lea & Flood, OOPSLA 2014;
the public-domain reference ``splitmix64.c`` by S. Vigna) applied to the
counter ``x = ((seed * 256 + s) * 2**40 + n + 1) * 0x9E3779B97F4A7C15 mod 2**64``.
Streams are 2**40 words apart, so any sub-range of any stream can be drawn
without the rest.  Uniforms are ``(z >> 11) * 2**-53``; normals come in
Box-Muller pairs from words ``2i`` and ``2i+1``.

Workload shapes (the MWA vital statistics of Section 2 / Table 1 of the paper:
512 tiles, 130816 baselines, 768 channels of 40 kHz, 8 s cadence) and the
readings used where the paper is silent:

* antennas uniform in a disc of radius 750 m, flat (U = 0);
* phase centre at declination = site latitude (-26.703 deg), hour angle
  H(t) = omega_E * t, t = 0 .. N_t-1 seconds, uvw by the standard
  ENU -> XYZ -> uvw rotation (Thompson, Moran & Swenson, ch. 4);
* channels nu_c = nu_0 + c * 40 kHz;
* sources l, m ~ U(-0.3, 0.3), fluxes dN/dS ~ S^-1.6 on [1, 20] Jy by inverse
  CDF, peel order = descending flux;
* true Jones = I + CN(0, 0.1^2) per complex entry (Re and Im each variance
  0.005), one per (source, antenna);
* noise sigma = 0.01 Jy on Re and Im of every polarisation product;
* optional position perturbation N(0, (1 arcmin)^2) per coordinate.
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, replace

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

OMEGA_EARTH = 7.2921159e-5          # rad / s (sidereal)
MWA_LAT_DEG = -26.703               # site latitude; not printed in the paper

# stream identifiers (fixed order: positions, antennas, sources, Jones, noise;
# then the Jones slopes over the band, drawn only by jones_slope())
S_ANT, S_SRC, S_JONES, S_NOISE, S_POS, S_SLOPE = 1, 2, 3, 4, 5, 6

_CHUNK = 1 << 20     # noise elements per work item


def splitmix64(seed: int, stream: int, idx) -> np.ndarray:
    """SplitMix64 output for counters ``idx`` of ``stream`` (uint64 array)."""
    idx = np.asarray(idx, dtype=np.uint64)
    base = np.uint64(((int(seed) * 256 + int(stream)) << 40) & 0xFFFFFFFFFFFFFFFF)
    with np.errstate(over="ignore"):
        z = (base + idx + np.uint64(1)) * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """n uniforms in [0, 1) from words offset .. offset+n-1."""
    z = splitmix64(seed, stream, np.arange(offset, offset + n, dtype=np.uint64))
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normals(seed: int, stream: int, idx) -> np.ndarray:
    """Standard normals with global indices ``idx`` (Box-Muller, FP64)."""
    idx = np.asarray(idx, dtype=np.int64)
    pair = (idx // 2).astype(np.uint64)
    z1 = splitmix64(seed, stream, pair * np.uint64(2))
    z2 = splitmix64(seed, stream, pair * np.uint64(2) + np.uint64(1))
    u1 = ((z1 >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)   # (0, 1]
    u2 = (z2 >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)           # [0, 1)
    r = np.sqrt(-2.0 * np.log(u1))
    return np.where(idx % 2 == 0, r * np.cos(2.0 * math.pi * u2), r * np.sin(2.0 * math.pi * u2))


def n_baselines(n_ant: int) -> int:
    return n_ant * (n_ant - 1) // 2


def baseline_pairs(n_ant: int) -> np.ndarray:
    """[n_bl][2] antenna pairs (i < j) in row-major upper-triangle order."""
    i, j = np.triu_indices(n_ant, k=1)
    return np.stack([i, j], axis=1).astype(np.int32)


@dataclass(frozen=True)
class Cadence:
    n_ant: int
    n_chan: int
    n_time: int
    n_src: int
    freq0_hz: float = 150e6
    dfreq_hz: float = 40e3
    dt_s: float = 1.0
    radius_m: float = 750.0
    lat_deg: float = MWA_LAT_DEG
    lmax: float = 0.3
    smin: float = 1.0
    smax: float = 20.0
    slope: float = -1.6
    jones_sigma: float = 0.1
    noise_sigma: float = 0.01
    pos_sigma_rad: float = 0.0
    precision: str = "mixed"        # "mixed" (complex64 cube) or "fp64" (complex128)
    seed: int = 100300

    @property
    def n_bl(self) -> int:
        return n_baselines(self.n_ant)

    @property
    def n_vis(self) -> int:
        return self.n_time * self.n_bl * self.n_chan

    def with_(self, **kw) -> "Cadence":
        return replace(self, **kw)

    # ---- geometry -------------------------------------------------------
    def ant_enu(self) -> np.ndarray:
        """[n_ant][3] east, north, up in metres (uniform in a flat disc)."""
        u = uniform01(self.seed, S_ANT, 2 * self.n_ant).reshape(self.n_ant, 2)
        r = self.radius_m * np.sqrt(u[:, 0])
        th = 2.0 * math.pi * u[:, 1]
        return np.stack([r * np.cos(th), r * np.sin(th), np.zeros(self.n_ant)], axis=1)

    def hour_angles(self) -> np.ndarray:
        return OMEGA_EARTH * self.dt_s * np.arange(self.n_time, dtype=np.float64)

    def uvw(self) -> np.ndarray:
        """[n_time][n_ant][3] antenna uvw in metres; baseline uvw = uvw_i - uvw_j."""
        enu = self.ant_enu()
        lat = math.radians(self.lat_deg)
        dec = lat
        e, n, up = enu[:, 0], enu[:, 1], enu[:, 2]
        x = -math.sin(lat) * n + math.cos(lat) * up
        y = e
        z = math.cos(lat) * n + math.sin(lat) * up
        out = np.empty((self.n_time, self.n_ant, 3))
        for t, h in enumerate(self.hour_angles()):
            sh, ch = math.sin(h), math.cos(h)
            sd, cd = math.sin(dec), math.cos(dec)
            out[t, :, 0] = sh * x + ch * y
            out[t, :, 1] = -sd * ch * x + sd * sh * y + cd * z
            out[t, :, 2] = cd * ch * x - cd * sh * y + sd * z
        return out

    def freqs(self) -> np.ndarray:
        return self.freq0_hz + self.dfreq_hz * np.arange(self.n_chan, dtype=np.float64)

    # ---- sky ------------------------------------------------------------
    def sources(self) -> np.ndarray:
        """[n_src][3] (l, m, S Jy), sorted by descending S (the peel order)."""
        u = uniform01(self.seed, S_SRC, 3 * self.n_src).reshape(self.n_src, 3)
        l = self.lmax * (2.0 * u[:, 0] - 1.0)
        m = self.lmax * (2.0 * u[:, 1] - 1.0)
        a = self.slope + 1.0                      # CDF ~ S^(slope+1)
        lo, hi = self.smin ** a, self.smax ** a
        s = (lo + u[:, 2] * (hi - lo)) ** (1.0 / a)
        order = np.argsort(-s, kind="stable")
        return np.stack([l, m, s], axis=1)[order]

    def perturbed_sources(self) -> np.ndarray:
        """sources() with (l, m) moved by N(0, pos_sigma_rad^2) per coordinate."""
        src = self.sources().copy()
        d = normals(self.seed, S_POS, np.arange(2 * self.n_src)).reshape(self.n_src, 2)
        src[:, :2] += self.pos_sigma_rad * d
        return src

    def jones(self) -> np.ndarray:
        """[n_src][n_ant][4] complex128 true Jones [XX, XY, YX, YY]."""
        k = self.n_src * self.n_ant * 4
        g = normals(self.seed, S_JONES, np.arange(2 * k)).reshape(self.n_src, self.n_ant, 4, 2)
        sd = self.jones_sigma / math.sqrt(2.0)
        j = sd * (g[..., 0] + 1j * g[..., 1])
        j[..., 0] += 1.0
        j[..., 3] += 1.0
        return j

    def jones_slope(self, sigma: float = 0.2) -> np.ndarray:
        """[n_src][n_ant][4] complex128 Jones slopes H for gains linear in frequency,
        J(c) = jones() + x_c H with x_c the channel's offset from the band centre in
        band widths (|x_c| <= 1/2): CN(0, sigma^2) per entry."""
        k = self.n_src * self.n_ant * 4
        g = normals(self.seed, S_SLOPE, np.arange(2 * k)).reshape(self.n_src, self.n_ant, 4, 2)
        sd = sigma / math.sqrt(2.0)
        return sd * (g[..., 0] + 1j * g[..., 1])

    def noise(self, index=None) -> np.ndarray:
        """Complex noise, sigma on Re and Im.  ``index`` are flat complex-element
        indices into the [n_time][n_bl][n_chan][4] cube (all of it if None)."""
        if index is None:
            index = np.arange(self.n_vis * 4, dtype=np.int64)
        index = np.asarray(index, dtype=np.int64).ravel()
        # element i takes normals 2i (Re) and 2i+1 (Im): the cosine and sine of
        # one Box-Muller pair (pair index i), the same values as normals() gives
        out = np.empty(index.shape, np.complex128)
        sigma = self.noise_sigma

        def fill(a):
            pair = index[a:a + _CHUNK].astype(np.uint64)
            z1 = splitmix64(self.seed, S_NOISE, pair * np.uint64(2))
            z2 = splitmix64(self.seed, S_NOISE, pair * np.uint64(2) + np.uint64(1))
            u1 = ((z1 >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)
            u2 = (z2 >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
            r = np.sqrt(-2.0 * np.log(u1))
            ang = 2.0 * math.pi * u2
            o = out[a:a + _CHUNK]
            o.real = r * np.cos(ang)
            o.imag = r * np.sin(ang)
            o.real *= sigma
            o.imag *= sigma

        starts = range(0, index.size, _CHUNK)
        if index.size > _CHUNK:
            with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
                list(ex.map(fill, starts))
        else:
            for a in starts:
                fill(a)
        return out


def noise_cube(cad: Cadence) -> np.ndarray:
    """[n_time][n_bl][n_chan][4] complex128 noise for the whole cadence."""
    return cad.noise().reshape(cad.n_time, cad.n_bl, cad.n_chan, 4)


# The five workloads: MWA-shaped cadences (Table 1 of the paper gives the
# 512-tile / 768-channel / 40 kHz / 8 s shape).  Seeds: 1003*100 + index.
CONFIGS = {
    1: Cadence(32, 16, 8, 5, freq0_hz=150e6, precision="fp64", seed=100301),
    2: Cadence(128, 128, 8, 50, freq0_hz=150e6, seed=100302),
    3: Cadence(512, 768, 8, 1000, freq0_hz=167e6, seed=100303),
    4: Cadence(128, 256, 8, 100, freq0_hz=150e6, pos_sigma_rad=2.909e-4, seed=100304),
    5: Cadence(512, 768, 8, 300, freq0_hz=167e6, pos_sigma_rad=2.909e-4, seed=100305),
}


def config(i: int, **kw) -> Cadence:
    c = CONFIGS[i]
    return c.with_(**kw) if kw else c
