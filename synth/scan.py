"""Seeded synthetic scans, noise bands, skies and timelines.

Shapes and statistics follow the paper's ground-based simulations (Sect. 5):
a constant-elevation back-and-forth raster over a flat patch, a half-wave
plate angle per sample, a Gaussian I/Q/U sky, and noise with a 1/f spectrum
P(f) = sigma^2 (1 + (f_knee/f)^alpha) that is stationary within each
(detector, interval) block.  The inverse-noise weight handed to the solver is
a symmetric banded Toeplitz matrix per block; its band is built here and
passed to both sides as data, so the oracle and the CUDA path consume the
identical coefficients.

Nothing here applies the pointing transpose, the band to a timeline, or any
preconditioner: those are the method and live on each side separately.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import os

import numpy as np

FS_HZ = 100.0          # sampling rate of every configured workload
SCAN_SPEED_PX = 0.14   # raster speed in pixels per sample (0.4 deg/s, ~1.7' pixels, 100 Hz)


@dataclass
class Scan:
    """Pointing and noise model of one scan (one map-making problem).

    Samples are stored detector-major: detector ``d`` owns samples
    ``[d*n_t, (d+1)*n_t)``.  Each detector timeline is cut into ``n_int`` equal
    stationary intervals; a block is one (detector, interval) pair and
    ``block_off`` holds the block boundaries.  ``band[block_band[b]]`` holds
    the Toeplitz coefficients c_0..c_lambda of block ``b``.
    """
    nx: int
    ny: int
    n_det: int
    n_t: int
    n_int: int
    half_bw: int
    pix: np.ndarray          # int32 [N]; -1 marks a flagged sample
    psi: np.ndarray          # float32 [N]; HWP angle in radians, [0, pi)
    block_off: np.ndarray    # int64 [n_blocks + 1]
    block_band: np.ndarray   # int32 [n_blocks]
    band: np.ndarray         # float64 [n_bands, half_bw + 1]
    f_knee: np.ndarray       # float64 [n_det]
    seed: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def n_pix(self) -> int:
        return self.nx * self.ny

    @property
    def n_samples(self) -> int:
        return int(self.pix.shape[0])

    @property
    def n_blocks(self) -> int:
        return int(self.block_off.shape[0] - 1)

    @property
    def n_bands(self) -> int:
        return int(self.band.shape[0])


def _next_pow2(n: int) -> int:
    p = 1
    while p < n:
        p *= 2
    return p


def toeplitz_band(half_bw: int, f_knee: float, alpha: float = 1.0,
                  sigma: float = 1.0, fs: float = FS_HZ) -> np.ndarray:
    """Coefficients c_0..c_lambda of a banded inverse-noise Toeplitz matrix.

    c_k is the inverse DFT of 1/P(f) on an L-point grid (L the power of two
    at least 8*lambda, at least 16), with the f = 0 bin set to 1/P(f_1), cut
    to |k| <= lambda.  The symbol S(w) = c_0 + 2 sum_k c_k cos(k w) of the cut
    band is then checked on a grid of 64*lambda points; if it is not positive
    c_0 is raised until it is, so every finite section of the matrix is SPD.
    """
    L = max(16, _next_pow2(8 * max(half_bw, 1)))
    f = np.fft.rfftfreq(L, 1.0 / fs)
    fpos = np.where(f > 0, f, f[1])
    P = sigma ** 2 * (1.0 + (f_knee / fpos) ** alpha) if f_knee > 0 else np.full_like(f, sigma ** 2)
    c = np.fft.irfft(1.0 / P, n=L)
    band = np.array(c[:half_bw + 1], dtype=np.float64)
    if half_bw > 0:
        M = _next_pow2(64 * half_bw)
        h = np.zeros(M)
        h[:half_bw + 1] = band
        h[M - half_bw:] = band[1:][::-1]
        S = np.fft.rfft(h).real
        smin = float(S.min())
        if smin <= 0.0:
            band[0] += -smin + 1e-6 * band[0]
    return band


def _each(fn, items, n_samples):
    """fn(i) for every item; on several host threads for large inputs (numpy releases the GIL in the
    element-wise and FFT work, and every item writes its own slice, so the values do not depend on
    the order)."""
    items = list(items)
    if n_samples < (1 << 22) or len(items) < 2:
        for i in items:
            fn(i)
        return
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1, len(items))) as ex:
        list(ex.map(fn, items))


def make_scan(nx: int, ny: int, n_det: int, n_t: int, n_int: int, half_bw: int,
              f_knee=1.0, alpha: float = 1.0, sigma: float = 1.0, seed: int = 0,
              speed: float = SCAN_SPEED_PX, flag_frac: float = 0.0,
              fs: float = FS_HZ, hwp: bool = True) -> Scan:
    """Back-and-forth raster scan of an nx x ny patch by ``n_det`` detectors.

    Azimuth: a triangle wave over [0, nx) at ``speed`` pixels per sample with
    a random phase per detector.  Elevation: a slow drift that crosses the
    patch once per detector timeline, with detector offsets spread over a
    quarter of the patch height.  HWP angle psi ~ U[0, pi) i.i.d. per sample;
    with ``hwp=False`` there is no half-wave plate: detector d keeps the
    polarisation angle (d mod 4) pi/4 of its place in the focal plane, turned
    slowly by the sky rotation (pi/4 over the timeline), so the polarised
    signal varies on scan time scales as in the paper's scans.
    ``f_knee`` is a scalar or a (lo, hi) range drawn uniformly per detector.
    A fraction ``flag_frac`` of samples is flagged (pixel -1).
    """
    if n_t % n_int != 0:
        raise ValueError("n_t must be a multiple of n_int")
    rng = np.random.default_rng(seed)
    N = n_det * n_t
    pix = np.empty(N, dtype=np.int32)
    t = np.arange(n_t, dtype=np.float64)
    x0 = rng.uniform(0.0, 2.0 * nx, size=n_det)
    y0 = rng.uniform(0.0, ny)
    st = speed * t
    ty = t * (ny / n_t)

    def raster(d):
        pos = np.mod(x0[d] + st, 2.0 * nx)
        np.subtract(2.0 * nx, pos, out=pos, where=pos >= nx)
        ix = np.minimum(pos.astype(np.int32), nx - 1)
        oy = d * (ny / 4.0) / n_det
        y = np.mod(y0 + oy + ty, ny)
        iy = np.minimum(y.astype(np.int32), ny - 1)
        np.multiply(iy, nx, out=iy)
        np.add(iy, ix, out=pix[d * n_t:(d + 1) * n_t])

    _each(raster, range(n_det), N)
    psi = rng.random(N, dtype=np.float32)
    psi *= np.float32(np.pi)
    if not hwp:
        rot = (np.pi / 4.0) * t / n_t
        for d in range(n_det):
            psi[d * n_t:(d + 1) * n_t] = np.mod((d % 4) * (np.pi / 4.0) + rot, np.pi).astype(np.float32)
    np.minimum(psi, np.nextafter(np.float32(np.pi), np.float32(0)), out=psi)
    if flag_frac > 0:
        pix[rng.random(N, dtype=np.float32) < flag_frac] = -1
    if np.ndim(f_knee) == 0:
        fk = np.full(n_det, float(f_knee))
    else:
        lo, hi = f_knee
        fk = rng.uniform(lo, hi, size=n_det)
    blen = n_t // n_int
    block_off = np.arange(n_det * n_int + 1, dtype=np.int64) * blen
    block_band = np.repeat(np.arange(n_det, dtype=np.int32), n_int)
    band = np.stack([toeplitz_band(half_bw, float(fk[d]), alpha, sigma, fs) for d in range(n_det)])
    return Scan(nx=nx, ny=ny, n_det=n_det, n_t=n_t, n_int=n_int, half_bw=half_bw,
                pix=pix, psi=psi, block_off=block_off, block_band=block_band,
                band=band, f_knee=fk, seed=seed,
                meta=dict(alpha=alpha, sigma=sigma, fs=fs, speed=speed, flag_frac=flag_frac, x0=x0, hwp=hwp))


# Ground-pickup bins of 0.08 deg (Sect. 5) with ~1.7' pixels: 2.8 pixels of azimuth per bin.
AZ_BIN_PX = 0.08 * 60.0 / 1.7


def make_templates(scan: Scan, bin_px: float = AZ_BIN_PX):
    """Scan geometry of the template filters: subscans and azimuth bins.

    A subscan is one azimuth sweep of the back-and-forth raster (the samples
    between two turnarounds), cut at block edges so every subscan lies in
    one stationary block.  The azimuth bin of a sample is floor(az / bin_px)
    over the sweep range [0, nx).  Returns (sub_off int64 [n_sub + 1],
    az_bin int32 [N], n_az_bins).
    """
    x0 = np.asarray(scan.meta["x0"], dtype=np.float64)
    speed = float(scan.meta.get("speed", SCAN_SPEED_PX))
    nx, n_t = scan.nx, scan.n_t
    t = np.arange(n_t, dtype=np.float64)
    n_bins = int(np.ceil(nx / bin_px))
    az_bin = np.empty(scan.n_samples, dtype=np.int32)
    cuts = [np.asarray(scan.block_off, dtype=np.int64)] + [None] * scan.n_det

    def sweeps(d):
        raw = x0[d] + speed * t
        sweep = np.floor(raw / nx).astype(np.int64)
        pos = np.mod(raw, 2.0 * nx)
        np.subtract(2.0 * nx, pos, out=pos, where=pos >= nx)
        az_bin[d * n_t:(d + 1) * n_t] = np.minimum((pos / bin_px).astype(np.int32), n_bins - 1)
        turns = np.nonzero(np.diff(sweep))[0] + 1
        cuts[d + 1] = turns.astype(np.int64) + d * n_t

    _each(sweeps, range(scan.n_det), scan.n_samples)
    sub_off = np.unique(np.concatenate(cuts))
    return sub_off, az_bin, n_bins


def make_sky(n_pix: int, seed: int = 0, sigma_i: float = 1.0, sigma_qu: float = 0.1) -> np.ndarray:
    """Gaussian sky [n_pix, 3]: I ~ N(0, sigma_i^2), Q, U ~ N(0, sigma_qu^2)."""
    rng = np.random.default_rng(seed + 7919)
    s = rng.standard_normal((n_pix, 3))
    s[:, 0] *= sigma_i
    s[:, 1:] *= sigma_qu
    return s


def make_noise(scan: Scan, seed: int = 0) -> np.ndarray:
    """1/f noise per stationary block, shaped in Fourier space (float64 [N]).

    For each block, white N(0, 1) samples are multiplied in the rFFT domain
    by sqrt(1 + (f_knee/f)^alpha) (the f = 0 bin takes the f_1 value) and
    scaled by sigma.  Blocks are independent.
    """
    rng = np.random.default_rng(seed + 104729)
    alpha = scan.meta.get("alpha", 1.0)
    sigma = scan.meta.get("sigma", 1.0)
    fs = scan.meta.get("fs", FS_HZ)
    n = np.empty(scan.n_samples, dtype=np.float64)
    blen = scan.n_t // scan.n_int
    f = np.fft.rfftfreq(blen, 1.0 / fs)
    fpos = np.where(f > 0, f, f[1] if f.shape[0] > 1 else 1.0)
    def shape_block(d):
        fk = float(scan.f_knee[d])
        shape = np.sqrt(1.0 + (fk / fpos) ** alpha) if fk > 0 else np.ones_like(f)
        w = n[d * scan.n_t:(d + 1) * scan.n_t].reshape(scan.n_int, blen)
        w[...] = np.fft.irfft(np.fft.rfft(w, axis=1) * shape, n=blen, axis=1) * sigma

    # the white samples are drawn in detector order first, so the stream is the same however the
    # Fourier shaping below is spread over host cores
    for d in range(scan.n_det):
        n[d * scan.n_t:(d + 1) * scan.n_t] = rng.standard_normal((scan.n_int, blen)).reshape(-1)
    _each(shape_block, range(scan.n_det), scan.n_samples)
    return n


def make_tod(scan: Scan, sky: np.ndarray | None, noise: np.ndarray | None) -> np.ndarray:
    """Timeline d_t = I_p + Q_p cos 2psi_t + U_p sin 2psi_t + n_t (float64 [N]).

    This is the data model the paper simulates (Sect. 2, Eq. datamodel); it
    only synthesises an input.  Flagged samples carry noise only.
    """
    N = scan.n_samples
    d = np.zeros(N, dtype=np.float64)
    if sky is not None:
        chunk = 1 << 20

        def fill(a):
            b = min(N, a + chunk)
            pix = scan.pix[a:b]
            ok = pix >= 0
            p = pix[ok]
            ang = 2.0 * scan.psi[a:b][ok].astype(np.float64)
            seg = d[a:b]
            seg[ok] = sky[p, 0] + sky[p, 1] * np.cos(ang) + sky[p, 2] * np.sin(ang)

        # chunks are independent (numpy releases the GIL in the element-wise work): the same values
        # as a serial loop, on several host cores
        _each(fill, range(0, N, chunk), N)
    if noise is not None:
        d += noise
    return d


def mc_lengths(n_rhs: int, lo: int, hi: int, seed: int = 0) -> np.ndarray:
    """Per right-hand-side timeline lengths (samples per detector), U[lo, hi]."""
    rng = np.random.default_rng(seed + 3)
    return rng.integers(lo, hi + 1, size=n_rhs).astype(np.int64)


# Workload shapes.  "c1".."c5" follow the configured map-making problems;
# "tiny"/"small" are the sizes the oracle runs in well under a second.
CONFIGS = {
    "tiny":  dict(nx=4, ny=4, n_det=2, n_t=512, n_int=2, half_bw=8, f_knee=1.0),
    "small": dict(nx=8, ny=8, n_det=4, n_t=4096, n_int=4, half_bw=64, f_knee=1.0),
    # Plain M_BD PCG: 32x32 patch, 8 det x 32768 samples, lambda 512, 8 intervals.
    "c1":    dict(nx=32, ny=32, n_det=8, n_t=32768, n_int=8, half_bw=512, f_knee=1.0),
    # Two-level vs M_BD: 256x256 patch, 128 det x 2^20, f_knee U[0.1, 2], lambda 2048, 64 intervals.
    "c2":    dict(nx=256, ny=256, n_det=128, n_t=1 << 20, n_int=64, half_bw=2048, f_knee=(0.1, 2.0)),
    # Batched Monte Carlo master scan: c1 geometry, 2^20 samples per detector, 4096-sample intervals.
    "c3":    dict(nx=32, ny=32, n_det=8, n_t=1 << 20, n_int=256, half_bw=512, f_knee=1.0),
    # Mixed precision at scale: 512x512 patch, 1024 det x 2^20 (lambda and intervals as c2).
    "c4":    dict(nx=512, ny=512, n_det=1024, n_t=1 << 20, n_int=64, half_bw=2048, f_knee=(0.1, 2.0)),
}


def scan_from_config(name: str, seed: int = 0, **overrides) -> Scan:
    cfg = dict(CONFIGS[name])
    cfg.update(overrides)
    return make_scan(seed=seed, **cfg)
