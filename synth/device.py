"""Seeded scans and timelines built on a CUDA device with torch, for request
streams too large to synthesise on the host (up to 1024 detectors x 2^20
samples per scan).

The scan geometry, the half-wave-plate model and the 1/f noise shaping are
those of ``make_scan``/``make_noise``/``make_tod`` (Sect. 5 of the paper): the
pixel indices equal make_scan's for the same seed and shape, while the HWP
angles, the sky and the noise come from torch's random streams.  Detectors
share a few noise bands.  Work is done in chunks of detectors so that the
temporaries stay at a few GB whatever the scan size.  Like the rest of this
package it only synthesises inputs: it never applies the pointing transpose,
a noise band to a timeline, or a preconditioner.
"""
from __future__ import annotations

import math

import numpy as np

from .scan import FS_HZ, SCAN_SPEED_PX, toeplitz_band

DET_CHUNK = 64


class DeviceScan:
    """Pointing (device tensors) and block structure (host arrays) of one scan."""

    def __init__(self, nx, n_det, n_t, n_int, half_bw, pix, psi, block_off, block_band, band, f_knee, seed):
        self.nx = self.ny = nx
        self.n_det, self.n_t, self.n_int, self.half_bw = n_det, n_t, n_int, half_bw
        self.pix, self.psi = pix, psi
        self.block_off, self.block_band, self.band = block_off, block_band, band
        self.f_knee = f_knee
        self.seed = seed

    @property
    def n_pix(self) -> int:
        return self.nx * self.ny

    @property
    def n_samples(self) -> int:
        return self.n_det * self.n_t


def make_scan_device(torch, dev, nx: int, n_det: int, n_t: int, n_int: int, half_bw: int, seed: int,
                     f_knees=(0.1, 0.5, 1.0, 2.0)) -> DeviceScan:
    """Back-and-forth raster of an nx x nx patch by n_det detectors (as ``make_scan``), HWP angle
    psi ~ U[0, pi) per sample.  Detector d takes f_knee = f_knees[d % len(f_knees)], so the scan
    has len(f_knees) noise bands."""
    if n_t % n_int != 0:
        raise ValueError("n_t must be a multiple of n_int")
    g = torch.Generator(device=dev).manual_seed(seed)
    rng = np.random.default_rng(seed)
    x0 = torch.from_numpy(rng.uniform(0.0, 2.0 * nx, size=n_det)).to(dev)
    y0 = float(rng.uniform(0.0, nx))
    t = torch.arange(n_t, device=dev, dtype=torch.float64)
    st = SCAN_SPEED_PX * t
    ty = t * (nx / n_t)
    pix = torch.empty(n_det * n_t, device=dev, dtype=torch.int32)
    for d0 in range(0, n_det, DET_CHUNK):
        d1 = min(n_det, d0 + DET_CHUNK)
        pos = torch.remainder(x0[d0:d1, None] + st[None, :], 2.0 * nx)
        pos = torch.where(pos >= nx, 2.0 * nx - pos, pos)
        ix = pos.to(torch.int32).clamp_(max=nx - 1)
        oy = torch.arange(d0, d1, device=dev, dtype=torch.float64)[:, None] * (nx / 4.0) / n_det
        iy = torch.remainder(y0 + oy + ty[None, :], float(nx)).to(torch.int32).clamp_(max=nx - 1)
        pix[d0 * n_t:d1 * n_t] = (iy * nx + ix).reshape(-1)
        del pos, ix, iy
    psi = torch.rand(n_det * n_t, generator=g, device=dev, dtype=torch.float32) * math.pi
    psi.clamp_(max=float(np.nextafter(np.float32(np.pi), np.float32(0))))
    nb = len(f_knees)
    fk = np.array([f_knees[d % nb] for d in range(n_det)], dtype=np.float64)
    blen = n_t // n_int
    block_off = np.arange(n_det * n_int + 1, dtype=np.int64) * blen
    block_band = np.repeat(np.arange(n_det, dtype=np.int32) % nb, n_int).astype(np.int32)
    band = np.stack([toeplitz_band(half_bw, float(f), 1.0, 1.0, FS_HZ) for f in f_knees[:min(nb, n_det)]])
    return DeviceScan(nx, n_det, n_t, n_int, half_bw, pix, psi, block_off, block_band, band, fk, seed)


def make_tod_device(torch, scan: DeviceScan, seed: int, sigma_qu: float = 0.1) -> "torch.Tensor":
    """Timeline d = I_p + Q_p cos 2psi + U_p sin 2psi + n (Sect. 2's data model) for a Gaussian sky
    (sigma_I = 1, sigma_QU = sigma_qu) and 1/f noise stationary per block, as float32 on the scan's
    device."""
    dev = scan.pix.device
    g = torch.Generator(device=dev).manual_seed(seed)
    sky = torch.randn((scan.n_pix, 3), generator=g, device=dev, dtype=torch.float64)
    sky[:, 1:] *= sigma_qu
    blen = scan.n_t // scan.n_int
    f = torch.fft.rfftfreq(blen, d=1.0 / FS_HZ, device=dev, dtype=torch.float64)
    f[0] = f[1]
    out = torch.empty(scan.n_samples, device=dev, dtype=torch.float32)
    for d0 in range(0, scan.n_det, DET_CHUNK):
        d1 = min(scan.n_det, d0 + DET_CHUNK)
        a, b = d0 * scan.n_t, d1 * scan.n_t
        p = scan.pix[a:b].long()
        ang = 2.0 * scan.psi[a:b].double()
        sig = sky[p, 0] + sky[p, 1] * torch.cos(ang) + sky[p, 2] * torch.sin(ang)
        del p, ang
        w = torch.randn(((d1 - d0) * scan.n_int, blen), generator=g, device=dev, dtype=torch.float64)
        fk = torch.from_numpy(np.repeat(scan.f_knee[d0:d1], scan.n_int)).to(dev)[:, None]
        shaped = torch.fft.irfft(torch.fft.rfft(w, dim=1) * torch.sqrt(1.0 + fk / f[None, :]), n=blen, dim=1)
        out[a:b] = (sig + shaped.reshape(-1)).float()
        del sig, w, shaped
    return out
