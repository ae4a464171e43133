"""Seeded synthetic inputs for ground-based polarised map-making.

This package draws every random number and builds every input array that the
CUDA path and the oracle consume: scan pointing (pixel index and HWP angle per
sample), the per-detector inverse-noise Toeplitz bands, a Gaussian I/Q/U sky
and 1/f noise timelines.  It holds none of the map-making arithmetic (no
pointing product, no filtering of a timeline by the band, no preconditioner);
both sides receive identical arrays from here.

Workload shapes follow the paper's ground-based simulations (Sect. 5: constant
elevation scans at 0.4 deg/s over a small patch, polarisation-sensitive
detectors behind a rotating half-wave plate) at the sizes named in ``CONFIGS``.
``synth.device`` builds the same kind of scan and timeline on a CUDA device
for request streams too large for the host.
"""
from .scan import (Scan, CONFIGS, make_scan, make_sky, make_noise, make_tod,
                   toeplitz_band, scan_from_config, mc_lengths, make_templates, AZ_BIN_PX)

__all__ = ["Scan", "CONFIGS", "make_scan", "make_sky", "make_noise", "make_tod",
           "toeplitz_band", "scan_from_config", "mc_lengths", "make_templates", "AZ_BIN_PX"]
