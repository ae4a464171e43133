"""The device scan generator (used for request streams too large for the host) draws the same
raster as the host generator: identical pixel indices for the same seed and shape, HWP angles in
[0, pi), the block layout and bands of make_scan's model.  Run on torch's CPU device."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
from synth.device import make_scan_device, make_tod_device  # noqa: E402


@pytest.mark.parametrize("nx,n_det,n_t,n_int", [(16, 3, 4096, 2), (64, 70, 2048, 1)])
def test_device_raster_matches_the_host_scan(nx, n_det, n_t, n_int):
    host = synth.make_scan(nx=nx, ny=nx, n_det=n_det, n_t=n_t, n_int=n_int, half_bw=32, seed=11)
    dev = make_scan_device(torch, "cpu", nx, n_det, n_t, n_int, 32, seed=11, f_knees=(0.5, 1.0))
    assert np.array_equal(dev.pix.numpy(), host.pix)
    psi = dev.psi.numpy()
    assert psi.dtype == np.float32 and psi.min() >= 0.0 and psi.max() < np.pi
    assert np.array_equal(dev.block_off, host.block_off)
    assert np.array_equal(dev.block_band, np.repeat(np.arange(n_det) % 2, n_int))
    assert np.allclose(dev.band[1], synth.toeplitz_band(32, 1.0))


def test_device_timeline_carries_the_sky_signal():
    dev = make_scan_device(torch, "cpu", 16, 4, 8192, 2, 32, seed=12)
    d = make_tod_device(torch, dev, seed=3).double().numpy()
    assert d.shape == (4 * 8192,) and np.isfinite(d).all()
    # the timeline is signal + noise with unit white level: its variance is about 1 (sky) + noise
    assert 1.0 < d.var() < 50.0
