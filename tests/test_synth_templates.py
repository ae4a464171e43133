"""The seeded template geometry (stand-in for the paper's constant-elevation scans, Sect. 4-5):
subscans are the azimuth sweeps between turnarounds, cut at block edges; azimuth bins of 0.08 deg
follow the raster's azimuth.  Checks the generator against the scan it describes."""
import numpy as np

import synth


def _scan(**over):
    cfg = dict(nx=16, ny=8, n_det=3, n_t=4096, n_int=4, half_bw=0, f_knee=0.0, seed=5, hwp=False)
    cfg.update(over)
    return synth.make_scan(**cfg)


def test_subscans_cover_the_timeline_and_respect_blocks():
    scan = _scan()
    so, az, nb = synth.make_templates(scan)
    assert so[0] == 0 and so[-1] == scan.n_samples and np.all(np.diff(so) > 0)
    assert set(scan.block_off.tolist()) <= set(so.tolist())          # block edges are subscan edges
    assert az.shape == (scan.n_samples,) and az.min() >= 0 and az.max() < nb
    # one sweep of a 16-pixel raster at 0.14 px/sample is ~114 samples; block cuts only shorten them
    lens = np.diff(so)
    assert lens.max() <= int(np.ceil(scan.nx / scan.meta["speed"])) + 1


def test_each_subscan_is_one_monotone_sweep_and_bins_follow_the_azimuth():
    scan = _scan()
    so, az, nb = synth.make_templates(scan)
    ix = np.where(scan.pix >= 0, scan.pix % scan.nx, -1)
    for s in range(len(so) - 1):
        a, b = so[s], so[s + 1]
        d = np.diff(az[a:b])
        assert np.all(d >= 0) or np.all(d <= 0)                      # the bin never turns back inside a sweep
        x = ix[a:b]
        dx = np.diff(x[x >= 0])
        assert np.all(dx >= 0) or np.all(dx <= 0)
    # the bin of a sample is the bin of its pixel's azimuth column (bins are wider than a pixel)
    ok = scan.pix >= 0
    col_bin = np.floor((ix[ok] + 0.5) / synth.AZ_BIN_PX).astype(int)
    assert np.mean(np.abs(az[ok] - col_bin) <= 1) == 1.0
    assert nb == int(np.ceil(scan.nx / synth.AZ_BIN_PX))


def test_generator_is_seeded():
    s1, s2 = _scan(), _scan()
    a1 = synth.make_templates(s1)
    a2 = synth.make_templates(s2)
    assert np.array_equal(a1[0], a2[0]) and np.array_equal(a1[1], a2[1])


def test_threaded_generation_gives_the_serial_values(monkeypatch):
    """Large inputs are generated on several host threads; the values equal a one-thread run."""
    import synth.scan as SC
    cfg = dict(nx=32, ny=32, n_det=4, n_t=1 << 20, n_int=4, half_bw=16, f_knee=1.0, seed=9, flag_frac=0.01)

    def run():
        scan = synth.make_scan(**cfg)
        n = synth.make_noise(scan, 9)
        so, az, _ = synth.make_templates(scan)
        return scan.pix, n, synth.make_tod(scan, synth.make_sky(scan.n_pix, 9), n), so, az

    threaded = run()
    monkeypatch.setattr(SC.os, "cpu_count", lambda: 1)
    serial = run()
    for a, b in zip(threaded, serial):
        assert np.array_equal(a, b)
