"""Full-size c2 checks in the launch configuration the benchmark times.

256x256 patch, 128 detectors x 2^20 samples, lambda 2048, 64 intervals,
mixed precision with the autotuned plan.  The oracle cannot form the whole
product at this size, so it computes sampled rows one by one; the solve is
checked through a property that holds at any size (noise-free data gives
back the sky, Sect. 2, Eq. estimator).
"""
import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_1801_08937_gb300")
MM = P.mapmaker


@pytest.fixture(scope="module")
def c2():
    scan = synth.scan_from_config("c2", seed=0)
    return scan, O.Problem.from_scan(scan)


def _rows_rel(gpu_rows, ref_rows):
    return np.linalg.norm(gpu_rows - ref_rows) / np.linalg.norm(ref_rows)


def test_c2_apply_A_sampled_rows(c2):
    scan, prob = c2
    rng = np.random.default_rng(0)
    pixels = [0, 255, 32768, 65535] + [int(p) for p in rng.integers(0, scan.n_pix, 4)]
    x = rng.standard_normal((scan.n_pix, 3))
    ref = O.apply_A_rows(prob, x, pixels)
    c = MM.Context(0, None, MM.MM_FP32_MIXED)
    c.setup_scan(scan)
    xd = torch.from_numpy(x[None]).cuda()
    y32 = c.apply_A(xd).cpu().numpy()[0]
    assert _rows_rel(y32[pixels], ref) < 1e-5           # float32 operator
    c.set_option("apply_precision", 2)
    ydf = c.apply_A(xd).cpu().numpy()[0]
    assert _rows_rel(ydf[pixels], ref) < 1e-11          # double-float product
    c.close()


def test_c2_rhs_sampled_rows_and_signal_only_solve(c2):
    scan, prob = c2
    sky = synth.make_sky(scan.n_pix, 3)
    d = synth.make_tod(scan, sky, None)
    rng = np.random.default_rng(1)
    pixels = [int(p) for p in rng.integers(0, scan.n_pix, 4)]
    c = MM.Context(0, None, MM.MM_FP32_MIXED)
    c.setup_scan(scan)
    dropped = c.build_bd(1e-3)
    assert dropped == 0
    tod = torch.from_numpy(d.astype(np.float32)).cuda()
    b = c.rhs(tod).cpu().numpy()[0]
    ref = O.rhs_rows(prob, d.astype(np.float32).astype(np.float64), pixels)
    assert _rows_rel(b[pixels], ref) < 1e-11
    # coarse space from a first M_BD run, then the two-level solve
    c.set_option("harvest", 120)
    xb, ib = c.solve(tod, MM.MM_PRECOND_BD, tol=1e-8, max_iter=1000)
    c.set_option("harvest", 0)
    c.build_coarse_from_solve(k=32)
    x2, i2 = c.solve(tod, MM.MM_PRECOND_2L, tol=1e-8, max_iter=1000)
    for x, info in ((xb, ib), (x2, i2)):
        assert info[0]["status"] == "MM_OK" and info[0]["true_rel_res"] <= 1e-8
        # noise-free data: the GLS map is the sky (float32 timeline: sky rounded to float32 samples)
        err = np.linalg.norm(x.cpu().numpy()[0] - sky) / np.linalg.norm(sky)
        assert err < 1e-6
    assert i2[0]["iters"] < ib[0]["iters"]
    c.close()
