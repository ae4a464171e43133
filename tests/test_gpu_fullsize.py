"""Full-size checks in the launch configuration the benchmark times.

c2: 256x256 patch, 128 detectors x 2^20 samples, lambda 2048, 64 intervals,
mixed precision with the autotuned plan.  c4 subset: the 512x512 geometry of
c4 with 16 of its 1024 detectors (1/64 of the data).  The oracle cannot form
the whole product at these sizes, so it computes sampled rows one by one --
patch corners, the least-hit pixels, pixels next to flagged samples and
random pixels -- and every row is compared element by element and per Stokes
parameter.  Solves are checked through a property that holds at any size
(noise-free data gives back the sky, Sect. 2, Eq. estimator) and, for noisy
data, against the float64-accurate GPU path.
"""
import numpy as np
import pytest

import oracle as O
import synth
from helpers import assert_close, oracle_problem

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_1801_08937_gb300")
MM = P.mapmaker


def _sub_problem(prob, blocks):
    """The oracle problem restricted to whole blocks: W is block diagonal, so a row of A x (or b)
    of a pixel depends only on the blocks holding its samples; the restricted problem keeps those
    samples in the same order with the same block boundaries."""
    offs = [(int(prob.block_off[b]), int(prob.block_off[b + 1])) for b in blocks]
    idx = np.concatenate([np.arange(a, e) for a, e in offs])
    new_off = np.concatenate([[0], np.cumsum([e - a for a, e in offs])])
    return O.Problem(prob.pix[idx], prob.psi[idx], new_off, prob.band, prob.block_band[blocks], prob.n_pix), idx


def oracle_rows(prob, pixels, x=None, d=None):
    """Rows of A x (or of b = P^T W d) for the listed pixels, each from the oracle's own row
    function on the blocks that hold that pixel's samples."""
    pix = np.asarray(pixels)
    ts = np.nonzero(np.isin(prob.pix, pix))[0]
    bs = np.searchsorted(prob.block_off, ts, side="right") - 1
    pt = prob.pix[ts]
    out = np.zeros((len(pix), 3))
    for i, p in enumerate(pix):
        blocks = np.unique(bs[pt == p])
        if blocks.size == 0:
            continue
        sub, idx = _sub_problem(prob, blocks)
        out[i] = (O.apply_A_rows(sub, x, [p]) if d is None else O.rhs_rows(sub, d[idx], [p]))[0]
    return out


def sample_pixels(scan, pix, n_random, seed, flagged=False):
    """Corners, the least-hit pixels, pixels seen right before or after a flagged sample, random."""
    rng = np.random.default_rng(seed)
    nx, ny = scan.nx, scan.ny
    hits = np.bincount(pix[pix >= 0], minlength=scan.n_pix)
    seen = np.nonzero(hits)[0]
    least = seen[np.argsort(hits[seen], kind="stable")[:12]]
    chosen = [0, nx - 1, (ny - 1) * nx, ny * nx - 1, (ny // 2) * nx + nx // 2] + [int(p) for p in least]
    if flagged:
        f = np.nonzero(pix < 0)[0]
        f = f[(f > 0) & (f < pix.size - 1)]
        nb = np.concatenate([pix[f - 1], pix[f + 1]])
        nb = nb[nb >= 0]
        chosen += [int(p) for p in rng.choice(np.unique(nb), size=min(24, np.unique(nb).size), replace=False)]
    chosen += [int(p) for p in rng.integers(0, scan.n_pix, n_random)]
    return sorted(set(chosen))


@pytest.fixture(scope="module")
def c2():
    scan = synth.scan_from_config("c2", seed=0)
    return scan, O.Problem.from_scan(scan)


def test_c2_apply_A_sampled_rows(c2):
    """64+ sampled rows of A x at c2: float32 operator within 1e-5, double-float within 1e-11."""
    scan, prob = c2
    pixels = sample_pixels(scan, scan.pix, 48, 0)
    assert len(pixels) >= 64
    x = np.random.default_rng(0).standard_normal((scan.n_pix, 3))
    ref = oracle_rows(prob, pixels, x=x)
    c = MM.Context(0, None, MM.MM_FP32_MIXED)
    c.setup_scan(scan)
    xd = torch.from_numpy(x[None]).cuda()
    y32 = c.apply_A(xd).cpu().numpy()[0]
    assert_close(y32[pixels], ref, 1e-5, "c2 A x rows, float32")
    c.set_option("apply_precision", 2)
    ydf = c.apply_A(xd).cpu().numpy()[0]
    assert_close(ydf[pixels], ref, 1e-11, "c2 A x rows, double-float")
    c.close()


def test_c2_flagged_apply_A_and_rhs_rows(c2):
    """The c2 scan with 0.1 % of its samples flagged: rows next to flagged samples and others."""
    scan, _ = c2
    rng = np.random.default_rng(7)
    pix = scan.pix.copy()
    pix[rng.random(pix.size) < 1e-3] = -1
    prob = O.Problem(pix, scan.psi, scan.block_off, scan.band, scan.block_band, scan.n_pix)
    pixels = sample_pixels(scan, pix, 28, 7, flagged=True)
    assert len(pixels) >= 64
    x = rng.standard_normal((scan.n_pix, 3))
    d = synth.make_tod(scan, synth.make_sky(scan.n_pix, 7), None).astype(np.float32)
    c = MM.Context(0, None, MM.MM_FP32_MIXED)
    c.setup_pointing(pix, scan.psi, scan.block_off, scan.block_band, scan.band, scan.n_pix, scan.n_det)
    y = c.apply_A(torch.from_numpy(x[None]).cuda()).cpu().numpy()[0]
    assert_close(y[pixels], oracle_rows(prob, pixels, x=x), 1e-5, "c2 flagged A x rows, float32")
    b = c.rhs(torch.from_numpy(d).cuda()).cpu().numpy()[0]
    assert_close(b[pixels], oracle_rows(prob, pixels, d=d.astype(np.float64)), 1e-11, "c2 flagged b rows")
    c.close()


def test_c2_rhs_sampled_rows_and_signal_only_solve(c2):
    scan, prob = c2
    sky = synth.make_sky(scan.n_pix, 3)
    d = synth.make_tod(scan, sky, None)
    pixels = sample_pixels(scan, scan.pix, 48, 1)
    c = MM.Context(0, None, MM.MM_FP32_MIXED)
    c.setup_scan(scan)
    dropped = c.build_bd(1e-3)
    assert dropped == 0
    tod = torch.from_numpy(d.astype(np.float32)).cuda()
    b = c.rhs(tod).cpu().numpy()[0]
    ref = oracle_rows(prob, pixels, d=d.astype(np.float32).astype(np.float64))
    assert_close(b[pixels], ref, 1e-11, "c2 b rows")
    # coarse space from a first M_BD run, then the two-level solve
    c.set_option("harvest", 120)
    xb, ib = c.solve(tod, MM.MM_PRECOND_BD, tol=1e-8, max_iter=1000)
    c.set_option("harvest", 0)
    c.build_coarse_from_solve(k=32)
    x2, i2 = c.solve(tod, MM.MM_PRECOND_2L, tol=1e-8, max_iter=1000)
    for x, info, name in ((xb, ib, "M_BD"), (x2, i2, "M_2l")):
        assert info[0]["status"] == "MM_OK" and info[0]["true_rel_res"] <= 1e-8
        # noise-free data: the GLS map is the sky (float32 timeline: sky rounded to float32 samples).
        # At a 1e-8 residual the map error is the solver's (Sect. 3, Eq. errnorm: up to kappa times
        # the residual): every Stokes column within 1e-6, the worst single pixel within 1e-5 ...
        assert_close(x.cpu().numpy()[0], sky, 1e-6, f"c2 noise-free {name} map vs sky, tol 1e-8", elem_tol=1e-5)
    assert i2[0]["iters"] < ib[0]["iters"]
    # ... and solved further, every pixel within 1e-6
    x3, i3 = c.solve(tod, MM.MM_PRECOND_2L, tol=1e-10, max_iter=1000)
    assert i3[0]["status"] == "MM_OK"
    assert_close(x3.cpu().numpy()[0], sky, 1e-6, "c2 noise-free M_2l map vs sky, tol 1e-10")
    c.close()


def test_c2_noisy_map_matches_float64_path(c2):
    """Noisy c2 data: the mixed-precision two-level map at a 1e-8 residual against the MM_FP64 path
    with double-float products converged to 1e-11 (per Stokes parameter, element by element)."""
    scan, _ = c2
    d = synth.make_tod(scan, synth.make_sky(scan.n_pix, 5), synth.make_noise(scan, 5))
    ref_ctx = MM.Context(0, None, MM.MM_FP64)
    ref_ctx.set_option("fp64_products", 2)
    ref_ctx.setup_scan(scan)
    ref_ctx.build_bd(1e-3)
    td = torch.from_numpy(d).cuda()
    xr, ir = ref_ctx.solve(td, MM.MM_PRECOND_BD, tol=1e-11, max_iter=3000)
    assert ir[0]["status"] == "MM_OK"
    ref = xr.cpu().numpy()[0]
    ref_ctx.close()
    c = MM.Context(0, None, MM.MM_FP32_MIXED)
    c.setup_scan(scan)
    c.build_bd(1e-3)
    tf = torch.from_numpy(d.astype(np.float32)).cuda()
    c.set_option("harvest", 120)
    xb, ib = c.solve(tf, MM.MM_PRECOND_BD, tol=1e-8, max_iter=1000)
    c.set_option("harvest", 0)
    c.build_coarse_from_solve(k=32)
    x2, i2 = c.solve(tf, MM.MM_PRECOND_2L, tol=1e-8, max_iter=1000)
    # the mixed path solves for the float32-rounded timeline; its GLS map differs from the float64
    # timeline's by the rounding of d (about 6e-8 relative), far below the tolerance
    for x, info, name in ((xb, ib, "M_BD"), (x2, i2, "M_2l")):
        assert info[0]["status"] == "MM_OK" and info[0]["true_rel_res"] <= 1e-8
        assert_close(x.cpu().numpy()[0], ref, 1e-6, f"c2 noisy {name} map vs float64 path, tol 1e-8",
                     elem_tol=1e-5)
    x3, i3 = c.solve(tf, MM.MM_PRECOND_2L, tol=1e-10, max_iter=1000)
    assert i3[0]["status"] == "MM_OK"
    assert_close(x3.cpu().numpy()[0], ref, 1e-6, "c2 noisy M_2l map vs float64 path, tol 1e-10")
    c.close()


# ---------------- c4 geometry, 1/64 of the detectors ----------------

@pytest.fixture(scope="module")
def c4sub():
    scan = synth.scan_from_config("c4", seed=0, n_det=16)
    return scan, O.Problem.from_scan(scan)


def test_c4_subset_rows_and_maps(c4sub):
    """c4 geometry (512x512, lambda 2048, 64 intervals) with 16 detectors: sampled rows of A x and b
    against the oracle; the noise-free two-level map against the sky; the noisy mixed-precision map
    against the float64-accurate GPU path."""
    scan, prob = c4sub
    prob_f, mbd, good = oracle_problem(scan)
    pixels = sample_pixels(scan, prob_f.pix, 48, 4)
    rng = np.random.default_rng(4)
    x = rng.standard_normal((scan.n_pix, 3))
    x[~good] = 0
    sky = synth.make_sky(scan.n_pix, 4)
    sky[~good] = 0
    d = synth.make_tod(scan, sky, None).astype(np.float32)
    c = MM.Context(0, None, MM.MM_FP32_MIXED)
    c.setup_scan(scan)
    assert c.build_bd(1e-3) == int((~good).sum())
    y = c.apply_A(torch.from_numpy(x[None]).cuda()).cpu().numpy()[0]
    assert_close(y[pixels], oracle_rows(prob_f, pixels, x=x), 1e-5, "c4/64 A x rows, float32")
    td = torch.from_numpy(d).cuda()
    b = c.rhs(td).cpu().numpy()[0]
    assert_close(b[pixels], oracle_rows(prob_f, pixels, d=d.astype(np.float64)), 1e-11, "c4/64 b rows")
    c.set_option("harvest", 64)
    xb, ib = c.solve(td, MM.MM_PRECOND_BD, tol=1e-8, max_iter=2000)
    c.set_option("harvest", 0)
    k = c.build_coarse_from_solve(k=64)
    assert k >= 32
    x2, i2 = c.solve(td, MM.MM_PRECOND_2L, tol=1e-8, max_iter=2000)
    for xm, info, name in ((xb, ib, "M_BD"), (x2, i2, "M_2l")):
        assert info[0]["status"] == "MM_OK"
        assert_close(xm.cpu().numpy()[0], sky, 1e-6, f"c4/64 noise-free {name} map vs sky, tol 1e-8", elem_tol=1e-5)
    x3, i3 = c.solve(td, MM.MM_PRECOND_2L, tol=1e-10, max_iter=2000)
    assert i3[0]["status"] == "MM_OK"
    assert_close(x3.cpu().numpy()[0], sky, 1e-6, "c4/64 noise-free M_2l map vs sky, tol 1e-10")
    # noisy data: mixed two-level map against the double-float MM_FP64 path
    dn = synth.make_tod(scan, synth.make_sky(scan.n_pix, 6), synth.make_noise(scan, 6))
    xm, im = c.solve(torch.from_numpy(dn.astype(np.float32)).cuda(), MM.MM_PRECOND_2L, tol=1e-8, max_iter=2000)
    assert im[0]["status"] == "MM_OK"
    c.close()
    r = MM.Context(0, None, MM.MM_FP64)
    r.set_option("fp64_products", 2)
    r.setup_scan(scan)
    r.build_bd(1e-3)
    xr, ir = r.solve(torch.from_numpy(dn).cuda(), MM.MM_PRECOND_BD, tol=1e-11, max_iter=4000)
    assert ir[0]["status"] == "MM_OK"
    r.close()
    assert_close(xm.cpu().numpy()[0], xr.cpu().numpy()[0], 1e-6, "c4/64 noisy M_2l map vs float64 path, tol 1e-8",
                 elem_tol=1e-5)
