"""Parity of the template-filtered operator (CUDA, through the C ABI) with the FP64 oracle.

A = P^T F P with F = F_B W^-1 F_G W^-1 F_B (Sect. 2.1 Eq. filtnoise, Sect. 4,
Sect. 5.1): Legendre subscan polynomials, azimuth-bin ground templates, white
block weights, and the differenced timeline d^- (pointing rows (0, cos, sin)).
Tolerances as for the band operator: float64 and double-float (option
"fp64_products" = 2) 1e-11, float32 1e-5 relative on A x; solved maps 1e-6
against an oracle solution converged to 1e-13.
"""
import numpy as np
import pytest

import oracle as O
import synth
from helpers import assert_close

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_1801_08937_gb300")
MM = P.mapmaker

TOL64 = 1e-11
TOL32 = 1e-5
GEOM = dict(nx=8, ny=8, n_det=8, n_t=4096, n_int=4, half_bw=0, f_knee=0.0)


def scan_tmpl(seed=0, flag_frac=0.01, **over):
    cfg = dict(GEOM)
    cfg.update(over)
    scan = synth.make_scan(seed=seed, flag_frac=flag_frac, hwp=False, **cfg)
    sub_off, az, nb = synth.make_templates(scan)
    return scan, sub_off, az, nb


def oracle_tp(scan, sub_off, az, nb, order, ground, qu_only):
    return O.TemplateProblem(scan.pix, scan.psi, scan.block_off, scan.band[scan.block_band, 0], scan.n_pix,
                             sub_off, order, az if ground else None, nb if ground else 0, qu_only)


def ctx_tmpl(scan, sub_off, az, nb, order, ground, qu_only, prec=MM.MM_FP64):
    c = MM.Context(0, None, prec)
    c.setup_scan(scan)
    c.set_templates(order, sub_off if order >= 0 else None, az if ground else None, nb if ground else 0, qu_only)
    return c


def kept(tp, rcond_min=1e-3):
    blocks, hits = O.bd_blocks_T(tp)
    good = O.select_pixels_T(blocks, hits, tp.stokes, rcond_min)
    tp = tp.with_pix(O.flag_samples(tp.pix, good))
    blocks, _ = O.bd_blocks_T(tp)
    return tp, good, O.bd_inverse_T(blocks, good, tp.stokes)


@pytest.mark.parametrize("order,ground,qu_only", [(0, True, 1), (1, True, 1), (3, True, 1), (2, False, 1),
                                                  (-1, True, 1), (1, True, 0), (3, True, 2), (0, False, 2)])
@pytest.mark.parametrize("prec", ["f64", "f32", "df"])
def test_apply_A_matches_oracle(order, ground, qu_only, prec):
    scan, so, az, nb = scan_tmpl(seed=1)
    tp = oracle_tp(scan, so, az, nb, order, ground, qu_only)
    c = ctx_tmpl(scan, so, az, nb, order, ground, qu_only, MM.MM_FP32_MIXED if prec == "f32" else MM.MM_FP64)
    if prec == "df":
        c.set_option("fp64_products", 2)
    x = np.random.default_rng(2).standard_normal((2, scan.n_pix, 3))
    y = c.apply_A(x)
    for r in range(2):
        assert_close(y[r], O.apply_A_T(tp, x[r]), (TOL32 if prec == "f32" else TOL64))
    c.close()


def test_rhs_matches_oracle_and_kills_polynomial_contamination():
    """b = P^T F d; adding per-subscan polynomials of order <= K to d leaves b unchanged (F B = 0)."""
    scan, so, az, nb = scan_tmpl(seed=3)
    tp = oracle_tp(scan, so, az, nb, 1, True, True)
    c = ctx_tmpl(scan, so, az, nb, 1, True, True)
    d = synth.make_tod(scan, synth.make_sky(scan.n_pix, 3), synth.make_noise(scan, 3))
    b = c.rhs(d)
    assert_close(b[0], O.rhs_T(tp, d), TOL64)
    rng = np.random.default_rng(4)
    d2 = d.copy()
    for k in range(len(so) - 1):
        a, e = so[k], so[k + 1]
        u = 2.0 * (np.arange(e - a) + 0.5) / (e - a) - 1.0
        d2[a:e] += 50.0 * rng.standard_normal() + 20.0 * rng.standard_normal() * u
    b2 = c.rhs(d2)
    assert_close(b2[0], b[0], 1e-9)
    c.close()


def test_bd_qu_only_matches_oracle():
    scan, so, az, nb = scan_tmpl(seed=5, ny=12)
    tp = oracle_tp(scan, so, az, nb, 1, True, True)
    c = ctx_tmpl(scan, so, az, nb, 1, True, True)
    dropped = c.build_bd(1e-3)
    tpk, good, mbd = kept(tp)
    assert dropped == int((~good).sum())
    r = np.random.default_rng(5).standard_normal((scan.n_pix, 3))
    assert_close(c.apply_precond(MM.MM_PRECOND_BD, r)[0], O.bd_apply(mbd, r), 1e-12)
    # after flagging, A is the oracle's A on the flagged pointing
    x = np.random.default_rng(6).standard_normal((scan.n_pix, 3))
    assert_close(c.apply_A(x)[0], O.apply_A_T(tpk, x), TOL64)
    c.close()


def _oracle_map(tp, mbd, d):
    b = O.rhs_T(tp, d).reshape(-1)
    return O.pcg(lambda v: O.apply_A_T(tp, v).reshape(-1), lambda v: O.bd_apply(mbd, v).reshape(-1), b,
                 tol=1e-13, max_iter=20000)[0]


@pytest.mark.parametrize("prec", [MM.MM_FP64, MM.MM_FP32_MIXED])
def test_solve_bd_and_two_level_match_oracle(prec):
    """Filtered d^- map with M_BD and with M_2l (Ritz vectors of M_BD A): both match the oracle map; the
    filters leave small eigenvalues that M_2l deflates, so it needs fewer iterations (Sect. 4.3, 7)."""
    scan, so, az, nb = scan_tmpl(seed=7)
    tp = oracle_tp(scan, so, az, nb, 1, True, True)
    sky = synth.make_sky(scan.n_pix, 7)
    sky[:, 0] = 0.0
    d = synth.make_tod(scan, sky, synth.make_noise(scan, 7))
    c = ctx_tmpl(scan, so, az, nb, 1, True, True, prec)
    c.build_bd(1e-3)
    tpk, good, mbd = kept(tp)
    xo = _oracle_map(tpk, mbd, d)
    tod = d.astype(c.tod_dtype)
    xb, ib = c.solve(tod, MM.MM_PRECOND_BD, tol=1e-10, max_iter=5000)
    assert ib[0]["status"] == "MM_OK"
    assert_close(xb[0], xo, 1e-6)
    assert np.abs(xb[0][:, 0]).max() == 0.0          # I is not solved for
    k = c.build_coarse(c.rhs(tod)[0], m_max=120, eps_arn=1e-10, k=24)
    assert k >= 8
    x2, i2 = c.solve(tod, MM.MM_PRECOND_2L, tol=1e-10, max_iter=5000)
    assert i2[0]["status"] == "MM_OK"
    assert_close(x2[0], xo, 1e-6)
    assert i2[0]["iters"] < ib[0]["iters"]
    c.close()


@pytest.mark.parametrize("stokes", [1, 2])
def test_double_float_products_rhs_and_two_level_solve(stokes):
    """MM_FP64 with "fp64_products" = 2: b, the PCG and Arnoldi products and the true residual run in
    double-float arithmetic; b matches the oracle to 1e-11, and the M_BD and M_2l maps match the oracle
    map (d^-) or satisfy the oracle's normal equations (d^+, which has a null vector)."""
    scan, so, az, nb = scan_tmpl(seed=13, flag_frac=0.0 if stokes == 2 else 0.01)
    order = 1 if stokes == 1 else 3
    tp = oracle_tp(scan, so, az, nb, order, True, stokes)
    sky = synth.make_sky(scan.n_pix, 13)
    if stokes == 1:
        sky[:, 0] = 0.0
    else:
        sky[:, 1:] = 0.0
    d = synth.make_tod(scan, sky, synth.make_noise(scan, 13))
    c = ctx_tmpl(scan, so, az, nb, order, True, stokes)
    c.set_option("fp64_products", 2)
    assert c.get_option("fp64_products") == 2
    c.build_bd(1e-3)
    tpk, good, mbd = kept(tp)
    b = c.rhs(d)[0]
    bo = O.rhs_T(tpk, d)
    assert_close(b, bo, TOL64)
    xb, ib = c.solve(d, MM.MM_PRECOND_BD, tol=1e-10, max_iter=5000)
    assert ib[0]["status"] == "MM_OK" and ib[0]["true_rel_res"] <= 1e-9
    k = c.build_coarse(b, m_max=120, eps_arn=1e-12, k=24)
    assert k >= 8
    x2, i2 = c.solve(d, MM.MM_PRECOND_2L, tol=1e-10, max_iter=5000)
    assert i2[0]["status"] == "MM_OK" and i2[0]["true_rel_res"] <= 1e-9
    assert i2[0]["iters"] < ib[0]["iters"]
    if stokes == 1:
        xo = _oracle_map(tpk, mbd, d)
        assert_close(xb[0], xo, 1e-6)
        assert_close(x2[0], xo, 1e-6)
    else:
        for x in (xb[0], x2[0]):
            assert np.linalg.norm(bo - O.apply_A_T(tpk, x)) <= 2e-10 * np.linalg.norm(bo)
    c.close()


def test_white_d_minus_without_filters_converges_in_one_iteration():
    """No templates, white weights, Q/U rows: A = M_BD^-1 exactly, so PCG with M_BD takes one step."""
    scan, so, az, nb = scan_tmpl(seed=8, flag_frac=0.0)
    c = ctx_tmpl(scan, so, az, nb, -1, False, True)
    c.build_bd()
    sky = synth.make_sky(scan.n_pix, 8)
    sky[:, 0] = 0.0
    d = synth.make_tod(scan, sky, synth.make_noise(scan, 8))
    x, info = c.solve(d, MM.MM_PRECOND_BD, tol=1e-10, max_iter=20)
    assert info[0]["iters"] == 1
    c.close()


def test_short_subscans_and_unbinned_samples():
    """Subscans shorter than K + 1 samples are fitted by all their points (order m - 1, output 0 there);
    samples with bin -1 belong to no ground column."""
    scan, so, az, nb = scan_tmpl(seed=9)
    so = np.unique(np.concatenate([so, so[:-1] + 1, so[:-1] + 2]))      # many 1- and 2-sample subscans
    so = so[so <= scan.n_samples]
    az = az.copy()
    az[::7] = -1
    tp = oracle_tp(scan, so, az, nb, 3, True, True)
    c = ctx_tmpl(scan, so, az, nb, 3, True, True)
    x = np.random.default_rng(9).standard_normal((scan.n_pix, 3))
    assert_close(c.apply_A(x)[0], O.apply_A_T(tp, x), TOL64)
    c.close()


def test_intensity_only_d_plus():
    """Summed timeline d^+ (Eq. d+, intensity maps of App. B, Legendre up to order 3): M_BD is the 1x1
    inverse; a constant I map is an exact null vector of A, so the solve is checked through the
    oracle's residual of the returned map and the null component left at 0."""
    scan, so, az, nb = scan_tmpl(seed=11, flag_frac=0.0)
    tp = oracle_tp(scan, so, az, nb, 3, True, 2)
    c = ctx_tmpl(scan, so, az, nb, 3, True, 2)
    dropped = c.build_bd(1e-3)
    tpk, good, mbd = kept(tp)
    assert dropped == int((~good).sum())
    r = np.random.default_rng(11).standard_normal((scan.n_pix, 3))
    assert_close(c.apply_precond(MM.MM_PRECOND_BD, r)[0], O.bd_apply(mbd, r), 1e-12)
    ones = np.zeros((scan.n_pix, 3))
    ones[good, 0] = 1.0
    assert np.abs(c.apply_A(ones)[0]).max() < 1e-9 * np.abs(c.apply_A(r)[0]).max()
    sky = synth.make_sky(scan.n_pix, 11)
    sky[:, 1:] = 0.0
    d = synth.make_tod(scan, sky, synth.make_noise(scan, 11))
    x, info = c.solve(d, MM.MM_PRECOND_BD, tol=1e-10, max_iter=5000)
    assert info[0]["status"] == "MM_OK"
    b = O.rhs_T(tpk, d)
    assert np.linalg.norm(b - O.apply_A_T(tpk, x[0])) <= 2e-10 * np.linalg.norm(b)
    assert np.abs(x[0][:, 1:]).max() == 0.0
    # two-level: the null direction's zero Ritz value is not deflated, E stays SPD
    k = c.build_coarse(c.rhs(d)[0], m_max=120, eps_arn=1e-12, k=24)
    assert k >= 8
    x2, i2 = c.solve(d, MM.MM_PRECOND_2L, tol=1e-10, max_iter=5000)
    assert i2[0]["status"] == "MM_OK" and i2[0]["true_rel_res"] <= 1e-9
    assert np.linalg.norm(b - O.apply_A_T(tpk, x2[0])) <= 2e-10 * np.linalg.norm(b)
    assert i2[0]["iters"] < info[0]["iters"]
    c.close()


def test_device_azimuth_bins_match_host():
    """mm_set_templates with the azimuth bins in device memory gives the same operator as from host memory."""
    torch = pytest.importorskip("torch")
    scan, so, az, nb = scan_tmpl(seed=12)
    x = np.random.default_rng(12).standard_normal((scan.n_pix, 3))
    c1 = ctx_tmpl(scan, so, az, nb, 1, True, 1)
    y1 = c1.apply_A(x)[0]
    c1.close()
    c2 = MM.Context(0, None, MM.MM_FP64)
    c2.setup_scan(scan)
    c2.set_templates(1, so, torch.from_numpy(az).cuda(), nb, 1)
    y2 = c2.apply_A(x)[0]
    c2.close()
    assert_close(y2, y1, 1e-13)


def test_template_argument_errors():
    scan, so, az, nb = scan_tmpl(seed=10)
    c = MM.Context(0, None, MM.MM_FP64)
    with pytest.raises(MM.MapMakerError) as e:
        c.set_templates(1, so, az, nb, True)           # no pointing yet
    assert e.value.status == MM.MM_ERR_STATE
    band_scan = synth.make_scan(seed=10, hwp=False, **dict(GEOM, half_bw=8, f_knee=1.0))
    c.setup_scan(band_scan)
    with pytest.raises(MM.MapMakerError) as e:
        c.set_templates(1, so, az, nb, True)           # a band weight, not white
    assert e.value.status == MM.MM_ERR_ARG
    c.setup_scan(scan)
    bad = so[so != scan.block_off[1]]                   # one subscan across a block edge
    with pytest.raises(MM.MapMakerError) as e:
        c.set_templates(1, bad, az, nb, True)
    assert e.value.status == MM.MM_ERR_ARG
    with pytest.raises(MM.MapMakerError) as e:
        c.set_templates(1, so, az, nb, 3)               # no such Stokes selection
    assert e.value.status == MM.MM_ERR_ARG
    with pytest.raises(MM.MapMakerError) as e:
        c.set_templates(4, so, az, nb, True)            # order above 3
    assert e.value.status == MM.MM_ERR_ARG
    c.set_templates(1, so, az, nb, True)
    c.build_bd()
    d = synth.make_tod(scan, None, synth.make_noise(scan, 10))
    with pytest.raises(MM.MapMakerError) as e:
        c.solve(np.stack([d, d]), MM.MM_PRECOND_BD, tol=1e-8, rhs_len=np.array([4096, 2048]))
    assert e.value.status == MM.MM_ERR_ARG
    c.close()
