"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: float64 operator 1e-11 relative (FFT rounding of a few ulp per
pass); float32 operator 1e-5 relative on A x; solved maps 1e-6 relative to
an oracle solution converged far below the PCG tolerance.
"""
import copy

import numpy as np
import pytest

import oracle as O
import synth
from helpers import assert_close, oracle_problem, scan_and_tod, truncated_problem

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_1801_08937_gb300")
MM = P.mapmaker

TOL64 = 1e-11
TOL32 = 1e-5


def ctx_for(scan, prec=MM.MM_FP64, filt=0, fft_log2=0, fft_len=0, half=1):
    c = MM.Context(0, None, prec)
    c.set_option("filter", filt)
    c.set_option("half_transform", half)
    if fft_log2:
        c.set_option("fft_log2", fft_log2)
    if fft_len:
        c.set_option("fft_len", fft_len)
    c.setup_scan(scan)
    return c


def ragged(scan, seed=0, min_len=40):
    """Re-cut every detector timeline into blocks of uneven length."""
    rng = np.random.default_rng(seed)
    offs = [0]
    bands = []
    for d in range(scan.n_det):
        t0, t1 = d * scan.n_t, (d + 1) * scan.n_t
        cuts = np.sort(rng.choice(np.arange(t0 + min_len, t1 - min_len), size=3, replace=False))
        pts = [p for p in cuts if p - offs[-1] >= min_len] + [t1]
        for p in pts:
            offs.append(int(p))
            bands.append(d % scan.n_bands)
    s = copy.copy(scan)
    s.block_off = np.array(offs, dtype=np.int64)
    s.block_band = np.array(bands, dtype=np.int32)
    return s


SMALL = dict(nx=8, ny=8, n_det=4, n_t=4096, n_int=4, half_bw=64, f_knee=1.0)


@pytest.mark.parametrize("filt,fft_len", [(1, 0), (2, 0), (2, 256), (2, 1024), (2, 576), (2, 768), (2, 1152),
                                          (2, 2304), (2, 4608)])
@pytest.mark.parametrize("prec", [MM.MM_FP64, MM.MM_FP32_MIXED])
def test_apply_A_matches_oracle(filt, fft_len, prec):
    """Direct band, overlap-save segments (L < n_b + lambda) and whole blocks, radix 2..16, 3 and 9."""
    scan = ragged(synth.make_scan(seed=1, flag_frac=0.01, **SMALL), seed=1)
    prob = O.Problem.from_scan(scan)
    c = ctx_for(scan, prec, filt, fft_len=fft_len)
    x = np.random.default_rng(2).standard_normal((2, scan.n_pix, 3))
    y = c.apply_A(x)
    for r in range(2):
        ref = O.apply_A(prob, x[r])
        assert_close(y[r], ref, (TOL64 if prec == MM.MM_FP64 else TOL32))


CT_LENGTHS = [2048, 4096, 4608, 8192, 9216, 12288, 16384, 18432]


@pytest.mark.parametrize("L", CT_LENGTHS)
@pytest.mark.parametrize("prec", [MM.MM_FP64, MM.MM_FP32_MIXED])
def test_apply_A_compile_time_lengths(L, prec):
    """Every compile-time transform of the two-segment kernel, as whole blocks (short blocks) and
    as segments (long blocks)."""
    if prec == MM.MM_FP64 and L > 12288:
        pytest.skip("float64 transform of this length exceeds shared memory")
    for cfg in (SMALL, dict(nx=8, ny=8, n_det=2, n_t=40960, n_int=2, half_bw=200, f_knee=1.0)):
        scan = synth.make_scan(seed=19, flag_frac=0.01, **cfg)
        prob = O.Problem.from_scan(scan)
        c = ctx_for(scan, prec, 2, fft_len=L, half=0)
        x = np.random.default_rng(19).standard_normal((scan.n_pix, 3))
        assert_close(c.apply_A(x)[0], O.apply_A(prob, x), (TOL64 if prec == MM.MM_FP64 else TOL32))


HALF_LENGTHS = [1152, 2048, 4608, 6144, 9216, 16384, 18432]


@pytest.mark.parametrize("L", HALF_LENGTHS)
@pytest.mark.parametrize("prec", ["f64", "f32", "df"])
def test_apply_A_half_length_transform(L, prec):
    """Whole blocks as L/2-point complex transforms with the paired real-spectrum step, against the
    oracle and the two-segment kernel: ragged blocks with unaligned starts and lengths, flagged
    samples, compile-time (L/2 = 2304, 4608, 8192, 9216) and run-time plans."""
    n_t = L - 64 - 7                     # every block fits one transform with its band
    scan = ragged(synth.make_scan(seed=31, flag_frac=0.01, nx=8, ny=8, n_det=3, n_t=n_t, n_int=1,
                                  half_bw=64, f_knee=1.0), seed=31)
    prob = O.Problem.from_scan(scan)
    x = np.random.default_rng(31).standard_normal((2, scan.n_pix, 3))
    tol = TOL32 if prec == "f32" else TOL64
    halves = (1,) if (prec != "f32" and L > 12288) else (1, 0)   # two segments of 16-byte points do not fit
    for half in halves:
        c = ctx_for(scan, MM.MM_FP64 if prec == "f64" else MM.MM_FP32_MIXED, 2, fft_len=L, half=half)
        if prec == "df":
            c.set_option("apply_precision", 2)
        y = c.apply_A(x)
        if prec != "df":
            assert c.get_option("plan_whole") == (2 if half else 1)
        for r in range(2):
            assert_close(y[r], O.apply_A(prob, x[r]), tol)
        c.close()


@pytest.mark.parametrize("L", [4608, 18432])
@pytest.mark.parametrize("products", [1, 2])
def test_rhs_half_length_transform(L, products):
    """b = P^T W d through the half-length transform (float64 and double-float), ragged blocks."""
    n_t = L - 64 - 7
    scan = ragged(synth.make_scan(seed=33, flag_frac=0.01, nx=8, ny=8, n_det=3, n_t=n_t, n_int=1,
                                  half_bw=64, f_knee=1.0), seed=33)
    d = synth.make_tod(scan, synth.make_sky(scan.n_pix, 33), synth.make_noise(scan, 33))
    prob = O.Problem.from_scan(scan)
    c = ctx_for(scan, MM.MM_FP32_MIXED, 2, fft_len=L)
    c.set_option("fp64_products", products)
    tod = d.astype(c.tod_dtype)
    assert_close(c.rhs(tod)[0], O.rhs(prob, tod.astype(np.float64)), TOL64)
    c.close()


@pytest.mark.parametrize("tile", [1024, 2048])
@pytest.mark.parametrize("lam", [0, 5, 16])
@pytest.mark.parametrize("prec", [MM.MM_FP32_MIXED, MM.MM_FP64])
def test_apply_A_direct_tiles(tile, lam, prec):
    """Direct band with the lean four-samples-per-thread float32 kernel (and float64), ragged blocks, flags."""
    scan = ragged(synth.make_scan(seed=27, flag_frac=0.02, **dict(SMALL, half_bw=lam)), seed=27)
    prob = O.Problem.from_scan(scan)
    c = ctx_for(scan, prec, 1)
    c.set_option("direct_tile", tile)
    x = np.random.default_rng(27).standard_normal((2, scan.n_pix, 3))
    y = c.apply_A(x)
    tol = TOL64 if prec == MM.MM_FP64 else TOL32
    for r in range(2):
        assert_close(y[r], O.apply_A(prob, x[r]), tol)
    d = synth.make_tod(scan, synth.make_sky(scan.n_pix, 27), synth.make_noise(scan, 27))
    c.build_bd()
    xs, info = c.solve(d.astype(c.tod_dtype), MM.MM_PRECOND_BD, tol=1e-10)
    assert info[0]["status"] == "MM_OK"


@pytest.mark.parametrize("lam,blen", [(0, 512), (3, 512), (150, 100), (64, 65), (200, 4096)])
def test_apply_A_band_edges(lam, blen):
    """Bands wider than blocks, zero bands, one-tap bands: truncation at block edges."""
    scan = synth.make_scan(nx=4, ny=4, n_det=2, n_t=blen * 4, n_int=4, half_bw=lam, f_knee=1.0, seed=3)
    prob = O.Problem.from_scan(scan)
    x = np.random.default_rng(3).standard_normal((scan.n_pix, 3))
    ref = O.apply_A(prob, x)
    for filt in (1, 2):
        if filt == 2 and 2 * lam + 32 > (1 << 13):
            continue
        c = ctx_for(scan, MM.MM_FP64, filt)
        assert_close(c.apply_A(x)[0], ref, TOL64)


@pytest.mark.parametrize("fft_len", [0, 4608, 8192, 12288])
def test_apply_A_double_float_matches_oracle(fft_len):
    """Double-float products reach float64-level agreement with the oracle."""
    scan = ragged(synth.make_scan(seed=20, flag_frac=0.01, **SMALL), seed=20)
    prob = O.Problem.from_scan(scan)
    c = ctx_for(scan, MM.MM_FP32_MIXED, 2 if fft_len else 0, fft_len=fft_len)
    c.set_option("apply_precision", 2)
    x = np.random.default_rng(20).standard_normal((2, scan.n_pix, 3))
    y = c.apply_A(x)
    for r in range(2):
        assert_close(y[r], O.apply_A(prob, x[r]), TOL64)


def test_apply_A_c1_full_size():
    scan = synth.scan_from_config("c1", seed=0)
    prob = O.Problem.from_scan(scan)
    x = np.random.default_rng(4).standard_normal((scan.n_pix, 3))
    ref = O.apply_A(prob, x)
    for prec, tol in ((MM.MM_FP64, TOL64), (MM.MM_FP32_MIXED, TOL32)):
        c = ctx_for(scan, prec)
        assert_close(c.apply_A(x)[0], ref, tol)


@pytest.mark.parametrize("prec,products", [(MM.MM_FP64, 1), (MM.MM_FP32_MIXED, 1), (MM.MM_FP32_MIXED, 2)])
@pytest.mark.parametrize("fft_len", [0, 1152, 4608, 8192])
def test_rhs_matches_oracle(prec, products, fft_len):
    """b = P^T W d to float64 accuracy: native float64 or double-float products."""
    scan, d, _ = scan_and_tod(SMALL, seed=5, flag_frac=0.01)
    prob = O.Problem.from_scan(scan)
    c = ctx_for(scan, prec, 2 if fft_len else 0, fft_len=fft_len)
    c.set_option("fp64_products", products)
    tod = d.astype(c.tod_dtype)
    b = c.rhs(tod)
    ref = O.rhs(prob, tod.astype(np.float64))
    assert_close(b[0], ref, TOL64)


def test_bd_build_and_apply_match_oracle():
    scan = synth.make_scan(seed=6, flag_frac=0.02, **SMALL)
    # make two pixels degenerate: a single angle and a single hit
    scan.psi[scan.pix == 5] = 0.3
    scan.pix[(scan.pix == 9)] = -1
    scan.pix[100] = 9
    prob, mbd, good = oracle_problem(scan)
    c = ctx_for(scan)
    dropped = c.build_bd(1e-3)
    assert dropped == int((~good).sum())
    r = np.random.default_rng(6).standard_normal((scan.n_pix, 3))
    z = c.apply_precond(MM.MM_PRECOND_BD, r)
    assert_close(z[0], O.bd_apply(mbd, r), 1e-12)
    # A after flagging equals the oracle's A on the flagged pointing
    x = np.random.default_rng(7).standard_normal((scan.n_pix, 3))
    assert_close(c.apply_A(x)[0], O.apply_A(prob, x), TOL64)


def _oracle_solution(prob, mbd, b):
    return O.pcg(lambda v: O.apply_A(prob, v).reshape(-1), lambda v: O.bd_apply(mbd, v).reshape(-1),
                 b.reshape(-1), tol=1e-13, max_iter=5000)[0]


@pytest.mark.parametrize("prec", [MM.MM_FP64, MM.MM_FP32_MIXED])
def test_solve_bd_matches_oracle(prec):
    scan, d, _ = scan_and_tod(SMALL, seed=8)
    prob, mbd, good = oracle_problem(scan)
    c = ctx_for(scan, prec)
    c.build_bd()
    tod = d.astype(c.tod_dtype)
    x, info = c.solve(tod, MM.MM_PRECOND_BD, tol=1e-10, max_iter=2000)
    assert info[0]["status"] == "MM_OK"
    assert info[0]["true_rel_res"] < 1e-9
    b = O.rhs(prob, tod.astype(np.float64))
    xo = _oracle_solution(prob, mbd, b)
    assert_close(x[0], xo, 1e-6)


@pytest.mark.parametrize("filt,fft_len", [(1, 0), (2, 4608), (2, 8192)])
def test_fp64_solve_with_double_float_products(filt, fft_len):
    """MM_FP64 with "fp64_products" = 2: every operator product of the solve (b, PCG, Arnoldi, A Z,
    the true residual) and mm_apply_A run in double-float arithmetic; A x matches the oracle to
    1e-11 and the M_BD and M_2l maps match the oracle map."""
    scan, d, _ = scan_and_tod(SMALL, seed=25, flag_frac=0.01)
    prob, mbd, good = oracle_problem(scan)
    c = ctx_for(scan, MM.MM_FP64, filt, fft_len=fft_len)
    c.set_option("fp64_products", 2)
    c.build_bd()
    xr = np.random.default_rng(25).standard_normal((scan.n_pix, 3))
    assert_close(c.apply_A(xr)[0], O.apply_A(prob, xr), TOL64)
    x, info = c.solve(d, MM.MM_PRECOND_BD, tol=1e-10, max_iter=2000)
    assert info[0]["status"] == "MM_OK" and info[0]["true_rel_res"] < 1e-9
    xo = _oracle_solution(prob, mbd, O.rhs(prob, d))
    assert_close(x[0], xo, 1e-6)
    k = c.build_coarse(None, m_max=60, eps_arn=1e-8, k=16)
    assert k >= 4
    x2, i2 = c.solve(d, MM.MM_PRECOND_2L, tol=1e-10, max_iter=2000)
    assert i2[0]["status"] == "MM_OK"
    assert_close(x2[0], xo, 1e-6)
    assert i2[0]["iters"] <= info[0]["iters"]
    c.close()


@pytest.mark.parametrize("products", [1, 2])
def test_mixed_true_residual_matches_oracle(products):
    """The mixed-precision solve forms its refinement residual as P^T W (d - P x) in one
    float64-accurate pass (native float64 or double-float); the residual it reports for the
    returned map equals the oracle's ||b - A x|| / ||b|| on that map."""
    scan, d, _ = scan_and_tod(SMALL, seed=23, flag_frac=0.01)
    prob, mbd, good = oracle_problem(scan)
    c = ctx_for(scan, MM.MM_FP32_MIXED)
    c.set_option("fp64_products", products)
    c.build_bd()
    tod = d.astype(c.tod_dtype)
    for tol in (1e-6, 1e-9):
        x, info = c.solve(tod, MM.MM_PRECOND_BD, tol=tol, max_iter=2000)
        assert info[0]["status"] == "MM_OK"
        b = O.rhs(prob, tod.astype(np.float64))
        r = b - O.apply_A(prob, x[0])
        ref = np.linalg.norm(r) / np.linalg.norm(b)
        assert ref <= tol
        # double-float / float64 rounding of the pass: ~1e-13 of ||b||, far below the residual
        assert abs(info[0]["true_rel_res"] - ref) <= 1e-3 * ref + 1e-11


def test_mixed_true_residual_uneven_batch():
    """The same for a batch of right-hand sides of uneven length (one pass for all of them)."""
    cfg = dict(nx=8, ny=8, n_det=4, n_t=8192, n_int=8, half_bw=32, f_knee=1.0)
    scan = synth.make_scan(seed=24, **cfg)
    lens = np.array([8192, 5001, 6400], dtype=np.int64)
    tods = np.stack([synth.make_tod(scan, synth.make_sky(scan.n_pix, 200 + i), synth.make_noise(scan, 200 + i))
                     for i in range(len(lens))]).astype(np.float32)
    c = ctx_for(scan, MM.MM_FP32_MIXED)
    c.build_bd()
    x, info = c.solve(tods, MM.MM_PRECOND_BD, tol=1e-9, max_iter=3000, rhs_len=lens)
    _, _, good = oracle_problem(scan)
    for i, L in enumerate(lens):
        assert info[i]["status"] == "MM_OK"
        prob, mbd, idx = truncated_problem(scan, int(L), good=good)
        b = O.rhs(prob, tods[i][idx].astype(np.float64))
        ref = np.linalg.norm(b - O.apply_A(prob, x[i])) / np.linalg.norm(b)
        assert ref <= 1e-9
        assert abs(info[i]["true_rel_res"] - ref) <= 1e-3 * ref + 1e-11


def test_signal_only_recovers_sky():
    scan, d, s = scan_and_tod(SMALL, seed=9, noise=False)
    prob, mbd, good = oracle_problem(scan)
    s[~good] = 0
    d = synth.make_tod(scan, s, None)
    c = ctx_for(scan)
    c.build_bd()
    x, info = c.solve(d, MM.MM_PRECOND_BD, tol=1e-12, max_iter=3000)
    assert_close(x[0], s, 1e-8)


def test_white_noise_converges_in_one_iteration():
    scan, d, _ = scan_and_tod(dict(SMALL, half_bw=0, f_knee=0.0), seed=10)
    c = ctx_for(scan)
    c.build_bd()
    x, info = c.solve(d, MM.MM_PRECOND_BD, tol=1e-10, max_iter=50)
    assert info[0]["iters"] == 1


def test_coarse_space_identities_and_ritz_values():
    scan, d, _ = scan_and_tod(SMALL, seed=11)
    prob, mbd, good = oracle_problem(scan)
    c = ctx_for(scan)
    c.build_bd()
    b = c.rhs(d)
    k = c.build_coarse(b[0], m_max=12, eps_arn=1e-14, k=6)
    assert k == 6
    Z, ritz = c.get_coarse()
    # oracle Arnoldi from the same start
    A_fn = lambda v: O.apply_A(prob, v).reshape(-1)  # noqa: E731
    M_fn = lambda v: O.bd_apply(mbd, v).reshape(-1)  # noqa: E731
    bo = O.rhs(prob, d).reshape(-1)
    W, H, m = O.arnoldi(lambda v: M_fn(A_fn(v)), M_fn(bo), 12, 1e-14)
    Zo, vals = O.ritz_basis(W, H, m, 6)
    np.testing.assert_allclose(np.sort(ritz), np.sort(vals), rtol=1e-7, atol=1e-9)
    # same subspace: projector difference
    Zg = Z.reshape(k, -1).T
    Pg = Zg @ Zg.T
    Po = Zo @ Zo.T
    assert np.linalg.norm(Pg - Po) < 1e-6
    # Eq. ident: M_2l A Z = Z, through the library's own operators
    AZ = c.apply_A(Z)
    MAZ = c.apply_precond(MM.MM_PRECOND_2L, AZ)
    assert_close(MAZ, Z, 1e-10)
    # M_2l A y = M_BD A y for y with Z^T A y = 0
    y = np.random.default_rng(11).standard_normal((scan.n_pix, 3))
    y[~good] = 0
    Ay = c.apply_A(y)[0].reshape(-1)
    AZf = AZ.reshape(k, -1).T
    E = Zg.T @ AZf
    y = y.reshape(-1) - Zg @ np.linalg.solve(E, AZf.T @ y.reshape(-1))
    y = y.reshape(scan.n_pix, 3)
    Ay = c.apply_A(y)
    np.testing.assert_allclose(c.apply_precond(MM.MM_PRECOND_2L, Ay), c.apply_precond(MM.MM_PRECOND_BD, Ay),
                               atol=1e-9 * np.abs(Ay).max())


@pytest.mark.parametrize("prec", [MM.MM_FP64, MM.MM_FP32_MIXED])
def test_solve_2l_beats_bd_and_matches_oracle(prec):
    cfg = dict(nx=8, ny=8, n_det=4, n_t=2048, n_int=2, half_bw=64, f_knee=2.0)
    scan, d, _ = scan_and_tod(cfg, seed=12)
    prob, mbd, good = oracle_problem(scan)
    c = ctx_for(scan, prec)
    c.build_bd()
    tod = d.astype(c.tod_dtype)
    xbd, ibd = c.solve(tod, MM.MM_PRECOND_BD, tol=1e-8, max_iter=2000)
    k = c.build_coarse(None, m_max=60, eps_arn=1e-10, k=8)
    assert k == 8
    x2l, i2l = c.solve(tod, MM.MM_PRECOND_2L, tol=1e-8, max_iter=2000)
    assert i2l[0]["status"] == "MM_OK" and ibd[0]["status"] == "MM_OK"
    assert i2l[0]["iters"] < ibd[0]["iters"]
    xo = _oracle_solution(prob, mbd, O.rhs(prob, tod.astype(np.float64)))
    assert_close(x2l[0], xo, 1e-6)
    assert_close(xbd[0], xo, 1e-6)


def test_batched_uneven_lengths_match_standalone_and_oracle():
    cfg = dict(nx=8, ny=8, n_det=4, n_t=8192, n_int=8, half_bw=32, f_knee=1.0)
    scan = synth.make_scan(seed=13, **cfg)
    lens = np.array([8192, 5000, 6143, 4097, 7777], dtype=np.int64)
    tods = np.stack([synth.make_tod(scan, synth.make_sky(scan.n_pix, 100 + i), synth.make_noise(scan, 100 + i))
                     for i in range(len(lens))])
    c = ctx_for(scan)
    c.build_bd()
    xb, ib = c.solve(tods, MM.MM_PRECOND_BD, tol=1e-10, max_iter=3000, rhs_len=lens)
    _, _, good = oracle_problem(scan)
    for i, L in enumerate(lens):
        assert ib[i]["status"] == "MM_OK"
        xs, is_ = c.solve(tods[i:i + 1], MM.MM_PRECOND_BD, tol=1e-10, max_iter=3000, rhs_len=lens[i:i + 1])
        assert_close(xb[i], xs[0], 1e-8)
        prob, mbd, idx = truncated_problem(scan, int(L), good=good)
        b = O.rhs(prob, tods[i][idx])
        xo = _oracle_solution(prob, mbd, b)
        assert_close(xb[i], xo, 1e-6)


def test_block_prefix_coarse_products_match_direct():
    """Uneven-length two-level batch: A_i Z from block-prefix products (whole blocks once per coarse
    space, plus each detector's partly covered block) gives the same preconditioner as forming every
    A_i Z directly -- same iteration counts and maps; an inconsistent A_i Z would change the counts."""
    cfg = dict(nx=8, ny=8, n_det=4, n_t=8192, n_int=8, half_bw=32, f_knee=1.0)
    scan = synth.make_scan(seed=25, **cfg)
    lens = np.array([8192, 5000, 6144, 4097, 1024, 7777], dtype=np.int64)
    tods = np.stack([synth.make_tod(scan, synth.make_sky(scan.n_pix, 300 + i), synth.make_noise(scan, 300 + i))
                     for i in range(len(lens))])
    res = {}
    for prefix in (0, 1):
        c = ctx_for(scan)
        c.set_option("coarse_prefix", prefix)
        c.set_option("coarse_fallback", 0)   # every right-hand side runs M_2l
        c.build_bd()
        b = c.rhs(tods[0])
        assert c.build_coarse(b[0], m_max=40, eps_arn=1e-12, k=12) == 12
        res[prefix] = c.solve(tods, MM.MM_PRECOND_2L, tol=1e-10, max_iter=500, rhs_len=lens)
        # twice: the second batch reuses the block-prefix products
        x2, i2 = c.solve(tods, MM.MM_PRECOND_2L, tol=1e-10, max_iter=500, rhs_len=lens)
        assert [i["iters"] for i in i2] == [i["iters"] for i in res[prefix][1]]
        c.close()
    (x0, i0), (x1, i1) = res[0], res[1]
    for r in range(len(lens)):
        assert i0[r]["status"] == "MM_OK" and i1[r]["status"] == "MM_OK"
        assert abs(i0[r]["iters"] - i1[r]["iters"]) <= 1
        # the 1024-sample right-hand side (whole blocks only, no partial block) leaves pixels seen a
        # few times: both maps meet the residual, but their difference scales with its condition number
        if lens[r] >= 4096:
            assert_close(x1[r], x0[r], 1e-8)


def test_device_pointers_and_stepwise_api():
    torch = pytest.importorskip("torch")
    scan, d, _ = scan_and_tod(SMALL, seed=14)
    c = ctx_for(scan)
    c.build_bd()
    dt = torch.from_numpy(d).cuda()
    x_host, info_h = c.solve(d, MM.MM_PRECOND_BD, tol=1e-9)
    x_dev, info_d = c.solve(dt, MM.MM_PRECOND_BD, tol=1e-9)
    assert_close(x_dev.cpu().numpy()[0], x_host[0], 1e-9)
    c.solve_begin(d, MM.MM_PRECOND_BD, tol=1e-9)
    done = False
    steps = 0
    while not done:
        done = c.solve_step(3)
        steps += 1
    x_step, info_s = c.solve_end()
    assert_close(x_step[0], x_host[0], 1e-9)
    assert info_s[0]["iters"] == info_h[0]["iters"]


def test_errors_are_reported():
    c = MM.Context(0, None, MM.MM_FP64)
    with pytest.raises(MM.MapMakerError) as e:
        c.build_bd()
    assert e.value.status == MM.MM_ERR_STATE
    scan = synth.make_scan(seed=0, **SMALL)
    bad = scan.pix.copy()
    bad[3] = scan.n_pix
    with pytest.raises(MM.MapMakerError) as e:
        c.setup_pointing(bad, scan.psi, scan.block_off, scan.block_band, scan.band, scan.n_pix, scan.n_det)
    assert e.value.status == MM.MM_ERR_ARG
    with pytest.raises(MM.MapMakerError):
        c.set_option("filter", 7)


def test_graph_replay_matches_eager():
    torch = pytest.importorskip("torch")
    cfg = dict(nx=8, ny=8, n_det=4, n_t=8192, n_int=8, half_bw=32, f_knee=1.0)
    scan = synth.make_scan(seed=15, **cfg)
    lens = np.array([8192, 5000, 7000], dtype=np.int64)
    tods = np.stack([synth.make_tod(scan, synth.make_sky(scan.n_pix, 300 + i), synth.make_noise(scan, 300 + i))
                     for i in range(3)])
    stream = torch.cuda.Stream()
    res = []
    for graphs in (0, 1):
        c = MM.Context(0, stream.cuda_stream, MM.MM_FP64)
        c.set_option("graphs", graphs)
        c.set_option("check_every", 5)
        c.setup_scan(scan)
        c.build_bd()
        c.build_coarse(c.rhs(tods[:1])[0], m_max=20, eps_arn=1e-8, k=4)
        x, info = c.solve(tods, MM.MM_PRECOND_2L, tol=1e-10, max_iter=500, rhs_len=lens)
        res.append((x, info))
        c.close()
    for i in range(3):
        assert res[1][1][i]["status"] == "MM_OK"
        assert res[1][1][i]["iters"] == res[0][1][i]["iters"]
        assert_close(res[1][0][i], res[0][0][i], 1e-9)


def test_harvested_lanczos_coarse_space_matches_oracle():
    cfg = dict(nx=8, ny=8, n_det=4, n_t=2048, n_int=2, half_bw=64, f_knee=2.0)
    scan, d, _ = scan_and_tod(cfg, seed=17)
    prob, mbd, good = oracle_problem(scan)
    c = ctx_for(scan)
    c.build_bd()
    m = 14
    c.set_option("harvest", m)
    x, info = c.solve(d, MM.MM_PRECOND_BD, tol=1e-10, max_iter=2000)
    assert info[0]["iters"] > m and c.get_option("harvested") == m
    k = c.build_coarse_from_solve(k=5)
    assert k == 5
    Z, ritz = c.get_coarse()
    A_fn = lambda v: O.apply_A(prob, v).reshape(-1)  # noqa: E731
    M_fn = lambda v: O.bd_apply(mbd, v).reshape(-1)  # noqa: E731
    al, be, V = O.pcg_lanczos(A_fn, M_fn, O.rhs(prob, d).reshape(-1), m)
    vals, Zo, T = O.lanczos_ritz(al, be, V, 5)
    np.testing.assert_allclose(np.sort(ritz), np.sort(vals), rtol=1e-8, atol=1e-10)
    Zg = Z.reshape(k, -1).T
    assert np.linalg.norm(Zg @ Zg.T - Zo @ Zo.T) < 1e-6
    AZ = c.apply_A(Z)
    assert_close(c.apply_precond(MM.MM_PRECOND_2L, AZ), Z, 1e-10)
    x2, i2 = c.solve(d, MM.MM_PRECOND_2L, tol=1e-10, max_iter=2000)
    assert i2[0]["status"] == "MM_OK" and i2[0]["iters"] < info[0]["iters"]
    assert_close(x2[0], x[0], 1e-7)


@pytest.mark.parametrize("prec", [MM.MM_FP64, MM.MM_FP32_MIXED])
def test_batched_two_level_uneven_lengths(prec):
    """Shared basis Z, per right-hand side AZ_i and E_i: every map matches its own problem."""
    cfg = dict(nx=8, ny=8, n_det=4, n_t=8192, n_int=8, half_bw=64, f_knee=2.0)
    scan = synth.make_scan(seed=18, **cfg)
    lens = np.array([8192, 4500, 6000, 7333], dtype=np.int64)
    tods = np.stack([synth.make_tod(scan, synth.make_sky(scan.n_pix, 400 + i), synth.make_noise(scan, 400 + i))
                     for i in range(len(lens))])
    c = ctx_for(scan, prec)
    c.set_option("coarse_fallback", 0)   # every right-hand side runs M_2l with its own A_i Z and E_i
    c.build_bd()
    tt = tods.astype(c.tod_dtype)
    c.build_coarse(c.rhs(tt[:1])[0], m_max=40, eps_arn=1e-8, k=8)
    xb, ib = c.solve(tt, MM.MM_PRECOND_2L, tol=1e-9, max_iter=2000, rhs_len=lens)
    xbd, ibd = c.solve(tt, MM.MM_PRECOND_BD, tol=1e-9, max_iter=2000, rhs_len=lens)
    _, _, good = oracle_problem(scan)
    for i, L in enumerate(lens):
        assert ib[i]["status"] == "MM_OK"
        assert ib[i]["iters"] <= ibd[i]["iters"]
        prob, mbd, idx = truncated_problem(scan, int(L), good=good)
        xo = _oracle_solution(prob, mbd, O.rhs(prob, tt[i][idx].astype(np.float64))).reshape(-1, 3)
        well = np.abs(mbd).reshape(scan.n_pix, -1).sum(axis=1) > 0   # pixels this prefix determines
        assert_close(xb[i][well], xo[well], 1e-6)


def test_uneven_two_level_batch_deflates_like_the_oracle():
    """A basis from the full-length operator deflates prefixes of the scan (Sect. 7's reuse of one
    basis): each right-hand side of an uneven batch takes as many two-level products as the
    oracle's PCG with M_2l built from the same Z and that prefix's own A_i Z, E_i and M_BD,i
    (Sect. 3.2, Eq. m2l), within 2, and clearly fewer than M_BD."""
    cfg = dict(nx=16, ny=16, n_det=4, n_t=32768, n_int=8, half_bw=128, f_knee=1.0)
    scan = synth.make_scan(seed=19, **cfg)
    lens = np.array([32768, 28672, 20000, 16384], dtype=np.int64)   # 20000: a partly covered block
    tods = np.stack([synth.make_tod(scan, synth.make_sky(scan.n_pix, 410 + i), synth.make_noise(scan, 410 + i))
                     for i in range(len(lens))])
    c = ctx_for(scan, MM.MM_FP64)
    c.set_option("coarse_fallback", 0)
    c.build_bd()
    k = c.build_coarse(c.rhs(tods[:1])[0], m_max=150, eps_arn=1e-12, k=16)
    Z, _ = c.get_coarse()
    _, ib = c.solve(tods, MM.MM_PRECOND_2L, tol=1e-8, max_iter=2000, rhs_len=lens)
    _, ibd = c.solve(tods, MM.MM_PRECOND_BD, tol=1e-8, max_iter=2000, rhs_len=lens)
    c.close()
    _, _, good = oracle_problem(scan)
    Zf = Z.reshape(k, -1).T
    for i, L in enumerate(lens):
        prob, mbd, idx = truncated_problem(scan, int(L), good=good)
        A = lambda v: O.apply_A(prob, v.reshape(-1, 3)).reshape(-1)  # noqa: E731
        Mb = lambda v: O.bd_apply(mbd, v).reshape(-1)  # noqa: E731
        AZ, _, Lc = O.coarse_space(A, Zf)
        b = O.rhs(prob, tods[i][idx]).reshape(-1)
        _, io = O.pcg(A, lambda v: O.m2l_apply(v, Mb, Zf, AZ, Lc), b, tol=1e-8, max_iter=2000)
        _, iob = O.pcg(A, Mb, b, tol=1e-8, max_iter=2000)
        assert abs(ib[i]["iters"] - io["iters"]) <= 2, (i, int(L), ib[i]["iters"], io["iters"])
        assert abs(ibd[i]["iters"] - iob["iters"]) <= 1, (i, int(L), ibd[i]["iters"], iob["iters"])
        assert ib[i]["precond_used"] == "M_2l"


def test_uneven_two_level_batch_with_a_prefix_blind_to_part_of_the_basis():
    """A prefix of about half the scan sees about half the patch (the elevation drifts across it
    once per timeline), so some direction of span Z lies where A_i vanishes and E_i = Z^T A_i Z is
    only semi-definite.  The batch still solves: that right-hand side keeps the columns of Z a
    pivoted Cholesky factorisation of E_i retains (option coarse_rank_min reports how many), takes
    no more products than M_BD, and its map matches the oracle on the pixels the prefix observes."""
    scan = synth.make_scan(nx=32, ny=32, n_det=8, n_t=1 << 17, n_int=32, half_bw=512, f_knee=1.0, seed=0)
    lens = np.array([1 << 17, 99079, 67820], dtype=np.int64)
    tods = np.stack([synth.make_tod(scan, synth.make_sky(scan.n_pix, 1000 + i), synth.make_noise(scan, 1000 + i))
                     for i in range(len(lens))])
    c = ctx_for(scan, MM.MM_FP64)
    c.set_option("coarse_fallback", 0)
    c.build_bd(1e-3)
    k = c.build_coarse(c.rhs(tods[:1])[0], m_max=200, eps_arn=1e-12, k=32)
    x2, i2 = c.solve(tods, MM.MM_PRECOND_2L, tol=1e-10, max_iter=2000, rhs_len=lens)
    assert c.get_option("coarse_rank_min") < k
    _, ib = c.solve(tods, MM.MM_PRECOND_BD, tol=1e-10, max_iter=2000, rhs_len=lens)
    c.close()
    _, _, good = oracle_problem(scan)
    for i, L in enumerate(lens):
        assert i2[i]["status"] == "MM_OK" and i2[i]["iters"] <= ib[i]["iters"], (i, i2[i]["iters"], ib[i]["iters"])
        if i == 2:
            prob, mbd, idx = truncated_problem(scan, int(L), good=good)
            xo = _oracle_solution(prob, mbd, O.rhs(prob, tods[i][idx])).reshape(-1, 3)
            well = np.abs(mbd).reshape(scan.n_pix, -1).sum(axis=1) > 0
            assert well.sum() < 0.8 * scan.n_pix          # the prefix leaves part of the map unobserved
            assert_close(x2[i][well], xo[well], 1e-6, "prefix blind to part of Z vs oracle")


def test_status_codes_not_converged_and_breakdown():
    scan, d, _ = scan_and_tod(SMALL, seed=23)
    c = ctx_for(scan)
    c.build_bd()
    x, info = c.solve(d, MM.MM_PRECOND_BD, tol=1e-14, max_iter=3)
    assert info[0]["status"] == "MM_ERR_NOT_CONVERGED" and info[0]["iters"] == 3
    assert np.isfinite(x).all()
    # an indefinite weight (negative diagonal) makes p^T A p <= 0: reported, not hidden
    bad = synth.make_scan(seed=24, **dict(SMALL, half_bw=4))
    bad.band = -np.abs(bad.band)
    cb = ctx_for(bad)
    cb.build_bd(0.0)
    with pytest.raises(MM.MapMakerError) as e:
        cb.solve(d, MM.MM_PRECOND_BD, tol=1e-10, max_iter=50)
    assert e.value.status == MM.MM_ERR_BREAKDOWN


def test_argument_and_state_errors():
    c = MM.Context(0, None, MM.MM_FP64)
    scan = synth.make_scan(seed=25, **SMALL)
    with pytest.raises(MM.MapMakerError) as e:
        c.solve(np.zeros(scan.n_samples), MM.MM_PRECOND_BD)
    assert e.value.status == MM.MM_ERR_STATE
    bo = scan.block_off.copy()
    bo[1] = bo[2]                                         # empty block
    with pytest.raises(MM.MapMakerError) as e:
        c.setup_pointing(scan.pix, scan.psi, bo, scan.block_band, scan.band, scan.n_pix, scan.n_det)
    assert e.value.status == MM.MM_ERR_ARG
    c.setup_scan(scan)
    c.build_bd()
    with pytest.raises(MM.MapMakerError) as e:
        c.solve(np.zeros(scan.n_samples), MM.MM_PRECOND_2L)   # no coarse space yet
    assert e.value.status == MM.MM_ERR_STATE
    with pytest.raises(MM.MapMakerError) as e:
        c.build_coarse(None, m_max=10, k=600)   # above the 512 limit
    assert e.value.status == MM.MM_ERR_ARG
    # an all-zero timeline solves to the zero map at once
    x, info = c.solve(np.zeros(scan.n_samples), MM.MM_PRECOND_BD, tol=1e-8)
    assert info[0]["iters"] == 0 and np.all(x == 0)


def test_single_pixel_single_block_extremes():
    """n_pix = 1, one detector, one block, band wider than the block."""
    rng = np.random.default_rng(26)
    n = 300
    pix = np.zeros(n, dtype=np.int32)
    psi = (rng.random(n) * np.pi).astype(np.float32)
    band = synth.toeplitz_band(400, 1.0)[None, :]
    prob = O.Problem(pix, psi, np.array([0, n]), band, np.array([0]), 1)
    x = rng.standard_normal((1, 3))
    for filt in (1, 2):
        c = MM.Context(0, None, MM.MM_FP64)
        c.set_option("filter", filt)
        c.setup_pointing(pix, psi, np.array([0, n]), np.array([0]), band, 1, 1)
        assert_close(c.apply_A(x)[0], O.apply_A(prob, x), TOL64)
        c.close()


def test_coarse_space_export_import_round_trip_and_fingerprint():
    """A checkpoint of the coarse space (Z, A Z, E^-1, Ritz values) installs into a fresh context on
    the same scan and gives the same M_2l; a checkpoint of another scan, a truncated or corrupted
    buffer, or another product precision is refused."""
    scan, d, _ = scan_and_tod(SMALL, seed=51)
    c = ctx_for(scan)
    c.build_bd()
    k = c.build_coarse(c.rhs(d)[0], m_max=20, eps_arn=1e-12, k=6)
    blob = c.export_coarse()
    x = np.random.default_rng(51).standard_normal((2, scan.n_pix, 3))
    y = c.apply_precond(MM.MM_PRECOND_2L, x)
    x1, i1 = c.solve(d, MM.MM_PRECOND_2L, tol=1e-10)
    c2 = ctx_for(scan)
    c2.build_bd()
    c2.import_coarse(blob)
    Z1, r1 = c.get_coarse()
    Z2, r2 = c2.get_coarse()
    assert Z2.shape[0] == k and np.array_equal(Z1, Z2) and np.array_equal(r1, r2)
    # same Z, A Z and E^-1; M_BD of the two contexts agrees to rounding (its sums use atomics)
    assert_close(c2.apply_precond(MM.MM_PRECOND_2L, x), y, 1e-13)
    x2, i2 = c2.solve(d, MM.MM_PRECOND_2L, tol=1e-10)
    assert abs(i2[0]["iters"] - i1[0]["iters"]) <= 1
    assert_close(x2[0], x1[0], 1e-11)
    # another scan (one angle changed), another precision, damaged buffers: refused
    other = copy.copy(scan)
    other.psi = scan.psi.copy()
    other.psi[100] += 0.5
    c3 = ctx_for(other)
    c3.build_bd()
    c4 = ctx_for(scan, MM.MM_FP32_MIXED)
    c4.build_bd()
    bad = bytearray(blob)
    bad[0] ^= 1
    for ctx, data in ((c3, blob), (c4, blob), (c2, blob[:-8]), (c2, bytes(bad))):
        with pytest.raises(MM.MapMakerError) as e:
            ctx.import_coarse(data)
        assert e.value.status == MM.MM_ERR_ARG
    for ctx in (c, c2, c3, c4):
        ctx.close()


def test_uneven_batch_falls_back_to_bd_for_other_lengths():
    """With "coarse_fallback" (default) a two-level batch of uneven length runs M_2l only for the
    right-hand sides of the basis's own length: the others run M_BD (same products and maps as an M_BD
    batch), and a batch with none of that length runs M_BD throughout."""
    cfg = dict(nx=8, ny=8, n_det=4, n_t=8192, n_int=8, half_bw=64, f_knee=2.0)
    scan = synth.make_scan(seed=52, **cfg)
    lens = np.array([8192, 4500, 6000, 8192, 7333], dtype=np.int64)
    tods = np.stack([synth.make_tod(scan, synth.make_sky(scan.n_pix, 500 + i), synth.make_noise(scan, 500 + i))
                     for i in range(len(lens))])
    c = ctx_for(scan)
    c.build_bd()
    c.build_coarse(c.rhs(tods[:1])[0], m_max=40, eps_arn=1e-10, k=8)
    assert c.get_option("coarse_len") == 8192
    x2, i2 = c.solve(tods, MM.MM_PRECOND_2L, tol=1e-10, max_iter=2000, rhs_len=lens)
    xb, ib = c.solve(tods, MM.MM_PRECOND_BD, tol=1e-10, max_iter=2000, rhs_len=lens)
    for i, L in enumerate(lens):
        assert i2[i]["status"] == "MM_OK" and ib[i]["status"] == "MM_OK"
        assert ib[i]["precond_used"] == "M_BD"
        if L == 8192:
            assert i2[i]["precond_used"] == "M_2l" and i2[i]["iters"] < ib[i]["iters"]
        else:
            assert i2[i]["precond_used"] == "M_BD"
            assert abs(i2[i]["iters"] - ib[i]["iters"]) <= 1
            assert_close(x2[i], xb[i], 1e-9)
    short = lens[[1, 2, 4]]
    x3, i3 = c.solve(tods[[1, 2, 4]], MM.MM_PRECOND_2L, tol=1e-10, max_iter=2000, rhs_len=short)
    for j, i in enumerate((1, 2, 4)):
        assert i3[j]["precond_used"] == "M_BD" and i3[j]["iters"] == ib[i]["iters"]
        assert_close(x3[j], xb[i], 1e-9)
    c.close()
