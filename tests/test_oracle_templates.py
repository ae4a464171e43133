"""Pins of the template-filter oracle (CPU) against facts the paper and the mathematics fix.

Sect. 2.1 (Eq. filt, Eq. filtnoise, Eq. unb), Sect. 4 (polynomial and ground
templates), Sect. 5.1 (simplified filter F_B W^-1 F_G W^-1 F_B, polarisation
from d^-).  None of these pins re-calls the oracle's own arithmetic: the
Legendre columns are checked against their textbook closed forms, the filter
against the subspaces it must annihilate or preserve, the ground fit
against a brute-force loop, the estimator against exact recovery.
"""
import copy
import json
import os

import numpy as np
import pytest

import oracle as O
import synth


def tproblem(nx=8, ny=4, n_det=4, n_t=512, n_int=2, order=1, ground=True, qu_only=True, seed=3, flag_frac=0.0,
             w_scale=1.0, hwp=False):
    scan = synth.make_scan(nx=nx, ny=ny, n_det=n_det, n_t=n_t, n_int=n_int, half_bw=0, f_knee=0.0, seed=seed,
                           flag_frac=flag_frac, hwp=hwp)
    sub_off, az, nb = synth.make_templates(scan)
    w_block = scan.band[scan.block_band, 0] * w_scale * (1.0 + 0.25 * np.arange(scan.n_blocks))
    tp = O.TemplateProblem(scan.pix, scan.psi, scan.block_off, w_block, scan.n_pix, sub_off, order,
                           az if ground else None, nb if ground else 0, qu_only)
    return scan, tp


def test_legendre_columns_are_the_textbook_polynomials():
    m = 37
    u = 2.0 * (np.arange(m) + 0.5) / m - 1.0
    B = O.legendre_basis(m, 3)
    np.testing.assert_allclose(B[:, 0], 1.0)
    np.testing.assert_allclose(B[:, 1], u)
    np.testing.assert_allclose(B[:, 2], 0.5 * (3 * u ** 2 - 1), atol=1e-15)
    np.testing.assert_allclose(B[:, 3], 0.5 * (5 * u ** 3 - 3 * u), atol=1e-15)


@pytest.mark.parametrize("order", [0, 1, 2, 3])
def test_polynomial_filter_annihilates_its_templates(order):
    """F_B B = 0 (Eq. filt): any polynomial of degree <= K in the sample index on each subscan."""
    scan, tp = tproblem(order=order, ground=False)
    rng = np.random.default_rng(order)
    y = np.zeros(scan.n_samples)
    for s in range(len(tp.sub_off) - 1):
        a, b = tp.sub_off[s], tp.sub_off[s + 1]
        i = np.arange(b - a, dtype=np.float64)
        y[a:b] = sum(rng.standard_normal() * i ** j for j in range(order + 1))
    out = O.filter_poly(y, tp.sample_weight(), tp.sub_off, order)
    assert np.abs(out).max() <= 1e-9 * np.abs(y).max()
    # one degree more is not annihilated
    a, b = tp.sub_off[0], tp.sub_off[1]
    z = np.zeros(scan.n_samples)
    z[a:b] = np.arange(b - a, dtype=np.float64) ** (order + 1)
    assert np.abs(O.filter_poly(z, tp.sample_weight(), tp.sub_off, order)).max() > 1e-3


def test_subscans_shorter_than_the_order_are_removed_entirely():
    """m <= K samples: the fit space (order m - 1) spans every timeline on the subscan, so F_B gives 0."""
    y = np.arange(1.0, 8.0)
    sub_off = np.array([0, 1, 3, 7])
    out = O.filter_poly(y, np.ones(7), sub_off, 3)
    assert np.abs(out[:3]).max() < 1e-12
    assert np.abs(out[3:]).max() < 1e-12          # 4 samples, cubic fit: exact as well


def test_polynomial_filter_keeps_the_orthogonal_complement():
    """A timeline orthogonal to every subscan's polynomials passes as W y (F_B = W - W B (...) B^T W)."""
    scan, tp = tproblem(order=2, ground=False)
    rng = np.random.default_rng(5)
    wv = tp.sample_weight()
    y = rng.standard_normal(scan.n_samples)
    for s in range(len(tp.sub_off) - 1):
        a, b = tp.sub_off[s], tp.sub_off[s + 1]
        V = np.vander(np.linspace(0.0, 1.0, b - a), 3, increasing=True)[:, :min(3, b - a)]
        Q, _ = np.linalg.qr(V)
        y[a:b] -= Q @ (Q.T @ y[a:b])
    np.testing.assert_allclose(O.filter_poly(y, wv, tp.sub_off, 2), wv * y, atol=1e-12)


def test_ground_filter_is_the_bin_mean_removal():
    """F_G y = w (y - mean of y over the sample's azimuth bin in its block), by a brute-force loop."""
    scan, tp = tproblem(order=-1, ground=True, flag_frac=0.05)
    rng = np.random.default_rng(6)
    y = rng.standard_normal(scan.n_samples)
    wv = tp.sample_weight()
    ref = np.empty_like(y)
    for blk in range(scan.n_blocks):
        a, b = scan.block_off[blk], scan.block_off[blk + 1]
        for t in range(a, b):
            same = [u for u in range(a, b) if tp.az_bin[u] == tp.az_bin[t]]
            ref[t] = wv[t] * (y[t] - sum(y[u] for u in same) / len(same))
    np.testing.assert_allclose(O.filter_ground(y, wv, scan.block_off, tp.az_bin, tp.n_az_bins), ref, atol=1e-12)
    # the ground template itself (any function of the bin, per block) is annihilated
    g = rng.standard_normal((scan.n_blocks, tp.n_az_bins))
    yg = np.concatenate([g[blk][tp.az_bin[scan.block_off[blk]:scan.block_off[blk + 1]]]
                         for blk in range(scan.n_blocks)])
    assert np.abs(O.filter_ground(yg, wv, scan.block_off, tp.az_bin, tp.n_az_bins)).max() < 1e-12


def test_simplified_filter_symmetric_positive_and_kills_polynomials():
    """F = F_B W^-1 F_G W^-1 F_B is symmetric (Sect. 5.1), positive semi-definite, and F B = 0."""
    scan, tp = tproblem(order=1, ground=True)
    rng = np.random.default_rng(7)
    u, v = rng.standard_normal((2, scan.n_samples))
    Fu, Fv = O.apply_F(tp, u), O.apply_F(tp, v)
    assert abs(v @ Fu - u @ Fv) <= 1e-12 * np.linalg.norm(Fu) * np.linalg.norm(v)
    assert u @ Fu >= 0 and v @ Fv >= 0
    a, b = tp.sub_off[3], tp.sub_off[4]
    p = np.zeros(scan.n_samples)
    p[a:b] = 2.0 - 0.5 * np.arange(b - a)
    assert np.abs(O.apply_F(tp, p)).max() < 1e-10


def test_dense_assembly_matches_matrix_free():
    """A = P^T F P assembled column by column equals the matrix-free product and is symmetric."""
    scan, tp = tproblem(order=1, ground=True, n_t=256)
    n = 3 * scan.n_pix
    A = np.column_stack([O.apply_A_T(tp, e.reshape(-1, 3)).reshape(-1) for e in np.eye(n)])
    np.testing.assert_allclose(A, A.T, atol=1e-10 * np.abs(A).max())
    x = np.random.default_rng(8).standard_normal(n)
    np.testing.assert_allclose(A @ x, O.apply_A_T(tp, x.reshape(-1, 3)).reshape(-1), atol=1e-10 * np.abs(A).max())
    # the I rows and columns vanish for the differenced timeline (Eq. d-)
    assert np.abs(A[0::3]).max() == 0.0 and np.abs(A[:, 0::3]).max() == 0.0


def test_constant_intensity_is_a_null_vector_of_the_filtered_d_plus_system():
    """d^+ rows (1, 0, 0): a constant I map gives a constant timeline, which every subscan's P_0
    template removes (Eq. filt), so A 1 = 0 exactly; Q and U rows and columns vanish."""
    scan, tp = tproblem(order=0, ground=False, qu_only=2)
    ones = np.zeros((scan.n_pix, 3))
    ones[:, 0] = 1.0
    assert np.abs(O.apply_A_T(tp, ones)).max() < 1e-12
    x = np.random.default_rng(12).standard_normal((scan.n_pix, 3))
    Ax = O.apply_A_T(tp, x)
    assert np.abs(Ax[:, 1:]).max() == 0.0 and np.abs(Ax[:, 0]).max() > 1e-3
    blocks, hits = O.bd_blocks_T(tp)
    good = O.select_pixels_T(blocks, hits, 2)
    inv = O.bd_inverse_T(blocks, good, 2)
    np.testing.assert_allclose(inv[good, 0, 0] * blocks[good, 0, 0], 1.0)
    assert np.abs(inv[:, 1:, :]).max() == 0.0


def _kept(tp):
    blocks, hits = O.bd_blocks_T(tp)
    good = O.select_pixels_T(blocks, hits, tp.stokes)
    tp = tp.with_pix(O.flag_samples(tp.pix, good))
    blocks, _ = O.bd_blocks_T(tp)
    return tp, good, O.bd_inverse_T(blocks, good, tp.stokes)


def test_filtered_estimator_is_unbiased_under_polynomial_contamination():
    """Eq. unb: d = P s + B a (no noise) gives s back exactly, whatever the template amplitudes."""
    scan, tp = tproblem(order=1, ground=True, n_det=4, n_t=1024, ny=4)
    tp, good, mbd = _kept(tp)
    rng = np.random.default_rng(9)
    s = synth.make_sky(scan.n_pix, 9)
    s[:, 0] = 0.0
    s[~good] = 0.0
    flagged = copy.copy(scan)
    flagged.pix = tp.pix.astype(np.int32)
    d = synth.make_tod(flagged, s, None)
    for k in range(len(tp.sub_off) - 1):
        a, b = tp.sub_off[k], tp.sub_off[k + 1]
        d[a:b] += 30.0 * rng.standard_normal() + 5.0 * rng.standard_normal() * O.legendre_basis(b - a, 1)[:, 1]
    b = O.rhs_T(tp, d).reshape(-1)
    x = O.pcg(lambda v: O.apply_A_T(tp, v).reshape(-1), lambda v: O.bd_apply(mbd, v).reshape(-1), b,
              tol=1e-13, max_iter=5000)[0]
    assert np.linalg.norm(x - s.reshape(-1)) <= 1e-8 * np.linalg.norm(s)


def test_filters_create_small_eigenvalues_that_two_level_removes():
    """Sect. 4.3 / 3.2: the filters leave small eigenvalues of M_BD A that slow PCG with M_BD; deflating
    the k smallest eigenvectors (M_2l) converges in fewer iterations."""
    scan, tp = tproblem(order=1, ground=True, n_det=4, n_t=1024, ny=4, nx=8)
    tp, good, mbd = _kept(tp)
    n = 3 * scan.n_pix
    idx = np.nonzero(np.repeat(good, 3) & np.tile([False, True, True], scan.n_pix))[0]
    A = np.column_stack([O.apply_A_T(tp, e.reshape(-1, 3)).reshape(-1) for e in np.eye(n)[idx]])[idx]
    M = np.column_stack([O.bd_apply(mbd, e.reshape(-1, 3)).reshape(-1) for e in np.eye(n)[idx]])[idx]
    ev, vec = np.linalg.eig(M @ A)
    ev = ev.real
    order = np.argsort(ev)
    assert ev[order[0]] < 0.05 * np.median(ev)
    b = A @ np.random.default_rng(10).standard_normal(len(idx))
    it_bd = O.pcg(lambda v: A @ v, lambda v: M @ v, b, tol=1e-10, max_iter=2000)[1]["iters"]
    Z = np.linalg.qr(vec[:, order[:8]].real)[0]
    AZ, _, L = O.coarse_space(lambda v: A @ v, Z)
    it_2l = O.pcg(lambda v: A @ v, lambda v: O.m2l_apply(v, lambda r: M @ r, Z, AZ, L), b,
                  tol=1e-10, max_iter=2000)[1]["iters"]
    assert it_2l < it_bd


def test_hand_worked_template_filters():
    """Four samples worked by hand (fixture tests/golden/hand_template_filters.json): order-0 and
    order-1 subscan fits, the ground bins alone, and order 1 around the ground bins."""
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "hand_template_filters.json")))
    for case in g["cases"]:
        az = None if case["az_bin"] is None else np.array(case["az_bin"])
        tp = O.TemplateProblem(g["pix"], g["psi"], g["block_off"], g["w_block"], g["n_pix"], g["subscan_off"],
                               case["poly_order"], az, case["n_az_bins"], g["stokes"])
        np.testing.assert_allclose(O.apply_A_T(tp, np.array(g["x"])), np.array(case["Ax"]), atol=1e-14)


def _subset(seed):
    scan, tp = tproblem(order=1, ground=True, n_det=4, n_t=1024, ny=4, nx=8, seed=seed)
    tp, good, mbd = _kept(tp)
    sky = synth.make_sky(scan.n_pix, seed)
    sky[:, 0] = 0.0
    d = synth.make_tod(scan, sky, synth.make_noise(scan, seed))
    A = lambda v: O.apply_A_T(tp, v.reshape(-1, 3)).reshape(-1)  # noqa: E731
    M = lambda v: O.bd_apply(mbd, v).reshape(-1)  # noqa: E731
    return A, M, O.rhs_T(tp, d).reshape(-1)


def test_simplified_reuse_of_a_deflation_basis_across_data_subsets():
    """Sect. 7 (divide and conquer): Ritz vectors computed on one data subset (another raster of the same
    patch) deflate the filtered system of a different subset; M_2l with that basis and the subset's own
    A Z and E needs fewer PCG iterations than M_BD (the "simplified" approach), and a basis from the
    subset itself (the "active" approach) fewer still."""
    A0, M0, b0 = _subset(11)
    W, H, m = O.arnoldi(lambda v: M0(A0(v)), M0(b0), 80, 1e-12)
    Z0, _ = O.ritz_basis(W, H, m, 16)
    for seed in (12, 13):
        A, M, b = _subset(seed)
        it_bd = O.pcg(A, M, b, tol=1e-8, max_iter=3000)[1]["iters"]
        AZ, _, L = O.coarse_space(A, Z0)
        it_simplified = O.pcg(A, lambda v: O.m2l_apply(v, M, Z0, AZ, L), b, tol=1e-8, max_iter=3000)[1]["iters"]
        W1, H1, m1 = O.arnoldi(lambda v: M(A(v)), M(b), 80, 1e-12)
        Z1, _ = O.ritz_basis(W1, H1, m1, 16)
        AZ1, _, L1 = O.coarse_space(A, Z1)
        it_active = O.pcg(A, lambda v: O.m2l_apply(v, M, Z1, AZ1, L1), b, tol=1e-8, max_iter=3000)[1]["iters"]
        assert it_active <= it_simplified < it_bd
