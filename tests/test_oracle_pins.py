"""Pins of the FP64 oracle to facts outside itself (CPU only).

Each test ties an oracle function to a hand-derived fixture, a dense
assembly, a closed form, an invariant the paper states, or a textbook
routine, chosen so that a dropped term, a wrong sign or index, or a band that
leaks across a block edge fails at least one of them.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLD, name)) as f:
        g = json.load(f)
    prob = O.Problem(np.array(g["pix"]), np.array(g["psi"], dtype=np.float32),
                     np.array(g["block_off"]), np.array(g["band"]), np.array(g["block_band"]),
                     g["n_pix"])
    return g, prob


def _tiny(seed=0, **kw):
    cfg = dict(synth.CONFIGS["tiny"])
    cfg.update(kw)
    return synth.make_scan(seed=seed, **cfg)


# ---------------- hand-derived fixtures ----------------

def test_hand_one_pixel():
    g, prob = _load("hand_one_pixel.json")
    A = O.dense_A(prob)
    np.testing.assert_allclose(A, g["A"], atol=1e-6)
    Ax = O.apply_A(prob, np.array(g["x"])).reshape(-1)
    np.testing.assert_allclose(Ax, g["Ax"], atol=1e-6)
    b = O.rhs(prob, np.array(g["d"])).reshape(-1)
    np.testing.assert_allclose(b, g["b"], atol=1e-6)
    blocks, hits = O.bd_blocks(prob)
    np.testing.assert_allclose(blocks[0], g["M_BD_inv"], atol=1e-6)
    assert hits[0] == 3


def test_hand_block_edge():
    g, prob = _load("hand_block_edge.json")
    Ax = O.apply_A(prob, np.array(g["x"])).reshape(-1)
    np.testing.assert_allclose(Ax, g["Ax"], atol=1e-12)


# ---------------- dense assembly and SPD ----------------

@pytest.mark.parametrize("seed", [0, 1, 2])
def test_apply_A_matches_dense(seed):
    scan = _tiny(seed, flag_frac=0.05)
    prob = O.Problem.from_scan(scan)
    A = O.dense_A(prob)
    rng = np.random.default_rng(seed)
    for _ in range(3):
        x = rng.standard_normal(prob.n)
        np.testing.assert_allclose(O.apply_A(prob, x).reshape(-1), A @ x, rtol=1e-12, atol=1e-12 * np.abs(A).sum())


def test_rhs_matches_dense():
    scan = _tiny(3)
    prob = O.Problem.from_scan(scan)
    d = np.random.default_rng(3).standard_normal(scan.n_samples)
    Pm = O.dense_P(prob)
    np.testing.assert_allclose(O.rhs(prob, d).reshape(-1), Pm.T @ O.dense_Ninv(prob) @ d, rtol=1e-12, atol=1e-11)


def _symbol_min(band):
    lam = band.shape[0] - 1
    M = 1 << 14
    h = np.zeros(M)
    h[:lam + 1] = band
    if lam:
        h[M - lam:] = band[1:][::-1]
    return np.fft.rfft(h).real.min()


def test_A_is_spd_and_symbol_bound():
    scan = _tiny(4)
    prob = O.Problem.from_scan(scan)
    A = O.dense_A(prob)
    assert np.allclose(A, A.T, rtol=0, atol=1e-13 * np.abs(A).max())
    ev = np.linalg.eigvalsh(A)
    assert ev[0] > 0
    # x^T A x = y^T W y >= S_min ||P x||^2 >= S_min lambda_min(P^T P) ||x||^2
    Pm = O.dense_P(prob)
    smin = min(_symbol_min(b) for b in scan.band)
    assert smin > 0
    assert ev[0] >= smin * np.linalg.eigvalsh(Pm.T @ Pm)[0] * (1 - 1e-9)


def test_band_symbol_positive_and_white_limit():
    for lam in (0, 3, 64, 512):
        for fk in (0.1, 1.0, 2.0):
            band = synth.toeplitz_band(lam, fk)
            assert _symbol_min(band) > 0
    # no 1/f component: W = I / sigma^2 exactly
    band = synth.toeplitz_band(16, 0.0, sigma=2.0)
    np.testing.assert_allclose(band, np.r_[0.25, np.zeros(16)], atol=1e-15)


# ---------------- M_BD closed form ----------------

def test_white_noise_bd_is_exact_inverse():
    """lambda = 0: W is diagonal, so A = M_BD^-1 and PCG with M_BD takes one step."""
    scan = _tiny(5, half_bw=0, f_knee=0.0)
    prob = O.Problem.from_scan(scan)
    blocks, hits = O.bd_blocks(prob)
    good = O.select_pixels(blocks, hits)
    prob = prob.with_pix(O.flag_samples(prob.pix, good))
    blocks, hits = O.bd_blocks(prob)
    good = O.select_pixels(blocks, hits)
    A = O.dense_A(prob)
    Abd = np.zeros_like(A)
    for p in range(prob.n_pix):
        Abd[3 * p:3 * p + 3, 3 * p:3 * p + 3] = blocks[p]
    np.testing.assert_allclose(A, Abd, atol=1e-12)
    mbd = O.bd_inverse(blocks, good)
    gi = np.repeat(good, 3)
    MA = np.zeros_like(A)
    for p in range(prob.n_pix):
        MA[3 * p:3 * p + 3] = mbd[p] @ A[3 * p:3 * p + 3]
    np.testing.assert_allclose(MA[np.ix_(gi, gi)], np.eye(gi.sum()), atol=1e-12)
    d = np.random.default_rng(5).standard_normal(scan.n_samples)
    b = O.rhs(prob, d).reshape(-1)
    x, info = O.pcg(lambda v: O.apply_A(prob, v).reshape(-1),
                    lambda v: O.bd_apply(mbd, v).reshape(-1), b, tol=1e-10)
    assert info["iters"] == 1 and info["true_rel_res"] < 1e-12


def test_bd_blocks_match_dense_diagonal_weight():
    scan = _tiny(6)
    prob = O.Problem.from_scan(scan)
    blocks, _ = O.bd_blocks(prob)
    Pm = O.dense_P(prob)
    Wd = np.diag(np.diag(O.dense_Ninv(prob)))
    D = Pm.T @ Wd @ Pm
    for p in range(prob.n_pix):
        np.testing.assert_allclose(blocks[p], D[3 * p:3 * p + 3, 3 * p:3 * p + 3], rtol=1e-12, atol=1e-12)


def test_pixel_selection_flags_degenerate_pixels():
    # a pixel seen at a single angle has a rank-1 block: it must be dropped
    pix = np.array([0, 0, 0, 0, 1, 1, 1, 1, 2], dtype=np.int64)
    psi = np.array([0.1, 0.9, 1.7, 2.5, 0.3, 0.3, 0.3, 0.3, 1.0], dtype=np.float32)
    prob = O.Problem(pix, psi, np.array([0, 9]), np.array([[1.0]]), np.array([0]), 3)
    blocks, hits = O.bd_blocks(prob)
    good = O.select_pixels(blocks, hits)
    assert good.tolist() == [True, False, False]
    assert O.flag_samples(pix, good).tolist() == [0, 0, 0, 0, -1, -1, -1, -1, -1]


# ---------------- solve ----------------

def _prepared(scan):
    prob = O.Problem.from_scan(scan)
    blocks, hits = O.bd_blocks(prob)
    good = O.select_pixels(blocks, hits)
    prob = prob.with_pix(O.flag_samples(prob.pix, good))
    blocks, hits = O.bd_blocks(prob)
    mbd = O.bd_inverse(blocks, good)
    return prob, mbd, good


def test_pcg_matches_direct_solve():
    scan = _tiny(7)
    prob, mbd, good = _prepared(scan)
    d = synth.make_tod(scan, synth.make_sky(scan.n_pix, 7), synth.make_noise(scan, 7))
    b = O.rhs(prob, d).reshape(-1)
    A = O.dense_A(prob)
    gi = np.repeat(good, 3)
    xd = np.zeros(prob.n)
    xd[gi] = np.linalg.solve(A[np.ix_(gi, gi)], b[gi])
    x, info = O.pcg(lambda v: O.apply_A(prob, v).reshape(-1),
                    lambda v: O.bd_apply(mbd, v).reshape(-1), b, tol=1e-12, max_iter=2000)
    assert info["converged"]
    np.testing.assert_allclose(x, xd, rtol=0, atol=1e-8 * np.abs(xd).max())


def test_signal_only_gives_the_sky_and_error_bound():
    """d = P s  =>  s_hat = s (Sect. 2, Eq. estimator is unbiased and exact without noise)."""
    scan = _tiny(8)
    prob, mbd, good = _prepared(scan)
    s = synth.make_sky(scan.n_pix, 8)
    s[~good] = 0.0
    d = synth.make_tod(scan, s, None)
    # flagged samples of dropped pixels carry no signal into the solve
    b = O.rhs(prob, d).reshape(-1)
    A = O.dense_A(prob)
    gi = np.repeat(good, 3)
    ev = np.linalg.eigvalsh(A[np.ix_(gi, gi)])
    kappa = ev[-1] / ev[0]
    xs = s.reshape(-1)
    errs = []

    def A_fn(v):
        return O.apply_A(prob, v).reshape(-1)

    x, info = O.pcg(A_fn, lambda v: O.bd_apply(mbd, v).reshape(-1), b, tol=1e-10, max_iter=2000)
    assert info["converged"]
    err = np.linalg.norm(x - xs) / np.linalg.norm(xs)
    # Sect. 3, Eq. errnorm with the unpreconditioned residual and kappa(A)
    assert err <= kappa * info["hist"][-1] * 1.0001
    assert err < 1e-6
    # the bound holds at every iterate as well
    for k in (1, 2, 5):
        xk, ik = O.pcg(A_fn, lambda v: O.bd_apply(mbd, v).reshape(-1), b, tol=0.0, max_iter=k)
        ek = np.linalg.norm(xk - xs) / np.linalg.norm(xs)
        errs.append(ek)
        assert ek <= kappa * ik["hist"][-1] * 1.0001


# ---------------- Arnoldi / Ritz ----------------

def _B_setup(seed=9):
    scan = _tiny(seed)
    prob, mbd, good = _prepared(scan)
    gi = np.repeat(good, 3)

    def A_fn(v):
        return O.apply_A(prob, v).reshape(-1)

    def M_fn(v):
        return O.bd_apply(mbd, v).reshape(-1)

    d = synth.make_tod(scan, synth.make_sky(scan.n_pix, seed), synth.make_noise(scan, seed))
    b = O.rhs(prob, d).reshape(-1)
    return prob, mbd, gi, A_fn, M_fn, b


def test_arnoldi_factorisation_and_orthonormality():
    prob, mbd, gi, A_fn, M_fn, b = _B_setup()
    m = 12
    W, H, mm = O.arnoldi(lambda v: M_fn(A_fn(v)), M_fn(b), m, 1e-14)
    assert mm == m and W.shape[1] == m + 1
    BW = np.stack([M_fn(A_fn(W[:, j])) for j in range(m)], axis=1)
    # Appendix A, Eq. factoriz: B W_m = W_m H_m + h_{m+1,m} w_{m+1} e_m^T = W_{m+1} H
    res = BW - W @ H
    assert np.linalg.norm(res) <= 1e-12 * np.linalg.norm(BW)
    np.testing.assert_allclose(W.T @ W, np.eye(m + 1), atol=1e-12)
    assert np.all(np.diag(H, -1) > 0)
    assert np.allclose(np.tril(H, -2), 0)


def test_ritz_residual_identity():
    prob, mbd, gi, A_fn, M_fn, b = _B_setup()
    m = 10
    W, H, mm = O.arnoldi(lambda v: M_fn(A_fn(v)), M_fn(b), m, 1e-14)
    lam, Y = np.linalg.eig(H[:m, :m])
    for i in range(m):
        if abs(lam[i].imag) > 1e-10:
            continue
        y = Y[:, i].real / np.linalg.norm(Y[:, i].real)
        v = W[:, :m] @ y
        lhs = np.linalg.norm(M_fn(A_fn(v)) - lam[i].real * v)
        # Appendix A, Eq. ritz: || B v - lambda v || = h_{m+1,m} |e_m^T y|
        assert lhs == pytest.approx(H[m, m - 1] * abs(y[-1]), rel=1e-6, abs=1e-12)


def test_ritz_values_reach_eigenvalues_of_MA():
    prob, mbd, gi, A_fn, M_fn, b = _B_setup()
    n_good = int(gi.sum())
    W, H, mm = O.arnoldi(lambda v: M_fn(A_fn(v)), M_fn(b), n_good + 2, 1e-10)
    Z, vals = O.ritz_basis(W, H, mm, mm)
    A = O.dense_A(prob)
    MA = np.zeros_like(A)
    for p in range(prob.n_pix):
        MA[3 * p:3 * p + 3] = mbd[p] @ A[3 * p:3 * p + 3]
    ev = np.sort(np.linalg.eigvals(MA[np.ix_(gi, gi)]).real)
    # the Krylov space of a random start is the whole kept space
    assert mm == n_good
    np.testing.assert_allclose(np.sort(vals), ev, rtol=1e-7, atol=1e-9)


# ---------------- two-level preconditioner ----------------

def _coarse(k=6, seed=10):
    prob, mbd, gi, A_fn, M_fn, b = _B_setup(seed)
    W, H, mm = O.arnoldi(lambda v: M_fn(A_fn(v)), M_fn(b), 20, 1e-12)
    Z, vals = O.ritz_basis(W, H, mm, k)
    AZ, E, L = O.coarse_space(A_fn, Z)
    return prob, mbd, gi, A_fn, M_fn, b, Z, AZ, E, L


def test_m2l_identities():
    prob, mbd, gi, A_fn, M_fn, b, Z, AZ, E, L = _coarse()

    def M2(v):
        return O.m2l_apply(v, M_fn, Z, AZ, L)

    # Sect. 3.2, Eq. ident: M_2l A Z = Z
    for i in range(Z.shape[1]):
        np.testing.assert_allclose(M2(A_fn(Z[:, i])), Z[:, i], atol=1e-10)
    # R A Z = 0 with R = 1 - A Z E^-1 Z^T
    Einv = np.linalg.inv(E)
    RAZ = AZ - AZ @ Einv @ (Z.T @ AZ)
    assert np.abs(RAZ).max() < 1e-10 * np.abs(AZ).max()
    # E is SPD
    assert np.linalg.eigvalsh(E)[0] > 0
    # M_2l A y = M_BD A y when Z^T A y = 0
    rng = np.random.default_rng(0)
    y = rng.standard_normal(prob.n) * np.repeat(gi, 3 // 3)
    y = y - Z @ np.linalg.solve(E, AZ.T @ y)   # A-orthogonal to range(Z)
    assert np.abs(AZ.T @ y).max() < 1e-10 * np.linalg.norm(y) * np.abs(AZ).max()
    np.testing.assert_allclose(M2(A_fn(y)), M_fn(A_fn(y)), atol=1e-9 * np.linalg.norm(y))


def test_m2l_invariant_to_basis_change():
    prob, mbd, gi, A_fn, M_fn, b, Z, AZ, E, L = _coarse()
    G = np.random.default_rng(1).standard_normal((Z.shape[1], Z.shape[1])) + 3 * np.eye(Z.shape[1])
    Z2 = Z @ G
    AZ2, E2, L2 = O.coarse_space(A_fn, Z2)
    v = np.random.default_rng(2).standard_normal(prob.n)
    np.testing.assert_allclose(O.m2l_apply(v, M_fn, Z2, AZ2, L2), O.m2l_apply(v, M_fn, Z, AZ, L),
                               rtol=1e-8, atol=1e-10)


def test_m2l_full_basis_converges_in_one_step():
    prob, mbd, gi, A_fn, M_fn, b = _B_setup(11)
    n_good = int(gi.sum())
    # an orthonormal basis of the whole kept space: M_2l = A^-1 there
    Q = np.linalg.qr(np.random.default_rng(3).standard_normal((n_good, n_good)))[0]
    Z = np.zeros((prob.n, n_good))
    Z[gi] = Q
    AZ, E, L = O.coarse_space(A_fn, Z)
    x, info = O.pcg(A_fn, lambda v: O.m2l_apply(v, M_fn, Z, AZ, L), b, tol=1e-9)
    assert info["iters"] == 1


def test_m2l_beats_bd_on_1f_noise():
    """Qualitative (Sect. 7): deflating the smallest Ritz values cuts PCG iterations."""
    scan = synth.make_scan(nx=8, ny=8, n_det=4, n_t=2048, n_int=2, half_bw=64, f_knee=2.0, seed=12)
    prob, mbd, good = _prepared(scan)

    def A_fn(v):
        return O.apply_A(prob, v).reshape(-1)

    def M_fn(v):
        return O.bd_apply(mbd, v).reshape(-1)

    d = synth.make_tod(scan, synth.make_sky(scan.n_pix, 12), synth.make_noise(scan, 12))
    b = O.rhs(prob, d).reshape(-1)
    _, ibd = O.pcg(A_fn, M_fn, b, tol=1e-8, max_iter=1000)
    W, H, mm = O.arnoldi(lambda v: M_fn(A_fn(v)), M_fn(b), 60, 1e-10)
    Z, _ = O.ritz_basis(W, H, mm, 8)
    AZ, E, L = O.coarse_space(A_fn, Z)
    _, i2l = O.pcg(A_fn, lambda v: O.m2l_apply(v, M_fn, Z, AZ, L), b, tol=1e-8, max_iter=1000)
    assert i2l["converged"] and ibd["converged"]
    assert i2l["iters"] < ibd["iters"]


# ---------------- sampled rows ----------------

def test_sampled_rows_match_full_product():
    scan = synth.make_scan(nx=8, ny=8, n_det=2, n_t=4096, n_int=4, half_bw=100, f_knee=1.0, seed=13,
                           flag_frac=0.01)
    prob = O.Problem.from_scan(scan)
    x = np.random.default_rng(13).standard_normal(prob.n)
    full = O.apply_A(prob, x)
    pix = [0, 7, 33, 63]
    np.testing.assert_allclose(O.apply_A_rows(prob, x, pix), full[pix], rtol=1e-12, atol=1e-12)


# ---------------- planted mistakes must be caught ----------------

def test_planted_sign_error_is_caught(monkeypatch):
    g, prob = _load("hand_one_pixel.json")
    real = O.mapmaking.weights

    def wrong(psi):
        w = real(psi)
        w[:, 2] *= -1.0
        return w

    monkeypatch.setattr(O.mapmaking, "weights", wrong)
    Ax = O.mapmaking.apply_A(prob, np.array(g["x"])).reshape(-1)
    assert not np.allclose(Ax, g["Ax"], atol=1e-6)


def test_planted_leaky_band_is_caught(monkeypatch):
    g, prob = _load("hand_block_edge.json")

    def leaky(y, block_off, band, block_band):
        c = np.asarray(band)[0]
        lam = c.shape[0] - 1
        kern = np.concatenate([c[::-1], c[1:]])
        return np.convolve(np.asarray(y, float), kern, mode="full")[lam:lam + len(y)]

    monkeypatch.setattr(O.mapmaking, "apply_Ninv", leaky)
    Ax = O.mapmaking.apply_A(prob, np.array(g["x"])).reshape(-1)
    assert not np.allclose(Ax, g["Ax"], atol=1e-9)


def test_planted_shifted_band_is_caught(monkeypatch):
    scan = _tiny(14)
    prob = O.Problem.from_scan(scan)
    A = O.dense_A(prob)

    def shifted(y, block_off, band, block_band):
        y = np.asarray(y, float)
        band = np.asarray(band)
        lam = band.shape[1] - 1
        z = np.empty_like(y)
        for b in range(len(block_off) - 1):
            o0, o1 = int(block_off[b]), int(block_off[b + 1])
            c = band[int(block_band[b])]
            kern = np.concatenate([c[::-1], c[1:]])
            z[o0:o1] = np.convolve(y[o0:o1], kern, mode="full")[lam + 1:lam + 1 + (o1 - o0)]
        return z

    monkeypatch.setattr(O.mapmaking, "apply_Ninv", shifted)
    x = np.random.default_rng(14).standard_normal(prob.n)
    assert not np.allclose(O.mapmaking.apply_A(prob, x).reshape(-1), A @ x, rtol=1e-6)


# ---------------- Lanczos vectors from an M_BD PCG run ----------------

def test_pcg_lanczos_relation_and_full_spectrum():
    prob, mbd, gi, A_fn, M_fn, b = _B_setup(16)
    n_good = int(gi.sum())
    m = 10
    al, be, V = O.pcg_lanczos(A_fn, M_fn, b, m)
    vals, Z, T = O.lanczos_ritz(al, be, V, m)
    # v_j are orthonormal in the M^-1 inner product: v_i^T A-free check via r = M^-1 z
    Minv = np.zeros((prob.n, prob.n))
    for p in range(prob.n_pix):
        if gi[3 * p]:
            Minv[3 * p:3 * p + 3, 3 * p:3 * p + 3] = np.linalg.inv(mbd[p])
    G = V.T @ Minv @ V
    np.testing.assert_allclose(G, np.eye(m), atol=1e-9)
    # B V_m = V_m T_m apart from the last column (the symmetric form of Eq. factoriz)
    BV = np.stack([M_fn(A_fn(V[:, j])) for j in range(m)], axis=1)
    R = BV - V @ T
    assert np.linalg.norm(R[:, :m - 1]) <= 1e-9 * np.linalg.norm(BV)
    # Ritz residual (the symmetric counterpart of Eq. ritz): for T_m s = theta s,
    # ||B V_m s - theta V_m s||_{M^-1} = |t_{m+1,m}| |e_m^T s|, t_{m+1,m} = -sqrt(beta_{m-1})/alpha_{m-1}
    al, be, V = O.pcg_lanczos(A_fn, M_fn, b, m + 1)
    _, _, T = O.lanczos_ritz(al[:m], be[:m], V[:, :m], m)
    th, S = np.linalg.eigh(T)
    t_next = np.sqrt(be[m - 1]) / al[m - 1]
    for i in (0, 1, m - 1):
        y = V[:, :m] @ S[:, i]
        res = M_fn(A_fn(y)) - th[i] * y
        lhs = np.sqrt(res @ Minv @ res)
        assert lhs == pytest.approx(t_next * abs(S[-1, i]), rel=1e-6, abs=1e-12)
    # a long run: Ritz values stay inside the spectrum of M_BD A and the extremes converge
    al, be, V = O.pcg_lanczos(A_fn, M_fn, b, n_good)
    vals, Z, T = O.lanczos_ritz(al, be, V, n_good)
    A = O.dense_A(prob)
    MA = np.zeros_like(A)
    for p in range(prob.n_pix):
        MA[3 * p:3 * p + 3] = mbd[p] @ A[3 * p:3 * p + 3]
    ev = np.sort(np.linalg.eigvals(MA[np.ix_(gi, gi)]).real)
    assert vals.min() >= ev[0] - 1e-9 and vals.max() <= ev[-1] + 1e-9
    assert abs(vals.min() - ev[0]) < 1e-9 and abs(vals.max() - ev[-1]) < 1e-9


def test_lanczos_deflation_satisfies_m2l_identity():
    prob, mbd, gi, A_fn, M_fn, b = _B_setup(17)
    al, be, V = O.pcg_lanczos(A_fn, M_fn, b, 25)
    vals, Z, T = O.lanczos_ritz(al, be, V, 6)
    AZ, E, L = O.coarse_space(A_fn, Z)
    for i in range(Z.shape[1]):
        np.testing.assert_allclose(O.m2l_apply(A_fn(Z[:, i]), M_fn, Z, AZ, L), Z[:, i], atol=1e-10)
    # the smallest Ritz pairs are accurate eigenpairs of B after 25 steps
    for i in range(2):
        y = Z[:, i]
        th = (y @ M_fn(A_fn(y))) / (y @ y)
        assert np.linalg.norm(M_fn(A_fn(y)) - th * y) < 1e-3 * np.linalg.norm(y) * abs(th) + 1e-6
