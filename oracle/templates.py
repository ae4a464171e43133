"""Template-filtered map-making of ground-based data (float64 numpy).

TEST INFRASTRUCTURE ONLY: the plain statement of the template-filtered
operator that the CUDA path computes, written from the paper; only the test
suite and the benchmark may use it.

The paper removes unwanted time-domain components whose shapes are known
but whose amplitudes are not (Sect. 2.1): for a template matrix X the
weighted filter is F_X = W - W X (X^T W X)^-1 X^T W (Eq. filtnoise), so that
F_X X = 0 (Eq. filt), and the estimator becomes
s = (P^T F P)^-1 P^T F d (Eq. unb).  For ground-based scans (Sect. 4) the
templates are piecewise low-order polynomials B over each azimuth sweep
(subscan), which take the 1/f and atmospheric drifts (Sect. 4.1, Eq.
polyfiltering), and the ground-pickup template G, one column per azimuth bin
with 1 where the sample's azimuth falls in the bin (Sect. 4.2).  With those
filters a diagonal weight W is enough, and the simulations use
piecewise-stationary white noise (Sect. 4.1); the filter actually used is
the explicitly symmetric F = F_B W^-1 F_G W^-1 F_B (Sect. 5.1).  The
polarisation solve works on the differenced timeline d^- (Sect. 5.1, Eq.
d-), whose pointing rows are (0, cos 2psi, sin 2psi).

Readings where the paper is silent (each also listed in the design notes):
  * W is diagonal with one weight w_b per stationary block (the block's c_0);
  * B holds the Legendre polynomials P_0..P_K of u = 2 (i + 1/2) / m - 1,
    i = 0..m-1 the sample index inside a subscan of m samples; every subscan
    lies inside one block; a subscan of m <= K samples takes order m - 1
    (its polynomials then span every timeline on it, and F_B removes it);
  * G has one column per azimuth bin and per block (one constant-elevation
    scan = one block); samples with bin -1 are in no column;
  * the filters act on every sample of the timeline, flagged ones included
    (they carry y_t = 0 from P and are not scattered back);
  * in the polarisation-only mode (stokes 1) the I column of P is zero; M_BD
    inverts the 2x2 (Q, U) block, I stays 0, and a pixel needs at least 2
    hits and lambda_min / lambda_max >= rcond_min of that block; in the
    intensity-only mode (stokes 2, the summed timeline d^+) the Q, U columns
    are zero, M_BD is 1 / (P^T W P)_II and a pixel needs 1 hit.

Parity unpinned: none of the functions here (pins in
tests/test_oracle_templates.py).
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import legendre

__all__ = ["TemplateProblem", "legendre_basis", "filter_poly", "filter_ground", "apply_F", "pointing_rows",
           "apply_A_T", "rhs_T", "bd_blocks_T", "select_pixels_T", "bd_inverse_T"]


class TemplateProblem:
    """Pointing, block weights and templates of one template-filtered problem."""

    def __init__(self, pix, psi, block_off, w_block, n_pix, sub_off, poly_order, az_bin, n_az_bins,
                 stokes=1):
        self.pix = np.asarray(pix, dtype=np.int64)
        self.psi = np.asarray(psi, dtype=np.float32)
        self.block_off = np.asarray(block_off, dtype=np.int64)
        self.w_block = np.asarray(w_block, dtype=np.float64)
        self.n_pix = int(n_pix)
        self.sub_off = np.asarray(sub_off, dtype=np.int64)
        self.poly_order = int(poly_order)
        self.az_bin = None if az_bin is None else np.asarray(az_bin, dtype=np.int64)
        self.n_az_bins = int(n_az_bins)
        self.stokes = int(stokes)   # 0: I, Q, U; 1: Q, U (d^-); 2: I (d^+)
        self.qu_only = self.stokes == 1

    def with_pix(self, pix):
        return TemplateProblem(pix, self.psi, self.block_off, self.w_block, self.n_pix, self.sub_off,
                               self.poly_order, self.az_bin, self.n_az_bins, self.stokes)

    def sample_weight(self) -> np.ndarray:
        """Diagonal of W: w_b on every sample of block b."""
        return np.repeat(self.w_block, np.diff(self.block_off))


def legendre_basis(m: int, order: int) -> np.ndarray:
    """Columns P_0..P_order of u = 2 (i + 1/2) / m - 1 for i = 0..m-1 (one subscan's block of B)."""
    u = (2.0 * (np.arange(m) + 0.5) / m) - 1.0
    return legendre.legvander(u, order)


def filter_poly(y, wv, sub_off, order) -> np.ndarray:
    """F_B y = W y - W B (B^T W B)^-1 B^T W y (Eq. filtnoise) with B block diagonal over subscans."""
    y = np.asarray(y, dtype=np.float64)
    out = wv * y
    if order < 0:
        return out
    for s in range(len(sub_off) - 1):
        a, b = int(sub_off[s]), int(sub_off[s + 1])
        if b <= a:
            continue
        B = legendre_basis(b - a, min(order, b - a - 1))
        w = wv[a:b]
        WB = w[:, None] * B
        coef = np.linalg.solve(B.T @ WB, WB.T @ y[a:b])
        out[a:b] -= WB @ coef
    return out


def filter_ground(y, wv, block_off, az_bin, n_bins) -> np.ndarray:
    """F_G y = W y - W G (G^T W G)^-1 G^T W y (Eq. filtnoise), G the azimuth-bin indicators of each block.

    G^T W G is diagonal (the weight in each bin), so the fit is the weighted
    mean of y over each bin of each block.
    """
    y = np.asarray(y, dtype=np.float64)
    out = wv * y
    if az_bin is None or n_bins <= 0:
        return out
    for blk in range(len(block_off) - 1):
        a, b = int(block_off[blk]), int(block_off[blk + 1])
        g = az_bin[a:b]
        ok = g >= 0
        w = wv[a:b][ok]
        num = np.bincount(g[ok], weights=w * y[a:b][ok], minlength=n_bins)
        den = np.bincount(g[ok], weights=w, minlength=n_bins)
        mean = np.divide(num, den, out=np.zeros_like(num), where=den > 0)
        seg = out[a:b]
        seg[ok] -= w * mean[g[ok]]
    return out


def apply_F(tp: TemplateProblem, y) -> np.ndarray:
    """z = F y with F = F_B W^-1 F_G W^-1 F_B (Sect. 5.1), applied right to left."""
    wv = tp.sample_weight()
    z = filter_poly(y, wv, tp.sub_off, tp.poly_order)
    z = filter_ground(z / wv, wv, tp.block_off, tp.az_bin, tp.n_az_bins)
    return filter_poly(z / wv, wv, tp.sub_off, tp.poly_order)


def pointing_rows(tp: TemplateProblem) -> np.ndarray:
    """Rows of P: (1, cos 2psi, sin 2psi); (0, cos 2psi, sin 2psi) for d^- (Sect. 5.1, Eq. d-);
    (1, 0, 0) for d^+ (Eq. d+)."""
    ang = 2.0 * tp.psi.astype(np.float64)
    first = np.zeros_like(ang) if tp.stokes == 1 else np.ones_like(ang)
    pol = 0.0 if tp.stokes == 2 else 1.0
    return np.stack([first, pol * np.cos(ang), pol * np.sin(ang)], axis=1)


def _P(tp, x):
    x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
    w = pointing_rows(tp)
    ok = tp.pix >= 0
    y = np.zeros(tp.pix.shape[0])
    y[ok] = np.einsum("ts,ts->t", w[ok], x[tp.pix[ok]])
    return y


def _Pt(tp, z):
    ok = tp.pix >= 0
    out = np.zeros((tp.n_pix, 3))
    np.add.at(out, tp.pix[ok], pointing_rows(tp)[ok] * np.asarray(z)[ok, None])
    return out


def apply_A_T(tp: TemplateProblem, x) -> np.ndarray:
    """A x = P^T F P x (Sect. 2.1, Eq. unb).  Returns [n_pix, 3]."""
    return _Pt(tp, apply_F(tp, _P(tp, x)))


def rhs_T(tp: TemplateProblem, d) -> np.ndarray:
    """b = P^T F d (Sect. 2.1, Eq. unb).  Returns [n_pix, 3]."""
    return _Pt(tp, apply_F(tp, np.asarray(d, dtype=np.float64)))


def bd_blocks_T(tp: TemplateProblem):
    """M_BD^-1 = P^T diag(W) P (Sect. 3.1, Eq. mbd) with the problem's pointing rows."""
    ok = tp.pix >= 0
    w = pointing_rows(tp)[ok]
    c0 = tp.sample_weight()[ok]
    blocks = np.zeros((tp.n_pix, 3, 3))
    np.add.at(blocks, tp.pix[ok], c0[:, None, None] * w[:, :, None] * w[:, None, :])
    hits = np.bincount(tp.pix[ok], minlength=tp.n_pix)
    return blocks, hits


def select_pixels_T(blocks, hits, stokes, rcond_min: float = 1e-3) -> np.ndarray:
    """Enough redundancy (Sect. 5): hits >= number of unknowns and a conditioned block."""
    stokes = int(stokes)
    if stokes == 2:
        return (hits >= 1) & (blocks[:, 0, 0] > 0)
    sub = blocks[:, 1:, 1:] if stokes == 1 else blocks
    ev = np.linalg.eigvalsh(sub)
    with np.errstate(divide="ignore", invalid="ignore"):
        rc = np.where(ev[:, -1] > 0, ev[:, 0] / ev[:, -1], 0.0)
    return (hits >= (2 if stokes == 1 else 3)) & (rc >= rcond_min)


def bd_inverse_T(blocks, good, stokes) -> np.ndarray:
    """M_BD: inverse of each kept block (its (Q, U) part for d^-, its I entry for d^+)."""
    inv = np.zeros_like(blocks)
    stokes = int(stokes)
    if good.any():
        if stokes == 2:
            inv[good, 0, 0] = 1.0 / blocks[good, 0, 0]
        elif stokes == 1:
            inv[good, 1:, 1:] = np.linalg.inv(blocks[good, 1:, 1:])
        else:
            inv[good] = np.linalg.inv(blocks[good])
    return inv
