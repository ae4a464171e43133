"""Oracle implementation (float64, numpy).  Test infrastructure only.

Notation follows the paper: P is the N_t x 3N_p pointing matrix, W = N^-1 the
inverse-noise weight (here a symmetric banded Toeplitz matrix per stationary
(detector, interval) block), A = P^T W P the system matrix, b = P^T W d the
right-hand side, M_BD the block-diagonal (Jacobi) preconditioner, Z the
deflation basis of Ritz vectors, E = Z^T A Z the coarse operator and M_2l the
two-level preconditioner.

Maps are arrays of shape [n_pix, 3] holding (I, Q, U) per pixel; the PCG and
Arnoldi routines work on the flattened vector of length n = 3 n_pix with
index 3p + s.

Readings where the paper is silent (each also listed in the design notes):
  * residual: PCG stops on the unpreconditioned ||b - A x_k|| / ||b|| taken
    from the recurrence; the true residual is reported at exit;
  * initial guess x_0 = 0;
  * pixel selection ("enough redundancy"): a pixel with fewer than 3 hits, or
    whose 3x3 block of M_BD^-1 has lambda_min/lambda_max < rcond_min, is
    dropped and its samples are flagged (pixel -1) before A is formed;
  * Arnoldi runs the classical Gram-Schmidt step of the algorithm twice per
    iteration (re-orthogonalisation) with the Euclidean inner product;
  * Ritz vectors: eigenpairs of H_m sorted by real part, the k smallest kept,
    a complex pair contributing its real and imaginary parts; Z is then
    orthonormalised (QR), which leaves M_2l unchanged.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "weights", "apply_P", "apply_Pt", "apply_Ninv", "apply_A", "rhs",
    "bd_blocks", "select_pixels", "flag_samples", "bd_inverse", "bd_apply",
    "pcg", "arnoldi", "ritz_basis", "coarse_space", "m2l_apply",
    "dense_P", "dense_Ninv", "dense_A", "apply_A_rows", "rhs_rows", "Problem", "pcg_lanczos", "lanczos_ritz",
]


def weights(psi: np.ndarray) -> np.ndarray:
    """Row of P for each sample: (1, cos 2psi_t, sin 2psi_t) (Sect. 2, Eq. datamodel)."""
    ang = 2.0 * np.asarray(psi, dtype=np.float64)
    return np.stack([np.ones_like(ang), np.cos(ang), np.sin(ang)], axis=1)


def apply_P(pix, psi, x) -> np.ndarray:
    """y = P x: y_t = I_p + Q_p cos 2psi_t + U_p sin 2psi_t; 0 for a flagged sample.

    Sect. 2, Eq. datamodel (three non-zeros per row of P).
    """
    pix = np.asarray(pix)
    x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
    w = weights(psi)
    ok = pix >= 0
    y = np.zeros(pix.shape[0], dtype=np.float64)
    y[ok] = np.einsum("ts,ts->t", w[ok], x[pix[ok]])
    return y


def apply_Pt(pix, psi, z, n_pix: int) -> np.ndarray:
    """m = P^T z: m_p = sum over samples t with p_t = p of z_t (1, cos 2psi_t, sin 2psi_t).

    Transpose of Sect. 2, Eq. datamodel; summed in sample order.
    """
    pix = np.asarray(pix)
    ok = pix >= 0
    w = weights(psi)[ok] * np.asarray(z, dtype=np.float64)[ok, None]
    out = np.zeros((n_pix, 3), dtype=np.float64)
    np.add.at(out, pix[ok], w)
    return out


def apply_Ninv(y, block_off, band, block_band) -> np.ndarray:
    """z = W y for a block-diagonal W of symmetric banded Toeplitz blocks.

    Within block [o_b, o_{b+1}):  z_t = sum_{|k| <= lambda, t-k in block} c_|k| y_{t-k}.
    W stands in the estimator's weight (Sect. 2, Eq. estimator; any SPD W
    gives an unbiased estimate).  The product is a full linear convolution of
    the block with the kernel (c_lambda .. c_1, c_0, c_1 .. c_lambda), of
    which the centred n_b outputs are kept.
    """
    y = np.asarray(y, dtype=np.float64)
    band = np.asarray(band, dtype=np.float64)
    lam = band.shape[1] - 1
    z = np.empty_like(y)
    for b in range(len(block_off) - 1):
        o0, o1 = int(block_off[b]), int(block_off[b + 1])
        c = band[int(block_band[b])]
        kern = np.concatenate([c[::-1], c[1:]])
        full = np.convolve(y[o0:o1], kern, mode="full")
        z[o0:o1] = full[lam:lam + (o1 - o0)]
    return z


class Problem:
    """Pointing plus noise weight of one map-making problem (read-only views)."""

    def __init__(self, pix, psi, block_off, band, block_band, n_pix):
        self.pix = np.asarray(pix, dtype=np.int64)
        self.psi = np.asarray(psi, dtype=np.float32)
        self.block_off = np.asarray(block_off, dtype=np.int64)
        self.band = np.asarray(band, dtype=np.float64)
        self.block_band = np.asarray(block_band, dtype=np.int64)
        self.n_pix = int(n_pix)

    @classmethod
    def from_scan(cls, scan):
        return cls(scan.pix, scan.psi, scan.block_off, scan.band, scan.block_band, scan.n_pix)

    def with_pix(self, pix):
        return Problem(pix, self.psi, self.block_off, self.band, self.block_band, self.n_pix)

    @property
    def n(self) -> int:
        return 3 * self.n_pix


def apply_A(prob: Problem, x) -> np.ndarray:
    """A x = P^T W P x (Sect. 3, Eq. linearsystem), matrix-free.  Returns [n_pix, 3]."""
    y = apply_P(prob.pix, prob.psi, x)
    z = apply_Ninv(y, prob.block_off, prob.band, prob.block_band)
    return apply_Pt(prob.pix, prob.psi, z, prob.n_pix)


def rhs(prob: Problem, d) -> np.ndarray:
    """b = P^T W d (Sect. 3, Eq. linearsystem).  Returns [n_pix, 3]."""
    z = apply_Ninv(np.asarray(d, dtype=np.float64), prob.block_off, prob.band, prob.block_band)
    return apply_Pt(prob.pix, prob.psi, z, prob.n_pix)


def bd_blocks(prob: Problem):
    """M_BD^-1 = P^T diag(W) P (Sect. 3.1, Eq. mbd): one 3x3 block per pixel.

    diag(W) of a Toeplitz block is its c_0.  Returns (blocks [n_pix,3,3], hits [n_pix]).
    """
    c0 = np.empty(prob.pix.shape[0])
    for b in range(len(prob.block_off) - 1):
        c0[prob.block_off[b]:prob.block_off[b + 1]] = prob.band[prob.block_band[b], 0]
    ok = prob.pix >= 0
    w = weights(prob.psi)[ok]
    outer = c0[ok, None, None] * w[:, :, None] * w[:, None, :]
    blocks = np.zeros((prob.n_pix, 3, 3))
    np.add.at(blocks, prob.pix[ok], outer)
    hits = np.bincount(prob.pix[ok], minlength=prob.n_pix)
    return blocks, hits


def select_pixels(blocks, hits, rcond_min: float = 1e-3) -> np.ndarray:
    """Pixels kept in the solve: at least 3 hits and lambda_min/lambda_max >= rcond_min.

    The paper drops samples of pixels without enough redundancy (Sect. 5);
    this threshold is the reading used throughout.
    """
    ev = np.linalg.eigvalsh(blocks)
    with np.errstate(divide="ignore", invalid="ignore"):
        rc = np.where(ev[:, 2] > 0, ev[:, 0] / ev[:, 2], 0.0)
    return (hits >= 3) & (rc >= rcond_min)


def flag_samples(pix, good) -> np.ndarray:
    """Samples of dropped pixels become flagged (-1), so they leave P entirely."""
    pix = np.array(pix, dtype=np.int64, copy=True)
    ok = pix >= 0
    bad = np.zeros_like(ok)
    bad[ok] = ~good[pix[ok]]
    pix[bad] = -1
    return pix


def bd_inverse(blocks, good) -> np.ndarray:
    """M_BD: the inverse of each kept 3x3 block; zero blocks for dropped pixels."""
    inv = np.zeros_like(blocks)
    if good.any():
        inv[good] = np.linalg.inv(blocks[good])
    return inv


def bd_apply(m_bd, r) -> np.ndarray:
    """z = M_BD r: per-pixel 3x3 matrix-vector product.  r, z are [n_pix, 3]."""
    return np.einsum("pij,pj->pi", m_bd, np.asarray(r).reshape(-1, 3))


def pcg(apply_A_fn, apply_M_fn, b, tol: float = 1e-8, max_iter: int = 500):
    """Preconditioned conjugate gradients (Sect. 3, Eq. pcg), x_0 = 0.

    Operators take and return flat vectors of length n.  Stops when the
    recurrence residual ||r_k|| / ||b|| <= tol or after max_iter products
    with A.  Returns (x, info) with iterations, the residual history and the
    true residual ||b - A x|| / ||b|| at exit.
    """
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    bn = np.linalg.norm(b)
    x = np.zeros_like(b)
    hist = [1.0]
    if bn == 0.0:
        return x, dict(iters=0, hist=hist, true_rel_res=0.0, converged=True)
    r = b.copy()
    z = apply_M_fn(r)
    p = z.copy()
    rz = float(r @ z)
    it = 0
    converged = False
    while it < max_iter:
        q = apply_A_fn(p)
        alpha = rz / float(p @ q)
        x += alpha * p
        r -= alpha * q
        it += 1
        hist.append(float(np.linalg.norm(r) / bn))
        if hist[-1] <= tol:
            converged = True
            break
        z = apply_M_fn(r)
        rz_new = float(r @ z)
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
    true = float(np.linalg.norm(b - apply_A_fn(x)) / bn)
    return x, dict(iters=it, hist=hist, true_rel_res=true, converged=converged)


def pcg_lanczos(apply_A_fn, apply_M_fn, b, m: int):
    """m steps of PCG (x_0 = 0) recording alpha_j, beta_j and v_j = z_j / sqrt(r_j^T z_j).

    Same recurrences as ``pcg``; the recorded quantities are the Lanczos
    description of B = M A that PCG builds as a by-product (used for the
    deflation basis instead of a separate Arnoldi run).
    """
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    r = b.copy()
    z = apply_M_fn(r)
    p = z.copy()
    rz = float(r @ z)
    alphas, betas, V = [], [], []
    for _ in range(m):
        V.append(z / np.sqrt(rz))
        q = apply_A_fn(p)
        alpha = rz / float(p @ q)
        r = r - alpha * q
        z = apply_M_fn(r)
        rz_new = float(r @ z)
        beta = rz_new / rz
        alphas.append(alpha)
        betas.append(beta)
        rz = rz_new
        p = z + beta * p
    return np.array(alphas), np.array(betas), np.stack(V, axis=1)


def lanczos_ritz(alphas, betas, V, k: int):
    """Ritz pairs of B = M A from the PCG coefficients.

    T_m has diagonal 1/alpha_j + beta_{j-1}/alpha_{j-1} and off-diagonal
    -sqrt(beta_j)/alpha_j; B V_m = V_m T_m + (a multiple of v_{m+1} e_m^T), the
    symmetric counterpart of Eq. factoriz (Appendix A).  Returns the k
    smallest Ritz values and the orthonormalised Ritz vectors V_m S.
    """
    m = len(alphas)
    T = np.zeros((m, m))
    for j in range(m):
        T[j, j] = 1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0)
        if j + 1 < m:
            T[j, j + 1] = T[j + 1, j] = -np.sqrt(betas[j]) / alphas[j]
    lam, S = np.linalg.eigh(T)
    Z = V[:, :m] @ S[:, :k]
    Q, _ = np.linalg.qr(Z)
    return lam[:k], Q, T


def arnoldi(apply_B_fn, r0, m_max: int, tol: float):
    """Arnoldi process on B (Appendix A, Algorithm arnoldi).

    w_1 = r_0 / ||r_0||; for j = 1..m: v = B w_j, h_ij = (v, w_i) for i <= j,
    v -= sum_i h_ij w_i (done twice, the second pass re-orthogonalising and
    adding to h), h_{j+1,j} = ||v||; stop when h_{j+1,j} <= tol, else
    w_{j+1} = v / h_{j+1,j}.  Returns (W [n, m+1 or m], H [(m+1), m], m)
    with the m-step factorisation B W_m = W_m H_m + h_{m+1,m} w_{m+1} e_m^T
    (Eq. factoriz); when the loop breaks, W has m columns.
    """
    r0 = np.asarray(r0, dtype=np.float64).reshape(-1)
    n = r0.shape[0]
    W = np.zeros((n, m_max + 1))
    H = np.zeros((m_max + 1, m_max))
    W[:, 0] = r0 / np.linalg.norm(r0)
    m = m_max
    broke = False
    for j in range(m_max):
        v = apply_B_fn(W[:, j])
        for _ in range(2):
            h = W[:, :j + 1].T @ v
            v = v - W[:, :j + 1] @ h
            H[:j + 1, j] += h
        H[j + 1, j] = np.linalg.norm(v)
        if H[j + 1, j] <= tol:
            m = j + 1
            broke = True
            break
        W[:, j + 1] = v / H[j + 1, j]
    if broke:
        return W[:, :m], H[:m + 1, :m], m
    return W[:, :m + 1], H[:m + 1, :m], m


def ritz_basis(W, H, m: int, k: int):
    """Deflation basis from Ritz pairs of H_m (Appendix A, Eq. ritz; Sect. 6).

    H_m y = lambda y; Ritz vectors v = W_m y.  The k pairs of smallest real
    part are kept; a complex conjugate pair adds the real and imaginary parts
    of one vector.  Returns (Z [n, k'] orthonormal, ritz values kept).
    """
    Hm = H[:m, :m]
    lam, Y = np.linalg.eig(Hm)
    order = np.argsort(lam.real, kind="stable")
    cols, vals = [], []
    used = np.zeros(m, dtype=bool)
    for i in order:
        if len(cols) >= k:
            break
        if used[i]:
            continue
        used[i] = True
        if abs(lam[i].imag) > 0:
            # mark the conjugate partner as used
            j = int(np.argmin(np.abs(lam - np.conj(lam[i])) + used * 1e300))
            used[j] = True
            cols.append(Y[:, i].real)
            vals.append(lam[i].real)
            if len(cols) < k:
                cols.append(Y[:, i].imag)
                vals.append(lam[i].real)
        else:
            cols.append(Y[:, i].real)
            vals.append(lam[i].real)
    Ysel = np.stack(cols, axis=1)
    Z = W[:, :m] @ Ysel
    Q, _ = np.linalg.qr(Z)
    return Q, np.array(vals)


def coarse_space(apply_A_fn, Z):
    """AZ, the coarse operator E = Z^T A Z (Sect. 3.2, Eq. m2l) and its Cholesky factor."""
    AZ = np.stack([apply_A_fn(Z[:, i]) for i in range(Z.shape[1])], axis=1)
    E = Z.T @ AZ
    E = 0.5 * (E + E.T)
    L = np.linalg.cholesky(E)
    return AZ, E, L


def m2l_apply(v, apply_Mbd_fn, Z, AZ, L):
    """M_2l v = M_BD (v - A Z E^-1 Z^T v) + Z E^-1 Z^T v (Sect. 3.2, Eq. m2l)."""
    v = np.asarray(v, dtype=np.float64).reshape(-1)
    t = Z.T @ v
    u = np.linalg.solve(L.T, np.linalg.solve(L, t))
    return apply_Mbd_fn(v - AZ @ u) + Z @ u


# -------- dense assembly for tiny problems --------

def dense_P(prob: Problem) -> np.ndarray:
    """The N_t x 3N_p pointing matrix as a dense array (Sect. 2, Eq. datamodel)."""
    N = prob.pix.shape[0]
    Pm = np.zeros((N, prob.n))
    w = weights(prob.psi)
    for t in range(N):
        p = int(prob.pix[t])
        if p >= 0:
            Pm[t, 3 * p:3 * p + 3] = w[t]
    return Pm


def dense_Ninv(prob: Problem) -> np.ndarray:
    """W as a dense N_t x N_t block-diagonal matrix of Toeplitz sections."""
    N = prob.pix.shape[0]
    Wm = np.zeros((N, N))
    lam = prob.band.shape[1] - 1
    for b in range(len(prob.block_off) - 1):
        o0, o1 = int(prob.block_off[b]), int(prob.block_off[b + 1])
        c = prob.band[prob.block_band[b]]
        for i in range(o0, o1):
            for j in range(max(o0, i - lam), min(o1, i + lam + 1)):
                Wm[i, j] = c[abs(i - j)]
    return Wm


def dense_A(prob: Problem) -> np.ndarray:
    """A = P^T W P assembled densely (Sect. 3, Eq. linearsystem)."""
    Pm = dense_P(prob)
    return Pm.T @ dense_Ninv(prob) @ Pm


# -------- sampled rows for full-size checks --------

def _rows_of_W(prob: Problem, y, pixels) -> np.ndarray:
    """sum_{t: p_t = p} w_t (W y)_t for the listed pixels, W y evaluated only where needed."""
    lam = prob.band.shape[1] - 1
    out = np.zeros((len(pixels), 3))
    for i, p in enumerate(pixels):
        ts = np.nonzero(prob.pix == p)[0]
        if ts.size == 0:
            continue
        bs = np.searchsorted(prob.block_off, ts, side="right") - 1
        w = weights(prob.psi[ts])
        for t, b, wt in zip(ts, bs, w):
            o0, o1 = int(prob.block_off[b]), int(prob.block_off[b + 1])
            j0, j1 = max(o0, t - lam), min(o1, t + lam + 1)
            c = prob.band[prob.block_band[b]]
            zt = float(c[np.abs(np.arange(j0, j1) - t)] @ y[j0:j1])
            out[i] += zt * wt
    return out


def apply_A_rows(prob: Problem, x, pixels) -> np.ndarray:
    """Rows (A x)_p for the listed pixels only, by the definition.

    (A x)_p = sum_{t: p_t = p} w_t z_t with z_t = sum_{|k|<=lambda, t-k in block} c_|k| y_{t-k}
    and y = P x.  Returns [len(pixels), 3].
    """
    return _rows_of_W(prob, apply_P(prob.pix, prob.psi, x), pixels)


def rhs_rows(prob: Problem, d, pixels) -> np.ndarray:
    """Rows b_p of b = P^T W d for the listed pixels only.  Returns [len(pixels), 3]."""
    return _rows_of_W(prob, np.asarray(d, dtype=np.float64), pixels)
