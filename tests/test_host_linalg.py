"""Host linear algebra of the coarse-space build (CPU): the Ritz values of the Arnoldi Hessenberg
matrix H_m and of the Lanczos tridiagonal matrix (Appendix A, Eq. ritz) and their eigenvectors,
against numpy's LAPACK eigen-solvers and the eigen-equation itself; the Cholesky factor of
E = Z^T A Z and its inverse (Sect. 3.2), and the triangular inverse that orthonormalises Z.

The library's host source is compiled here with g++ together with a small extern "C" shim, so no
GPU is needed.
"""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1801_08937_gb300", "csrc")

SHIM = r"""
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <string>
#include <thread>
#include <vector>
#include "common.cuh"
namespace mm {
std::mutex& smem_config_mutex() {
    static std::mutex m;
    return m;
}
}  // namespace mm
extern "C" int t_tri_eigvals(const double* d, const double* e, int n, double* w) {
    std::vector<double> dd(d, d + n), ee(e, e + (n > 1 ? n - 1 : 0)), ww;
    if (!mm::host_tridiag_eigvals(dd, ee, n, ww)) return 0;
    for (int i = 0; i < n; ++i) w[i] = ww[i];
    return 1;
}
extern "C" int t_tri_eigvec(const double* d, const double* e, int n, double lam, double* v) {
    std::vector<double> dd(d, d + n), ee(e, e + (n > 1 ? n - 1 : 0)), vv;
    if (!mm::host_tridiag_eigvec(dd, ee, n, lam, vv)) return 0;
    for (int i = 0; i < n; ++i) v[i] = vv[i];
    return 1;
}
extern "C" int t_ritz(const double* H, const double* d, const double* e, int m, int k, int kmax, double eps,
                      double* C, double* vals, int* ksel) {
    std::vector<double> c, v;
    int rs;
    if (H) {
        std::vector<double> h(H, H + (size_t)m * m);
        rs = mm::host_ritz_hess(h, m, k, kmax, eps, c, v);
    } else {
        std::vector<double> dd(d, d + m), ee(e, e + (m > 1 ? m - 1 : 1));
        rs = mm::host_ritz_tridiag(dd, ee, m, k, kmax, eps, c, v);
    }
    *ksel = (int)v.size();
    if (rs == 0) {
        for (size_t i = 0; i < c.size(); ++i) C[i] = c[i];
        for (size_t i = 0; i < v.size(); ++i) vals[i] = v[i];
    }
    return rs;
}
extern "C" int t_layout(const int64_t* bo, int nb, const int64_t* so, int ns, int order, int32_t* blk_sub,
                        double* ginv, char* err) {
    std::vector<int64_t> b(bo, bo + nb + 1), s(so, so + ns + 1);
    std::vector<int32_t> bs;
    std::vector<double> g;
    std::string e;
    if (!mm::host_template_layout(b, s, order, bs, g, e)) {
        std::strncpy(err, e.c_str(), 255);
        return 0;
    }
    for (size_t i = 0; i < bs.size(); ++i) blk_sub[i] = bs[i];
    for (size_t i = 0; i < g.size(); ++i) ginv[i] = g[i];
    return 1;
}
extern "C" void t_lanczos(const double* al, const double* be, int m, double* d, double* e) {
    std::vector<double> a(al, al + m), b(be, be + m), dd, ee;
    mm::host_lanczos_tridiag(a, b, m, dd, ee);
    for (int i = 0; i < m; ++i) d[i] = dd[i];
    for (int i = 0; i + 1 < m; ++i) e[i] = ee[i];
}
// raise_smem_once from 8 threads with sizes in 1..4000 in a scattered order: the configuration
// calls must come in increasing order (never lowering) and end at the largest size asked for
extern "C" int t_raise_smem(long long* last, int* calls, long long* largest) {
    std::atomic<size_t> configured{0};
    std::vector<size_t> seen;
    std::vector<std::thread> th;
    for (int t = 0; t < 8; ++t)
        th.emplace_back([&, t] {
            for (int i = 0; i < 500; ++i) {
                const size_t sm = 1 + (size_t)((i * 8 + t) * 2654435761u % 4000u);
                mm::raise_smem_once(configured, sm, [&](size_t v) { seen.push_back(v); });
            }
        });
    for (auto& x : th) x.join();
    size_t mx = 0;
    for (int t = 0; t < 8; ++t)
        for (int i = 0; i < 500; ++i) mx = std::max(mx, 1 + (size_t)((i * 8 + t) * 2654435761u % 4000u));
    *largest = (long long)mx;
    for (size_t i = 1; i < seen.size(); ++i)
        if (seen[i] <= seen[i - 1]) return 0;
    *last = (long long)configured.load();
    *calls = (int)seen.size();
    return seen.empty() ? 0 : (seen.back() == configured.load() ? 1 : 0);
}
extern "C" int t_chol_inv(const double* A, int n, double* L, double* inv) {
    std::vector<double> a(A, A + (size_t)n * n), v;
    if (!mm::host_cholesky(a, n)) return 0;
    mm::host_spd_inverse_from_chol(a, n, v);
    for (size_t i = 0; i < (size_t)n * n; ++i) { L[i] = a[i]; inv[i] = v[i]; }
    return 1;
}
extern "C" int t_pivoted_inv(const double* A, int n, double tol, double* inv) {
    std::vector<double> a(A, A + (size_t)n * n), v;
    const int r = mm::host_pivoted_spd_inverse(a, n, tol, v);
    for (size_t i = 0; i < (size_t)n * n; ++i) inv[i] = v[i];
    return r;
}
extern "C" void t_upper_inv(const double* R, int n, double* Ri) {
    std::vector<double> r(R, R + (size_t)n * n), v;
    mm::host_upper_inverse(r, n, v);
    for (size_t i = 0; i < (size_t)n * n; ++i) Ri[i] = v[i];
}
extern "C" int t_eigvals(const double* H, int m, double* wr, double* wi) {
    std::vector<double> h(H, H + (size_t)m * m), r, i;
    if (!mm::host_hess_eigvals(h, m, r, i)) return 0;
    for (int j = 0; j < m; ++j) { wr[j] = r[j]; wi[j] = i[j]; }
    return 1;
}
extern "C" int t_eigvec(const double* H, int m, double wr, double wi, double* vr, double* vi) {
    std::vector<double> h(H, H + (size_t)m * m), r, i;
    if (!mm::host_hess_eigvec(h, m, wr, wi, r, i)) return 0;
    for (int j = 0; j < m; ++j) { vr[j] = r[j]; vi[j] = i[j]; }
    return 1;
}
"""


def _cuda_include():
    for nvcc in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if nvcc and os.path.exists(nvcc):
            inc = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "include")
            if os.path.exists(os.path.join(inc, "cuda_runtime.h")):
                return inc
    return None


@pytest.fixture(scope="module")
def eig(tmp_path_factory):
    inc = _cuda_include()
    if inc is None or shutil.which("g++") is None:
        pytest.skip("g++ or the CUDA headers are missing")
    d = tmp_path_factory.mktemp("host_linalg")
    shim = d / "shim.cpp"
    shim.write_text(SHIM)
    so = d / "libhostlinalg.so"
    subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread", "-I", inc, "-I", CSRC, "-x", "c++",
                    os.path.join(CSRC, "host_linalg.cpp"), "-x", "none", str(shim), "-o", str(so)], check=True)
    lib = C.CDLL(str(so))
    P = C.POINTER(C.c_double)
    lib.t_eigvals.argtypes = [P, C.c_int, P, P]
    lib.t_eigvec.argtypes = [P, C.c_int, C.c_double, C.c_double, P, P]
    lib.t_chol_inv.argtypes = [P, C.c_int, P, P]
    lib.t_tri_eigvals.argtypes = [P, P, C.c_int, P]
    lib.t_tri_eigvec.argtypes = [P, P, C.c_int, C.c_double, P]
    I64 = C.POINTER(C.c_int64)
    lib.t_layout.argtypes = [I64, C.c_int, I64, C.c_int, C.c_int, C.POINTER(C.c_int32), P, C.c_char_p]
    lib.t_lanczos.argtypes = [P, P, C.c_int, P, P]
    lib.t_raise_smem.argtypes = [C.POINTER(C.c_longlong), C.POINTER(C.c_int), C.POINTER(C.c_longlong)]
    lib.t_ritz.argtypes = [P, P, P, C.c_int, C.c_int, C.c_int, C.c_double, P, P, C.POINTER(C.c_int)]
    lib.t_upper_inv.argtypes = [P, C.c_int, P]
    lib.t_pivoted_inv.argtypes = [P, C.c_int, C.c_double, P]

    def p(a):
        return a.ctypes.data_as(P)

    def vals(H):
        H = np.ascontiguousarray(H, dtype=np.float64)
        m = H.shape[0]
        wr, wi = np.zeros(m), np.zeros(m)
        assert lib.t_eigvals(p(H), m, p(wr), p(wi)) == 1
        return wr + 1j * wi

    def vec(H, lam):
        H = np.ascontiguousarray(H, dtype=np.float64)
        m = H.shape[0]
        vr, vi = np.zeros(m), np.zeros(m)
        assert lib.t_eigvec(p(H), m, lam.real, lam.imag, p(vr), p(vi)) == 1
        return vr + 1j * vi

    def chol_inv(A):
        A = np.ascontiguousarray(A, dtype=np.float64)
        n = A.shape[0]
        L, inv = np.zeros((n, n)), np.zeros((n, n))
        ok = lib.t_chol_inv(p(A), n, p(L), p(inv))
        return (L, inv) if ok == 1 else None

    def pivoted_inv(A, tol):
        A = np.ascontiguousarray(A, dtype=np.float64)
        inv = np.zeros_like(A)
        r = lib.t_pivoted_inv(p(A), A.shape[0], float(tol), p(inv))
        return r, inv

    def upper_inv(R):
        R = np.ascontiguousarray(R, dtype=np.float64)
        Ri = np.zeros_like(R)
        lib.t_upper_inv(p(R), R.shape[0], p(Ri))
        return Ri

    def tri(d, e):
        d = np.ascontiguousarray(d, dtype=np.float64)
        e = np.ascontiguousarray(e if len(e) else np.zeros(1), dtype=np.float64)
        w = np.zeros(len(d))
        assert lib.t_tri_eigvals(p(d), p(e), len(d), p(w)) == 1
        return w

    def tri_vec(d, e, lam):
        d = np.ascontiguousarray(d, dtype=np.float64)
        e = np.ascontiguousarray(e if len(e) else np.zeros(1), dtype=np.float64)
        v = np.zeros(len(d))
        assert lib.t_tri_eigvec(p(d), p(e), len(d), float(lam), p(v)) == 1
        return v

    def ritz(H=None, d=None, e=None, k=0, eps=0.0, kmax=512):
        m = H.shape[0] if H is not None else len(d)
        Cm, v, ks = np.zeros(m * m), np.zeros(m), C.c_int(0)
        args = [p(np.ascontiguousarray(H, dtype=np.float64)) if H is not None else None,
                p(np.ascontiguousarray(d, dtype=np.float64)) if d is not None else None,
                p(np.ascontiguousarray(e if len(e) else np.zeros(1), dtype=np.float64)) if e is not None else None]
        rs = lib.t_ritz(*args, m, k, kmax, eps, p(Cm), p(v), C.byref(ks))
        if rs != 0:
            return rs, None, None
        return 0, Cm[:m * ks.value].reshape(m, ks.value), v[:ks.value]

    def layout(block_off, so, order):
        bo = np.ascontiguousarray(block_off, dtype=np.int64)
        sv = np.ascontiguousarray(so, dtype=np.int64)
        bs = np.zeros(len(bo), np.int32)
        g = np.zeros(16 * (len(sv) - 1))
        err = C.create_string_buffer(256)
        ok = lib.t_layout(bo.ctypes.data_as(I64), len(bo) - 1, sv.ctypes.data_as(I64), len(sv) - 1, order,
                          bs.ctypes.data_as(C.POINTER(C.c_int32)), p(g), err)
        if not ok:
            return err.value.decode()
        return bs, g.reshape(-1, 4, 4)

    def lanczos(al, be):
        al = np.ascontiguousarray(al, dtype=np.float64)
        be = np.ascontiguousarray(be, dtype=np.float64)
        m = len(al)
        d, e = np.zeros(m), np.zeros(max(1, m - 1))
        lib.t_lanczos(p(al), p(be), m, p(d), p(e))
        return d, e[:m - 1]

    def raise_smem():
        last, calls, largest = C.c_longlong(0), C.c_int(0), C.c_longlong(0)
        ok = lib.t_raise_smem(C.byref(last), C.byref(calls), C.byref(largest))
        return ok, last.value, calls.value, largest.value

    vals.chol_inv = chol_inv
    vals.raise_smem = raise_smem
    vals.lanczos = lanczos
    vals.layout = layout
    vals.ritz = ritz
    vals.tri = tri
    vals.tri_vec = tri_vec
    vals.upper_inv = upper_inv
    vals.pivoted_inv = pivoted_inv
    return vals, vec


def _arnoldi(B, m, seed):
    n = B.shape[0]
    rng = np.random.default_rng(seed)
    W = np.zeros((n, m + 1))
    H = np.zeros((m + 1, m))
    w = rng.standard_normal(n)
    W[:, 0] = w / np.linalg.norm(w)
    for j in range(m):
        v = B @ W[:, j]
        for _ in range(2):
            h = W[:, :j + 1].T @ v
            v -= W[:, :j + 1] @ h
            H[:j + 1, j] += h
        H[j + 1, j] = np.linalg.norm(v)
        W[:, j + 1] = v / H[j + 1, j]
    return H[:m, :m]


def _match(a, b):
    """Largest distance from each value of a to the nearest unused value of b."""
    b = list(b)
    worst = 0.0
    for x in sorted(a, key=lambda z: (z.real, z.imag)):
        i = int(np.argmin([abs(x - y) for y in b]))
        worst = max(worst, abs(x - b.pop(i)))
    return worst


def test_ritz_values_of_a_preconditioned_spd_operator(eig):
    """H_m of Arnoldi on B = D A (D, A SPD, so B is similar to an SPD matrix): the eigenvalues equal
    LAPACK's, are real and positive, and the smallest ones' eigenvectors satisfy H v = lambda v."""
    vals, vec = eig
    rng = np.random.default_rng(0)
    n, m = 400, 150
    Q = np.linalg.qr(rng.standard_normal((n, n)))[0]
    ev = np.concatenate([np.geomspace(1e-4, 0.3, 40), 1.0 + 0.5 * rng.random(n - 40)])
    A = (Q * ev) @ Q.T
    B = (0.5 + rng.random(n))[:, None] * A
    H = _arnoldi(B, m, 1)
    lam = vals(H)
    ref = np.linalg.eigvals(H)
    hn = np.abs(H).max()
    assert _match(lam, ref) <= 1e-12 * hn
    assert np.abs(lam.imag).max() <= 1e-6 * hn and lam.real.min() > 0
    for x in sorted(lam, key=lambda z: z.real)[:12]:
        v = vec(H, x)
        assert abs(np.linalg.norm(v) - 1.0) < 1e-12
        assert np.linalg.norm(H @ v - x * v) <= 1e-11 * hn


def test_complex_pairs_of_a_random_hessenberg_matrix(eig):
    """A random upper Hessenberg matrix has complex conjugate pairs: values match LAPACK, pairs come out
    exactly conjugate, and the complex eigenvectors satisfy the eigen-equation."""
    vals, vec = eig
    rng = np.random.default_rng(2)
    m = 60
    H = np.triu(rng.standard_normal((m, m)), -1)
    lam = vals(H)
    ref = np.linalg.eigvals(H)
    hn = np.abs(H).max()
    assert _match(lam, ref) <= 1e-10 * hn
    cplx = lam[lam.imag != 0]
    assert len(cplx) >= 4
    assert _match(cplx, np.conj(cplx)) == 0.0
    for x in cplx[:6]:
        v = vec(H, x)
        assert np.linalg.norm(H @ v - x * v) <= 1e-10 * hn * max(1.0, abs(x))


def test_symmetric_tridiagonal_lanczos_matrix(eig):
    """The Lanczos matrix T (symmetric tridiagonal, positive definite): real values equal eigvalsh."""
    vals, vec = eig
    rng = np.random.default_rng(3)
    m = 80
    d = 1.0 + rng.random(m)
    e = 0.4 * rng.random(m - 1)
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    lam = vals(T)
    assert np.abs(lam.imag).max() == 0.0
    np.testing.assert_allclose(np.sort(lam.real), np.linalg.eigvalsh(T), atol=1e-13)
    lo = np.sort(lam.real)[0]
    v = vec(T, lo + 0j)
    assert np.linalg.norm(T @ v - lo * v) <= 1e-12


@pytest.mark.parametrize("case", ["one", "rotation", "triangular", "zero", "identity", "jordan"])
def test_degenerate_matrices(eig, case):
    vals, vec = eig
    if case == "one":
        H, ref = np.array([[2.5]]), [2.5]
    elif case == "rotation":
        H, ref = np.array([[0.0, 1.0], [-1.0, 0.0]]), [1j, -1j]
    elif case == "triangular":
        H = np.triu(np.arange(1.0, 17.0).reshape(4, 4))
        ref = np.diag(H)
    elif case == "zero":
        H, ref = np.zeros((5, 5)), np.zeros(5)
    elif case == "identity":
        H, ref = np.eye(6), np.ones(6)
    else:   # a 3x3 Jordan block: one defective eigenvalue
        H, ref = np.eye(3) * 2.0 + np.diag([1.0, 1.0], 1), [2.0, 2.0, 2.0]
    lam = vals(H)
    assert _match(lam, np.asarray(ref, dtype=complex)) <= (1e-5 if case == "jordan" else 1e-14)
    if case != "zero":
        x = lam[0]
        v = vec(H, x)
        assert abs(np.linalg.norm(v) - 1.0) < 1e-12
        assert np.linalg.norm(H @ v - x * v) <= 1e-8 * max(1.0, np.abs(H).max())


@pytest.mark.parametrize("n", [1, 7, 96])
def test_cholesky_and_spd_inverse(eig, n):
    """E = L L^T with L lower triangular (LAPACK's factor), E^-1 equal to numpy's inverse; a matrix
    that is not positive definite is refused."""
    vals, _ = eig
    rng = np.random.default_rng(n)
    B = rng.standard_normal((n, n))
    E = B @ B.T + n * np.eye(n)
    L, inv = vals.chol_inv(E)
    np.testing.assert_allclose(np.triu(L, 1), 0.0)
    np.testing.assert_allclose(L, np.linalg.cholesky(E), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(inv, np.linalg.inv(E), rtol=1e-10, atol=1e-13)
    np.testing.assert_allclose(inv, inv.T, rtol=0, atol=0)
    if n > 1:
        E[0, 0] = -1.0
        assert vals.chol_inv(E) is None


@pytest.mark.parametrize("n,visible", [(6, 6), (12, 7), (32, 20)])
def test_pivoted_inverse_of_a_semidefinite_coarse_operator(eig, n, visible):
    """E = Z^T A Z where A sees only part of the map (a prefix of a scan): `visible` directions of
    span Z lie where A is positive definite, the others where A is zero, mixed over all columns.
    The kept index set S has that size, inv equals (E_SS)^-1 on S and 0 elsewhere, and the coarse
    correction Z inv Z^T acts on the range of A like the pseudo-inverse one (Sect. 3.2)."""
    vals, _ = eig
    rng = np.random.default_rng(n + visible)
    N, rank = 3 * n, visible + 4
    Q, _ = np.linalg.qr(rng.standard_normal((N, N)))
    A = Q[:, :rank] @ np.diag(rng.uniform(0.5, 2.0, rank)) @ Q[:, :rank].T
    parts = [Q[:, :rank] @ rng.standard_normal((rank, visible)), Q[:, rank:rank + n - visible]]
    Z, _ = np.linalg.qr(np.hstack(parts) @ np.linalg.qr(rng.standard_normal((n, n)))[0])
    E = Z.T @ A @ Z
    E = 0.5 * (E + E.T)
    r, inv = vals.pivoted_inv(E, 1e-10)
    assert r == visible
    S = np.where(np.abs(inv).sum(axis=1) > 0)[0]
    assert len(S) == r
    np.testing.assert_allclose(inv[np.ix_(S, S)], np.linalg.inv(E[np.ix_(S, S)]), rtol=1e-9, atol=1e-12)
    P = Z @ inv @ Z.T
    P_ref = Z @ np.linalg.pinv(E, rcond=1e-9) @ Z.T
    np.testing.assert_allclose(A @ P @ A, A @ P_ref @ A, atol=1e-9 * np.abs(A).max())
    if r == n:
        np.testing.assert_allclose(inv, np.linalg.inv(E), rtol=1e-9, atol=1e-12)
    assert vals.pivoted_inv(np.zeros((4, 4)), 1e-10)[0] == 0


@pytest.mark.parametrize("n", [1, 5, 80])
def test_upper_triangular_inverse(eig, n):
    vals, _ = eig
    rng = np.random.default_rng(10 + n)
    R = np.triu(rng.standard_normal((n, n))) + 3.0 * np.eye(n)
    Ri = vals.upper_inv(R)
    np.testing.assert_allclose(np.tril(Ri, -1), 0.0)
    np.testing.assert_allclose(R @ Ri, np.eye(n), atol=1e-12)


def _tridiag(d, e):
    return np.diag(d) + np.diag(e, 1) + np.diag(e, -1)


@pytest.mark.parametrize("case", ["lanczos", "large", "diagonal", "wilkinson", "split", "tiny_offdiag", "one",
                                  "two"])
def test_symmetric_tridiagonal_solver(eig, case):
    """The dedicated solver of the Lanczos matrix: values equal LAPACK's eigvalsh to round-off of ||T||,
    eigenvectors satisfy T v = lambda v and are orthogonal for separated values."""
    vals, _ = eig
    rng = np.random.default_rng(sum(map(ord, case)))
    if case == "lanczos":       # the Lanczos matrix of a PCG run: 1/alpha_j + beta_{j-1}/alpha_{j-1}, -sqrt(beta_j)/alpha_j
        al = 0.5 + rng.random(120)
        be = 0.8 * rng.random(119)
        d = 1.0 / al + np.concatenate([[0.0], be / al[:-1]])
        e = -np.sqrt(be) / al[:-1]
    elif case == "large":
        d, e = rng.standard_normal(700), rng.standard_normal(699)
    elif case == "diagonal":
        d, e = rng.standard_normal(9), np.zeros(8)
    elif case == "wilkinson":   # W21+: pairs of nearly equal eigenvalues
        d, e = np.abs(np.arange(-10.0, 11.0)), np.ones(20)
    elif case == "split":       # two unreduced blocks
        d, e = rng.standard_normal(12), rng.standard_normal(11)
        e[5] = 0.0
    elif case == "tiny_offdiag":
        d, e = np.arange(1.0, 11.0), 1e-17 * np.ones(9)
    elif case == "one":
        d, e = np.array([3.25]), np.zeros(0)
    else:
        d, e = np.array([1.0, 1.0]), np.array([2.0])
    T = _tridiag(d, e)
    w = np.sort(vals.tri(d, e))
    ref = np.linalg.eigvalsh(T)
    tn = max(1.0, np.abs(T).sum(axis=1).max())
    np.testing.assert_allclose(w, ref, rtol=0, atol=1e-13 * tn)
    gaps = np.diff(ref)
    pick = [i for i in range(len(ref)) if (i == 0 or gaps[i - 1] > 1e-6 * tn) and (i == len(ref) - 1 or gaps[i] > 1e-6 * tn)]
    V = []
    for i in pick[:10]:
        v = vals.tri_vec(d, e, w[i])
        assert abs(np.linalg.norm(v) - 1.0) < 1e-12
        assert np.linalg.norm(T @ v - w[i] * v) <= 1e-12 * tn
        V.append(v)
    if len(V) > 1:
        G = np.array(V) @ np.array(V).T
        assert np.abs(G - np.eye(len(V))).max() < 1e-8


def test_ritz_selection_smallest_real_pairs(eig):
    """The k smallest Ritz pairs of H_m by real part, in ascending order, with H C = C diag(theta)."""
    vals, _ = eig
    rng = np.random.default_rng(20)
    n, m = 300, 80
    Q = np.linalg.qr(rng.standard_normal((n, n)))[0]
    A = (Q * np.concatenate([np.geomspace(1e-3, 0.2, 20), 1.0 + rng.random(n - 20)])) @ Q.T
    H = _arnoldi((0.5 + rng.random(n))[:, None] * A, m, 21)
    rs, Cm, th = vals.ritz(H=H, k=10)
    assert rs == 0 and Cm.shape == (m, 10)
    full = np.sort(np.linalg.eigvals(H).real)
    ref = full[:10]
    np.testing.assert_allclose(th, ref, rtol=1e-10)
    assert np.all(np.diff(th) >= 0)
    np.testing.assert_allclose(H @ Cm, Cm * th, atol=1e-10 * np.abs(H).max())
    # k <= 0: every value below eps_lambda
    rs, Cm, th = vals.ritz(H=H, k=0, eps=0.1)
    assert rs == 0 and np.all(th < 0.1) and len(th) == int((full < 0.1).sum())
    assert vals.ritz(H=H, k=0, eps=1e-9)[0] == 2              # nothing below: no Ritz value selected
    # k <= 0 keeps at most kmax vectors (the coarse-space kernels' capacity)
    rs, Cm, th = vals.ritz(H=H, k=0, eps=10.0, kmax=7)
    assert rs == 0 and Cm.shape == (m, 7)
    np.testing.assert_allclose(th, full[:7], rtol=1e-10)


def test_ritz_selection_splits_complex_pairs_and_skips_null_values(eig):
    vals, _ = eig
    # block diagonal: a rotation-scaling block (values 1 +- 2i), then 3 and 5, and an exact 0 (null direction)
    H = np.zeros((5, 5))
    H[0:2, 0:2] = [[1.0, 2.0], [-2.0, 1.0]]
    H[2, 2], H[3, 3], H[4, 4] = 3.0, 5.0, 0.0
    H[1, 2] = 0.3
    H[3, 4] = 0.2
    rs, Cm, th = vals.ritz(H=H, k=3)
    assert rs == 0 and Cm.shape == (5, 3)
    np.testing.assert_allclose(th, [1.0, 1.0, 3.0], atol=1e-13)      # the 0 is skipped, the pair gives 2 columns
    P = Cm[:, :2]                                                    # real and imaginary parts span an invariant plane
    R = H @ P - P @ np.linalg.lstsq(P, H @ P, rcond=None)[0]
    assert np.abs(R).max() < 1e-12
    np.testing.assert_allclose(H @ Cm[:, 2], 3.0 * Cm[:, 2], atol=1e-12)
    # k = 1 stops inside the pair: one column only
    rs, Cm, th = vals.ritz(H=H, k=1)
    assert rs == 0 and Cm.shape == (5, 1)


def test_ritz_selection_of_the_lanczos_tridiagonal(eig):
    vals, _ = eig
    rng = np.random.default_rng(22)
    al = 0.5 + rng.random(60)
    be = 0.8 * rng.random(59)
    d = 1.0 / al + np.concatenate([[0.0], be / al[:-1]])
    e = -np.sqrt(be) / al[:-1]
    T = _tridiag(d, e)
    rs, Cm, th = vals.ritz(d=d, e=e, k=8)
    assert rs == 0 and Cm.shape == (60, 8)
    np.testing.assert_allclose(th, np.linalg.eigvalsh(T)[:8], atol=1e-13 * np.abs(T).sum(axis=1).max())
    np.testing.assert_allclose(Cm.T @ Cm, np.eye(8), atol=1e-10)
    np.testing.assert_allclose(T @ Cm, Cm * th, atol=1e-11)


@pytest.mark.parametrize("order", [0, 1, 2, 3])
def test_template_layout_gram_inverses_and_block_map(eig, order):
    """Per subscan, (B^T B)^-1 of the Legendre columns P_0..P_min(K, m-1) at u = 2 (i + 1/2) / m - 1
    equals numpy's inverse of legvander's Gram matrix (short subscans take order m - 1); every block
    maps to its first subscan."""
    from numpy.polynomial import legendre
    vals, _ = eig
    block_off = np.array([0, 100, 100, 230, 300])         # one empty block
    so = np.array([0, 1, 3, 40, 100, 101, 150, 230, 300])   # subscans of 1, 2, 37, 60, 1, 49, 80, 70 samples
    bs, g = vals.layout(block_off, so, order)
    assert list(bs) == [0, 4, 4, 7, 8]
    for s in range(len(so) - 1):
        m = so[s + 1] - so[s]
        K = min(order, m - 1)
        u = 2.0 * (np.arange(m) + 0.5) / m - 1.0
        B = legendre.legvander(u, K)
        ref = np.linalg.inv(B.T @ B)
        np.testing.assert_allclose(g[s, :K + 1, :K + 1], ref, rtol=1e-11, atol=1e-13)
        assert np.all(g[s, K + 1:, :] == 0.0) and np.all(g[s, :, K + 1:] == 0.0)


def test_template_layout_rejects_bad_subscans(eig):
    vals, _ = eig
    bo = np.array([0, 100, 200])
    assert vals.layout(bo, [0, 50, 150, 200], 1) == "every subscan must lie inside one block"
    assert vals.layout(bo, [0, 50, 50, 100, 200], 1) == "subscan_off must be strictly increasing"
    bs, g = vals.layout(bo, [0, 100, 200], -1)               # no polynomials: blocks as subscans, no Gram data
    assert list(bs) == [0, 1, 2] and np.all(g == 0.0)


def _angle(A, B):
    """Sine of the largest principal angle between the column spans of A and B (equal dimensions)."""
    qa, _ = np.linalg.qr(A)
    qb, _ = np.linalg.qr(B)
    return float(np.linalg.norm(qa - qb @ (qb.T @ qa), 2))


def _tiny_problem():
    import synth
    from helpers import oracle_problem
    scan = synth.make_scan(seed=3, **synth.CONFIGS["small"])
    prob, mbd, good = oracle_problem(scan)
    d = synth.make_tod(scan, synth.make_sky(scan.n_pix, 3), synth.make_noise(scan, 3))
    return prob, mbd, d


def test_coarse_space_from_a_harvested_solve_matches_the_oracle(eig):
    """Host side of mm_build_coarse_from_solve against the oracle: T_m from the PCG coefficients of an
    M_BD run equals the oracle's Lanczos matrix, its k smallest Ritz values match, and V_m C spans the
    oracle's deflation basis."""
    import oracle as O
    vals, _ = eig
    prob, mbd, d = _tiny_problem()
    A = lambda v: O.apply_A(prob, v).reshape(-1)
    M = lambda v: O.bd_apply(mbd, v).reshape(-1)
    b = O.rhs(prob, d).reshape(-1)
    al, be, V = O.pcg_lanczos(A, M, b, 40)
    lam, Q, T = O.lanczos_ritz(al, be, V, 8)
    dd, ee = vals.lanczos(al, be)
    np.testing.assert_allclose(dd, np.diag(T), rtol=1e-15)
    np.testing.assert_allclose(ee, np.diag(T, 1), rtol=1e-15)
    rs, Cm, th = vals.ritz(d=dd, e=ee, k=8)
    assert rs == 0
    np.testing.assert_allclose(th, lam, rtol=1e-10)
    assert _angle(V @ Cm, Q) < 1e-8


def test_coarse_space_from_arnoldi_matches_the_oracle(eig):
    """Host side of mm_build_coarse: the Ritz selection from the Arnoldi H_m of B = M_BD A gives the
    oracle's Ritz values and spans the oracle's deflation basis W_m Y."""
    import oracle as O
    vals, _ = eig
    prob, mbd, d = _tiny_problem()
    A = lambda v: O.apply_A(prob, v).reshape(-1)
    M = lambda v: O.bd_apply(mbd, v).reshape(-1)
    r0 = M(O.rhs(prob, d).reshape(-1))
    W, H, m = O.arnoldi(lambda v: M(A(v)), r0, 40, 1e-12)
    Q, ref = O.ritz_basis(W, H, m, 8)
    rs, Cm, th = vals.ritz(H=H[:m, :m], k=8)
    assert rs == 0 and Cm.shape[1] == len(ref)
    np.testing.assert_allclose(th, ref, rtol=1e-9)
    assert _angle(W[:, :m] @ Cm, Q) < 1e-7


@pytest.mark.parametrize("stokes", [1, 2])
def test_ritz_selection_on_template_filtered_operators(eig, stokes):
    """Arnoldi H_m of M_BD A under the template filters (clustered small eigenvalues; for d^+ an exact
    null vector, the constant intensity map): the host selection skips the null Ritz value, keeps the
    k smallest of the rest as the oracle's eigen-solve orders them, and spans the same basis."""
    import oracle as O
    import synth
    vals, _ = eig
    scan = synth.make_scan(nx=8, ny=4, n_det=4, n_t=1024, n_int=2, half_bw=0, f_knee=0.0, seed=3, hwp=False)
    so, az, nb = synth.make_templates(scan)
    order = 1 if stokes == 1 else 0
    tp = O.TemplateProblem(scan.pix, scan.psi, scan.block_off, scan.band[scan.block_band, 0], scan.n_pix, so,
                           order, az, nb, stokes)
    blocks, hits = O.bd_blocks_T(tp)
    good = O.select_pixels_T(blocks, hits, stokes)
    tp = tp.with_pix(O.flag_samples(tp.pix, good))
    blocks, _ = O.bd_blocks_T(tp)
    mbd = O.bd_inverse_T(blocks, good, stokes)
    B = lambda v: O.bd_apply(mbd, O.apply_A_T(tp, v.reshape(-1, 3))).reshape(-1)
    r0 = np.random.default_rng(4).standard_normal(3 * scan.n_pix)
    r0[0::3] *= float(stokes != 1)                                # d^-: the I entries are not unknowns
    if stokes == 2:
        r0[1::3] = r0[2::3] = 0.0                                 # d^+: nor are Q and U
    W, H, m = O.arnoldi(B, r0, 60, 1e-12)
    Hm = H[:m, :m]
    lam = np.linalg.eigvals(Hm)
    wmax = np.abs(lam.real).max()
    kept = np.sort(lam.real[np.abs(lam.real) > 1e-10 * wmax])
    rs, Cm, th = vals.ritz(H=Hm, k=10)
    assert rs == 0 and len(th) == 10
    np.testing.assert_allclose(th, kept[:10], rtol=1e-8, atol=1e-12 * wmax)
    assert np.all(np.abs(th) > 1e-10 * wmax)
    if stokes == 2:
        # r0 has a component along the constant intensity map, so the Krylov space holds the null
        # direction and H_m a zero Ritz value, which the selection leaves out
        assert np.abs(lam.real).min() <= 1e-10 * wmax
    Q, ref = O.ritz_basis(W, H, m, 40)
    ref = ref[np.abs(ref) > 1e-10 * wmax][:10]
    np.testing.assert_allclose(th, ref, rtol=1e-8, atol=1e-12 * wmax)


def test_shared_memory_configuration_only_rises_under_concurrent_launchers(eig):
    """Contexts set up on several host threads launch the same kernels: the dynamic shared-memory
    configuration is raised in increasing order only, ending at the largest size any thread asked for."""
    vals, _ = eig
    ok, last, calls, largest = vals.raise_smem()
    assert ok == 1 and last == largest and 1 <= calls <= largest
