// Small dense float64 linear algebra on the host: the eigen-solve of the
// Arnoldi Hessenberg matrix H_m (Appendix A, Eq. ritz; m up to about a
// thousand) and of the Lanczos tridiagonal matrix, the Cholesky factor of the
// coarse operator E = Z^T A Z (Sect. 3.2) and the triangular inverses used to
// orthonormalise Z.
//
// Eigenvalues: Francis double-shift QR iteration in real arithmetic on the
// active window of the upper Hessenberg matrix (3-element Householder
// reflectors chase the bulge; 1x1 and 2x2 blocks deflate from the bottom; an
// exceptional shift every tenth iteration without deflation).  Only the
// window is updated, which is all the eigenvalues need.  Eigenvectors, for
// the wanted eigenvalues only: inverse iteration with one Hessenberg LU of
// (H - sigma I) (pivoting between adjacent rows) and three solves from a
// fixed start vector; real arithmetic for a real eigenvalue.  The symmetric
// tridiagonal Lanczos matrix has its own solver: implicit QR steps with the
// Wilkinson shift (O(m) per step) and inverse iteration with a tridiagonal
// LU (O(m) per solve).
#include <algorithm>
#include <array>
#include <cstdint>
#include <cmath>
#include <complex>
#include <map>
#include <string>
#include <vector>

#include "common.cuh"

namespace mm {

using cd = std::complex<double>;

namespace {

double max_abs(const std::vector<double>& H, int n) {
    double h = 0.0;
    for (size_t i = 0; i < (size_t)n * n; ++i) h = std::max(h, std::fabs(H[i]));
    return h;
}

// Eigenvalues of the 2x2 block [[a, b], [c, d]].
void eig2(double a, double b, double c, double d, double& r1, double& i1, double& r2, double& i2) {
    const double mid = 0.5 * (a + d), p = 0.5 * (a - d);
    const double disc = p * p + b * c;
    if (disc >= 0.0) {
        const double sq = std::sqrt(disc);
        r1 = mid + sq;
        r2 = mid - sq;
        i1 = i2 = 0.0;
    } else {
        const double sq = std::sqrt(-disc);
        r1 = r2 = mid;
        i1 = sq;
        i2 = -sq;
    }
}

// Unit 2-norm, largest component real and positive.
bool normalise(std::vector<double>& y) {
    double nrm = 0.0;
    int imax = 0;
    for (size_t i = 0; i < y.size(); ++i) {
        nrm += y[i] * y[i];
        if (std::fabs(y[i]) > std::fabs(y[imax])) imax = (int)i;
    }
    nrm = std::sqrt(nrm);
    if (!(nrm > 0) || !std::isfinite(nrm)) return false;
    const double f = (y[imax] < 0 ? -1.0 : 1.0) / nrm;
    for (double& v : y) v *= f;
    return true;
}
bool normalise(std::vector<cd>& y) {
    double nrm = 0.0;
    int imax = 0;
    for (size_t i = 0; i < y.size(); ++i) {
        nrm += std::norm(y[i]);
        if (std::abs(y[i]) > std::abs(y[imax])) imax = (int)i;
    }
    nrm = std::sqrt(nrm);
    if (!(nrm > 0) || !std::isfinite(nrm)) return false;
    const cd ph = std::abs(y[imax]) > 0 ? std::conj(y[imax]) / std::abs(y[imax]) : cd(1, 0);
    for (cd& v : y) v *= ph / nrm;
    return true;
}

// sum_j a[j] b[j] with four independent partial sums (the back-substitution
// is otherwise one serial chain of dependent additions).
template <typename S>
S dot4(const S* a, const S* b, int len) {
    S s0 = S(0), s1 = S(0), s2 = S(0), s3 = S(0);
    int j = 0;
    for (; j + 4 <= len; j += 4) {
        s0 += a[j] * b[j];
        s1 += a[j + 1] * b[j + 1];
        s2 += a[j + 2] * b[j + 2];
        s3 += a[j + 3] * b[j + 3];
    }
    for (; j < len; ++j) s0 += a[j] * b[j];
    return (s0 + s1) + (s2 + s3);
}

// Inverse iteration for the eigenvector of the upper Hessenberg H (n x n,
// row-major) closest to sigma; S is double or complex.  The LU of
// (H - sigma I) is formed in one pass over H (the pivot row is carried in a
// buffer; rows of U are stored packed from their diagonal).  Tiny pivots are
// replaced by a perturbation of the order of 1e-14 ||H||.
template <typename S>
bool inverse_iteration(const std::vector<double>& H, int n, S sigma, double hnorm, std::vector<S>& y) {
    const double tiny = 1e-14 * (hnorm > 0 ? hnorm : 1.0);
    std::vector<size_t> off(n + 1);
    off[0] = 0;
    for (int i = 0; i < n; ++i) off[i + 1] = off[i] + (size_t)(n - i);
    std::vector<S> u(off[n]);
    std::vector<char> swp(n, 0);
    std::vector<S> mult(n, S(0));
    std::vector<S> bufa(n), bufb(n);
    S* cur = bufa.data();
    S* nxt = bufb.data();
    for (int j = 0; j < n; ++j) cur[j] = H[j];
    cur[0] -= sigma;
    for (int k = 0; k + 1 < n; ++k) {
        const double* hr = &H[(size_t)(k + 1) * n];
        for (int j = k; j < n; ++j) nxt[j] = hr[j];
        nxt[k + 1] -= sigma;
        if (std::abs(nxt[k]) > std::abs(cur[k])) {
            swp[k] = 1;
            std::swap(cur, nxt);
        }
        if (std::abs(cur[k]) < tiny) cur[k] = tiny;
        const S f = nxt[k] / cur[k];
        mult[k] = f;
        S* ur = &u[off[k]];
        for (int j = k; j < n; ++j) ur[j - k] = cur[j];
        for (int j = k + 1; j < n; ++j) nxt[j] -= f * cur[j];
        std::swap(cur, nxt);
    }
    if (std::abs(cur[n - 1]) < tiny) cur[n - 1] = tiny;
    u[off[n - 1]] = cur[n - 1];
    y.resize(n);
    for (int i = 0; i < n; ++i) y[i] = S(1.0 + 0.01 * ((i * 7919) % 101));
    for (int sweep = 0; sweep < 3; ++sweep) {
        for (int k = 0; k + 1 < n; ++k) {
            if (swp[k]) std::swap(y[k], y[k + 1]);
            y[k + 1] -= mult[k] * y[k];
        }
        for (int i = n - 1; i >= 0; --i) {
            const S* ur = &u[off[i]];
            y[i] = (y[i] - dot4(ur + 1, &y[i + 1], n - i - 1)) / ur[0];
        }
        if (!normalise(y)) return false;
    }
    return true;
}

}  // namespace

bool host_hess_eigvals(const std::vector<double>& H, int n, std::vector<double>& wr, std::vector<double>& wi) {
    std::vector<double> a(H.begin(), H.begin() + (size_t)n * n);
    auto A = [&](int i, int j) -> double& { return a[(size_t)i * n + j]; };
    wr.assign(n, 0.0);
    wi.assign(n, 0.0);
    const double hnorm = max_abs(H, n);
    const double eps = 2.220446049250313e-16;
    int hi = n - 1, its = 0, total = 0;
    while (hi >= 0) {
        int l = hi;
        for (; l > 0; --l) {
            double s = std::fabs(A(l - 1, l - 1)) + std::fabs(A(l, l));
            if (s == 0.0) s = hnorm;
            if (std::fabs(A(l, l - 1)) <= eps * s) {
                A(l, l - 1) = 0.0;
                break;
            }
        }
        if (l == hi) {
            wr[hi] = A(hi, hi);
            --hi;
            its = 0;
            continue;
        }
        if (l == hi - 1) {
            eig2(A(hi - 1, hi - 1), A(hi - 1, hi), A(hi, hi - 1), A(hi, hi), wr[hi - 1], wi[hi - 1], wr[hi], wi[hi]);
            hi -= 2;
            its = 0;
            continue;
        }
        if (++total > 40 * n + 100) return false;
        ++its;
        // shifts: the eigenvalues of the trailing 2x2 block (sum s, product t)
        double s, t;
        if (its % 10 == 0) {
            const double ex = std::fabs(A(hi, hi - 1)) + std::fabs(A(hi - 1, hi - 2));
            const double s1 = A(hi, hi) + 0.75 * ex, s2 = A(hi, hi) - 0.4375 * ex;
            s = s1 + s2;
            t = s1 * s2;
        } else {
            s = A(hi - 1, hi - 1) + A(hi, hi);
            t = A(hi - 1, hi - 1) * A(hi, hi) - A(hi - 1, hi) * A(hi, hi - 1);
        }
        // first column of (H - s1 I)(H - s2 I) = H^2 - s H + t I on the window
        double x = A(l, l) * A(l, l) + A(l, l + 1) * A(l + 1, l) - s * A(l, l) + t;
        double y = A(l + 1, l) * (A(l, l) + A(l + 1, l + 1) - s);
        double z = A(l + 1, l) * A(l + 2, l + 1);
        for (int k = l; k < hi; ++k) {
            const bool three = k + 2 <= hi;
            if (k > l) {
                x = A(k, k - 1);
                y = A(k + 1, k - 1);
                z = three ? A(k + 2, k - 1) : 0.0;
            }
            const double nrm = std::sqrt(x * x + y * y + z * z);
            if (nrm == 0.0) continue;
            const double alpha = x >= 0.0 ? -nrm : nrm;
            const double v0 = x - alpha, v1 = y, v2 = z;
            const double beta = 2.0 / (v0 * v0 + v1 * v1 + v2 * v2);
            // rows k..k+2 from the left
            for (int j = std::max(l, k - 1); j <= hi; ++j) {
                const double w = beta * (v0 * A(k, j) + v1 * A(k + 1, j) + (three ? v2 * A(k + 2, j) : 0.0));
                A(k, j) -= w * v0;
                A(k + 1, j) -= w * v1;
                if (three) A(k + 2, j) -= w * v2;
            }
            if (k > l) {
                A(k, k - 1) = alpha;
                A(k + 1, k - 1) = 0.0;
                if (three) A(k + 2, k - 1) = 0.0;
            }
            // columns k..k+2 from the right
            const int iend = std::min(k + 3, hi);
            for (int i = l; i <= iend; ++i) {
                const double w = beta * (A(i, k) * v0 + A(i, k + 1) * v1 + (three ? A(i, k + 2) * v2 : 0.0));
                A(i, k) -= w * v0;
                A(i, k + 1) -= w * v1;
                if (three) A(i, k + 2) -= w * v2;
            }
        }
    }
    // near-real values are made real, so conjugate pairs and real values are unambiguous
    for (int j = 0; j < n; ++j)
        if (std::fabs(wi[j]) <= 1e-12 * (std::hypot(wr[j], wi[j]) + hnorm * 1e-3)) wi[j] = 0.0;
    return true;
}

bool host_hess_eigvec(const std::vector<double>& H, int n, double wr, double wi, std::vector<double>& vr,
                      std::vector<double>& vi, double hnorm) {
    if (hnorm < 0.0) hnorm = max_abs(H, n);
    const double pert = 1e-13 * (hnorm > 0 ? hnorm : 1.0);
    vr.assign(n, 0.0);
    vi.assign(n, 0.0);
    if (wi == 0.0) {
        std::vector<double> y;
        if (!inverse_iteration<double>(H, n, wr + pert, hnorm, y)) return false;
        vr = y;
        return true;
    }
    std::vector<cd> y;
    if (!inverse_iteration<cd>(H, n, cd(wr + pert, wi), hnorm, y)) return false;
    for (int i = 0; i < n; ++i) {
        vr[i] = y[i].real();
        vi[i] = y[i].imag();
    }
    return true;
}

bool host_tridiag_eigvals(const std::vector<double>& d_in, const std::vector<double>& e_in, int n,
                          std::vector<double>& w) {
    // implicit symmetric QR steps with the Wilkinson shift on the unreduced
    // window [l, hi]; a Givens rotation on (k, k+1) chases the bulge, which
    // sits at (k+1, k-1) before step k
    w.assign(d_in.begin(), d_in.begin() + n);
    std::vector<double>& d = w;
    std::vector<double> e(e_in.begin(), e_in.begin() + std::max(0, n - 1));
    const double eps = 2.220446049250313e-16;
    int hi = n - 1, total = 0;
    while (hi > 0) {
        if (std::fabs(e[hi - 1]) <= eps * (std::fabs(d[hi - 1]) + std::fabs(d[hi]))) {
            e[hi - 1] = 0.0;
            --hi;
            continue;
        }
        int l = hi - 1;
        while (l > 0 && std::fabs(e[l - 1]) > eps * (std::fabs(d[l - 1]) + std::fabs(d[l]))) --l;
        if (l > 0) e[l - 1] = 0.0;
        if (++total > 30 * n + 100) return false;
        const double delta = 0.5 * (d[hi - 1] - d[hi]);
        const double eh = e[hi - 1];
        const double den = delta + (delta >= 0.0 ? 1.0 : -1.0) * std::hypot(delta, eh);
        const double mu = den != 0.0 ? d[hi] - eh * eh / den : d[hi];
        double x = d[l] - mu, z = e[l], bulge = 0.0;
        for (int k = l; k < hi; ++k) {
            if (k > l) {
                x = e[k - 1];
                z = bulge;
            }
            const double r = std::hypot(x, z);
            const double c = r != 0.0 ? x / r : 1.0, sn = r != 0.0 ? z / r : 0.0;
            if (k > l) e[k - 1] = r;
            const double a = d[k], b = e[k], f = d[k + 1];
            d[k] = c * c * a + 2.0 * c * sn * b + sn * sn * f;
            d[k + 1] = sn * sn * a - 2.0 * c * sn * b + c * c * f;
            e[k] = c * sn * (f - a) + (c * c - sn * sn) * b;
            if (k + 1 < hi) {
                bulge = sn * e[k + 1];
                e[k + 1] = c * e[k + 1];
            }
        }
    }
    return true;
}

bool host_tridiag_eigvec(const std::vector<double>& d, const std::vector<double>& e, int n, double lam,
                         std::vector<double>& v) {
    // inverse iteration with the LU of T - sigma I (row interchanges between
    // neighbours; U has two superdiagonals), three solves from a fixed start
    double tnorm = 0.0;
    for (int i = 0; i < n; ++i) tnorm = std::max(tnorm, std::fabs(d[i]) + (i > 0 ? std::fabs(e[i - 1]) : 0.0) +
                                                         (i + 1 < n ? std::fabs(e[i]) : 0.0));
    const double scale = tnorm > 0 ? tnorm : 1.0;
    const double sigma = lam + 1e-13 * scale, tiny = 1e-14 * scale;
    std::vector<double> u0(n), u1(n, 0.0), u2(n, 0.0), mult(n, 0.0);
    std::vector<char> swp(n, 0);
    double c0 = d[0] - sigma, c1 = n > 1 ? e[0] : 0.0, c2 = 0.0;   // pivot row at columns k, k+1, k+2
    for (int k = 0; k + 1 < n; ++k) {
        double n0 = e[k], n1 = d[k + 1] - sigma, n2 = k + 2 < n ? e[k + 1] : 0.0;
        if (std::fabs(n0) > std::fabs(c0)) {
            swp[k] = 1;
            std::swap(c0, n0);
            std::swap(c1, n1);
            std::swap(c2, n2);
        }
        if (std::fabs(c0) < tiny) c0 = tiny;
        const double f = n0 / c0;
        mult[k] = f;
        u0[k] = c0;
        u1[k] = c1;
        u2[k] = c2;
        c0 = n1 - f * c1;
        c1 = n2 - f * c2;
        c2 = 0.0;
    }
    if (std::fabs(c0) < tiny) c0 = tiny;
    u0[n - 1] = c0;
    v.resize(n);
    for (int i = 0; i < n; ++i) v[i] = 1.0 + 0.01 * ((i * 7919) % 101);
    for (int sweep = 0; sweep < 3; ++sweep) {
        for (int k = 0; k + 1 < n; ++k) {
            if (swp[k]) std::swap(v[k], v[k + 1]);
            v[k + 1] -= mult[k] * v[k];
        }
        for (int i = n - 1; i >= 0; --i) {
            double s = v[i];
            if (i + 1 < n) s -= u1[i] * v[i + 1];
            if (i + 2 < n) s -= u2[i] * v[i + 2];
            v[i] = s / u0[i];
        }
        if (!normalise(v)) return false;
    }
    return true;
}

namespace {

// The selection of the Ritz pairs (Appendix A, Eq. ritz) from the values
// wr + i wi; vec(idx, er, ei) computes the vector of value idx.  Sorted by
// real part, the k smallest are kept (k <= 0: those below eps_lambda, at
// most kmax of them, the size the coarse-space kernels hold); a
// complex pair gives its real and imaginary parts (its partner is not taken
// again); values at the round-off level of the largest are skipped: they
// belong to null directions of A (e.g. a constant intensity map under
// polynomial templates), which A Z cannot deflate and which would make
// E = Z^T A Z singular.
template <typename VecFn>
int select_ritz(int m, int k, int kmax, double eps_lambda, const std::vector<double>& wr,
                const std::vector<double>& wi, VecFn vec, std::vector<double>& C, std::vector<double>& vals) {
    std::vector<int> order(m);
    for (int i = 0; i < m; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return wr[a] < wr[b]; });
    std::vector<char> used(m, 0);
    std::vector<std::vector<double>> cols;
    vals.clear();
    const int kwant = std::min(k > 0 ? k : kmax, m);
    double wmax = 0.0;
    for (int i = 0; i < m; ++i) wmax = std::max(wmax, std::fabs(wr[i]));
    const double wnull = 1e-10 * wmax;
    std::vector<double> er, ei;
    for (int idx : order) {
        if ((int)cols.size() >= kwant) break;
        if (used[idx]) continue;
        if (std::fabs(wr[idx]) <= wnull) continue;
        if (k <= 0 && !(wr[idx] < eps_lambda)) break;
        used[idx] = 1;
        if (!vec(idx, er, ei)) return 1;
        cols.push_back(er);
        vals.push_back(wr[idx]);
        if (wi[idx] != 0.0) {
            int partner = -1;
            double best = 1e300;
            for (int j2 = 0; j2 < m; ++j2) {
                if (used[j2]) continue;
                const double dd = std::fabs(wr[j2] - wr[idx]) + std::fabs(wi[j2] + wi[idx]);
                if (dd < best) {
                    best = dd;
                    partner = j2;
                }
            }
            if (partner >= 0) used[partner] = 1;
            if ((int)cols.size() < kwant) {
                cols.push_back(ei);
                vals.push_back(wr[idx]);
            }
        }
    }
    const int ksel = (int)cols.size();
    if (ksel == 0) return 2;
    C.assign((size_t)m * ksel, 0.0);
    for (int r = 0; r < m; ++r)
        for (int c = 0; c < ksel; ++c) C[(size_t)r * ksel + c] = cols[c][r];
    return 0;
}

}  // namespace

int host_ritz_hess(const std::vector<double>& H, int m, int k, int kmax, double eps_lambda, std::vector<double>& C,
                   std::vector<double>& vals) {
    std::vector<double> wr, wi;
    if (!host_hess_eigvals(H, m, wr, wi)) return 1;
    const double hnorm = max_abs(H, m);
    auto vec = [&](int idx, std::vector<double>& er, std::vector<double>& ei) {
        return host_hess_eigvec(H, m, wr[idx], wi[idx], er, ei, hnorm);
    };
    return select_ritz(m, k, kmax, eps_lambda, wr, wi, vec, C, vals);
}

int host_ritz_tridiag(const std::vector<double>& d, const std::vector<double>& e, int m, int k, int kmax,
                      double eps_lambda, std::vector<double>& C, std::vector<double>& vals) {
    std::vector<double> wr;
    if (!host_tridiag_eigvals(d, e, m, wr)) return 1;
    const std::vector<double> wi(m, 0.0);
    auto vec = [&](int idx, std::vector<double>& er, std::vector<double>& ei) {
        ei.assign(m, 0.0);
        return host_tridiag_eigvec(d, e, m, wr[idx], er);
    };
    return select_ritz(m, k, kmax, eps_lambda, wr, wi, vec, C, vals);
}

bool host_cholesky(std::vector<double>& A, int n) {
    for (int j = 0; j < n; ++j) {
        double d = A[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) d -= A[(size_t)j * n + k] * A[(size_t)j * n + k];
        if (!(d > 0.0) || !std::isfinite(d)) return false;
        const double ljj = std::sqrt(d);
        A[(size_t)j * n + j] = ljj;
        for (int i = j + 1; i < n; ++i) {
            double s = A[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) s -= A[(size_t)i * n + k] * A[(size_t)j * n + k];
            A[(size_t)i * n + j] = s / ljj;
        }
        for (int k = j + 1; k < n; ++k) A[(size_t)j * n + k] = 0.0;
    }
    return true;
}

void host_spd_inverse_from_chol(const std::vector<double>& L, int n, std::vector<double>& inv) {
    // M = L^-1 row by row (row i = (e_i - sum_{k<i} L_ik M_k) / L_ii), then
    // inv = M^T M as a sum of outer products of the rows of M; row-major
    // throughout
    std::vector<double> M((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) {
        double* mi = &M[(size_t)i * n];
        mi[i] = 1.0;
        for (int k = 0; k < i; ++k) {
            const double f = L[(size_t)i * n + k];
            if (f == 0.0) continue;
            const double* mk = &M[(size_t)k * n];
            for (int c = 0; c <= k; ++c) mi[c] -= f * mk[c];
        }
        const double d = 1.0 / L[(size_t)i * n + i];
        for (int c = 0; c <= i; ++c) mi[c] *= d;
    }
    inv.assign((size_t)n * n, 0.0);
    for (int k = 0; k < n; ++k) {
        const double* mk = &M[(size_t)k * n];
        for (int a = 0; a <= k; ++a) {
            const double f = mk[a];
            if (f == 0.0) continue;
            double* ra = &inv[(size_t)a * n];
            for (int b = 0; b <= a; ++b) ra[b] += f * mk[b];
        }
    }
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < a; ++b) inv[(size_t)b * n + a] = inv[(size_t)a * n + b];
}

// Inverse of a symmetric positive semi-definite E restricted to the index set S
// that a diagonally pivoted Cholesky factorisation keeps: pivots are taken
// largest remaining Schur-complement diagonal first, and the factorisation
// stops once that diagonal falls to rel_tol times the largest diagonal of E.
// inv holds (E_SS)^-1 on S x S and 0 elsewhere, so that for E = Z^T A Z,
// Z inv Z^T = Z_S (Z_S^T A Z_S)^-1 Z_S^T: the coarse correction of the basis
// reduced to the columns in S.  Returns |S| (0 when E has no positive
// diagonal; -1 if the kept block is not positive definite after all).
int host_pivoted_spd_inverse(const std::vector<double>& E, int n, double rel_tol, std::vector<double>& inv) {
    inv.assign((size_t)n * n, 0.0);
    std::vector<double> d(n);
    double dmax = 0.0;
    for (int i = 0; i < n; ++i) {
        d[i] = E[(size_t)i * n + i];
        if (std::isfinite(d[i])) dmax = std::max(dmax, d[i]);
    }
    if (!(dmax > 0.0)) return 0;
    std::vector<int> S;
    std::vector<char> used(n, 0);
    std::vector<std::vector<double>> cols;   // columns of the pivoted factor, indexed by original row
    for (int r = 0; r < n; ++r) {
        int p = -1;
        double best = rel_tol * dmax;
        for (int i = 0; i < n; ++i)
            if (!used[i] && d[i] > best) {
                best = d[i];
                p = i;
            }
        if (p < 0) break;
        std::vector<double> l(n, 0.0);
        const double lp = std::sqrt(d[p]);
        for (int i = 0; i < n; ++i) {
            if (used[i] || i == p) continue;
            double v = E[(size_t)i * n + p];
            for (const auto& c : cols) v -= c[i] * c[p];
            l[i] = v / lp;
            d[i] -= l[i] * l[i];
        }
        l[p] = lp;
        used[p] = 1;
        S.push_back(p);
        cols.push_back(std::move(l));
    }
    const int m = (int)S.size();
    std::vector<double> Es((size_t)m * m), Einv;
    for (int a = 0; a < m; ++a)
        for (int b = 0; b < m; ++b) Es[(size_t)a * m + b] = E[(size_t)S[a] * n + S[b]];
    if (!host_cholesky(Es, m)) return -1;
    host_spd_inverse_from_chol(Es, m, Einv);
    for (int a = 0; a < m; ++a)
        for (int b = 0; b < m; ++b) inv[(size_t)S[a] * n + S[b]] = Einv[(size_t)a * m + b];
    return m;
}

void host_upper_inverse(const std::vector<double>& R, int n, std::vector<double>& Rinv) {
    // row i of R^-1 = (e_i - sum_{k>i} R_ik row k of R^-1) / R_ii, from the last row up
    Rinv.assign((size_t)n * n, 0.0);
    for (int i = n - 1; i >= 0; --i) {
        double* ri = &Rinv[(size_t)i * n];
        ri[i] = 1.0;
        for (int k = i + 1; k < n; ++k) {
            const double f = R[(size_t)i * n + k];
            if (f == 0.0) continue;
            const double* rk = &Rinv[(size_t)k * n];
            for (int c = k; c < n; ++c) ri[c] -= f * rk[c];
        }
        const double d = 1.0 / R[(size_t)i * n + i];
        for (int c = i; c < n; ++c) ri[c] *= d;
    }
}

void host_lanczos_tridiag(const std::vector<double>& alpha, const std::vector<double>& beta, int m,
                          std::vector<double>& d, std::vector<double>& e) {
    // PCG with M_BD is the Lanczos process of B = M_BD A in the M_BD^-1 inner
    // product; its coefficients give T_m with diagonal
    // 1/alpha_j + beta_{j-1}/alpha_{j-1} and off-diagonal -sqrt(beta_j)/alpha_j
    d.assign(m, 0.0);
    e.assign(std::max(1, m - 1), 0.0);
    for (int j = 0; j < m; ++j) {
        d[j] = 1.0 / alpha[j] + (j > 0 ? beta[j - 1] / alpha[j - 1] : 0.0);
        if (j + 1 < m) e[j] = -std::sqrt(std::max(0.0, beta[j])) / alpha[j];
    }
}

bool host_template_layout(const std::vector<int64_t>& block_off, const std::vector<int64_t>& so, int poly_order,
                          std::vector<int32_t>& blk_sub, std::vector<double>& ginv, std::string& err) {
    const int nb = (int)block_off.size() - 1, ns = (int)so.size() - 1;
    blk_sub.assign(nb + 1, 0);
    int b = 0;
    for (int s = 0; s < ns; ++s) {
        if (so[s + 1] <= so[s]) {
            err = "subscan_off must be strictly increasing";
            return false;
        }
        while (block_off[b + 1] <= so[s]) blk_sub[++b] = s;
        if (so[s] < block_off[b] || so[s + 1] > block_off[b + 1]) {
            err = "every subscan must lie inside one block";
            return false;
        }
    }
    while (b < nb) blk_sub[++b] = ns;
    for (int bb = 0; bb < nb; ++bb)
        if (so[blk_sub[bb]] != block_off[bb]) {
            err = "block boundaries must be subscan boundaries";
            return false;
        }
    // G = B^T B of the Legendre columns P_0..P_Ks at u_i = 2 (i + 1/2) / m - 1,
    // Ks = min(K, m - 1), inverted once per distinct subscan length
    ginv.assign((size_t)ns * 16, 0.0);
    if (poly_order < 0) return true;
    std::map<int64_t, std::array<double, 16>> cache;
    for (int s = 0; s < ns; ++s) {
        const int64_t m = so[s + 1] - so[s];
        auto it = cache.find(m);
        if (it == cache.end()) {
            const int K = (int)std::min<int64_t>(poly_order, m - 1), n = K + 1;
            std::vector<double> G((size_t)n * n, 0.0), Gi;
            for (int64_t i = 0; i < m; ++i) {
                const double u = 2.0 * ((double)i + 0.5) / (double)m - 1.0;
                const double p[4] = {1.0, u, 1.5 * u * u - 0.5, (2.5 * u * u - 1.5) * u};
                for (int j = 0; j < n; ++j)
                    for (int l = 0; l < n; ++l) G[(size_t)j * n + l] += p[j] * p[l];
            }
            if (!host_cholesky(G, n)) {
                err = "singular subscan Gram matrix";
                return false;
            }
            host_spd_inverse_from_chol(G, n, Gi);
            std::array<double, 16> g{};
            for (int j = 0; j < n; ++j)
                for (int l = 0; l < n; ++l) g[j * 4 + l] = Gi[(size_t)j * n + l];
            it = cache.emplace(m, g).first;
        }
        std::copy(it->second.begin(), it->second.end(), ginv.begin() + (size_t)s * 16);
    }
    return true;
}

}  // namespace mm
