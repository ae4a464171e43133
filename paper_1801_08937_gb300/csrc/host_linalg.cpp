// Small dense float64 linear algebra on the host: the eigen-solve of the
// Arnoldi Hessenberg matrix H_m (Appendix A, Eq. ritz; m <= a few hundred),
// the Cholesky factor of the coarse operator E = Z^T A Z (Sect. 3.2) and the
// triangular inverses used to orthonormalise Z.
//
// Eigenvalues: single-shift QR iteration on the complex upper Hessenberg
// matrix with Wilkinson shifts and Givens rotations (deflating from the
// bottom).  Eigenvectors: inverse iteration with the Hessenberg LU of
// (H - lambda I), three sweeps from a fixed start vector.
#include <cmath>
#include <complex>
#include <vector>

#include "common.cuh"

namespace mm {

using cd = std::complex<double>;

static bool hess_eigenvalues(std::vector<cd> a, int n, std::vector<cd>& ev) {
    auto A = [&](int i, int j) -> cd& { return a[(size_t)i * n + j]; };
    ev.assign(n, cd(0, 0));
    const double eps = 2.220446049250313e-16;
    int hi = n - 1;
    int iter = 0, total = 0;
    while (hi >= 0) {
        if (hi == 0) {
            ev[0] = A(0, 0);
            break;
        }
        int l = hi;
        while (l > 0) {
            const double s = std::abs(A(l - 1, l - 1)) + std::abs(A(l, l));
            if (std::abs(A(l, l - 1)) <= eps * (s > 0 ? s : 1.0)) {
                A(l, l - 1) = 0.0;
                break;
            }
            --l;
        }
        if (l == hi) {
            ev[hi] = A(hi, hi);
            --hi;
            iter = 0;
            continue;
        }
        if (++total > 60 * n + 200) return false;
        ++iter;
        // Wilkinson shift from the trailing 2x2 block
        cd mu;
        const cd p = A(hi - 1, hi - 1), q = A(hi - 1, hi), r = A(hi, hi - 1), d = A(hi, hi);
        if (iter % 11 == 10) {
            mu = d + std::abs(r) * 0.75;   // exceptional shift
        } else {
            const cd half = 0.5 * (p - d);
            const cd disc = std::sqrt(half * half + q * r);
            const cd m1 = d - q * r / (half + disc), m2 = d - q * r / (half - disc);
            const bool use1 = std::abs(half + disc) >= std::abs(half - disc);
            mu = use1 ? m1 : m2;
            if (!std::isfinite(mu.real()) || !std::isfinite(mu.imag())) mu = d;
        }
        // QR step on the active block [l, hi]
        const int m = hi - l + 1;
        std::vector<double> cs(m);
        std::vector<cd> sn(m);
        for (int k = l; k <= hi; ++k) A(k, k) -= mu;
        for (int k = l; k < hi; ++k) {
            const cd x = A(k, k), y = A(k + 1, k);
            const double ax = std::abs(x), ay = std::abs(y);
            const double rr = std::hypot(ax, ay);
            double c;
            cd s;
            if (rr == 0.0) {
                c = 1.0;
                s = 0.0;
            } else if (ax == 0.0) {
                c = 0.0;
                s = std::conj(y) / ay;
            } else {
                c = ax / rr;
                s = (x / ax) * std::conj(y) / rr;
            }
            cs[k - l] = c;
            sn[k - l] = s;
            for (int j = k; j <= hi; ++j) {
                const cd u = A(k, j), v = A(k + 1, j);
                A(k, j) = c * u + s * v;
                A(k + 1, j) = -std::conj(s) * u + c * v;
            }
        }
        for (int k = l; k < hi; ++k) {
            const double c = cs[k - l];
            const cd s = sn[k - l];
            const int iend = (k + 2 < hi) ? k + 2 : hi;
            for (int i = l; i <= iend; ++i) {
                const cd u = A(i, k), v = A(i, k + 1);
                A(i, k) = u * c + v * std::conj(s);
                A(i, k + 1) = -u * s + v * c;
            }
        }
        for (int k = l; k <= hi; ++k) A(k, k) += mu;
    }
    return true;
}

// Solve (H - sigma I) y = b for upper Hessenberg H with partial pivoting
// between adjacent rows; tiny pivots are replaced by a perturbation.
static void hess_shifted_solve(const std::vector<double>& H, int n, cd sigma, std::vector<cd>& b, double hnorm) {
    std::vector<cd> a((size_t)n * n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) a[(size_t)i * n + j] = H[(size_t)i * n + j] - (i == j ? sigma : cd(0));
    auto A = [&](int i, int j) -> cd& { return a[(size_t)i * n + j]; };
    const double tiny = 1e-14 * (hnorm > 0 ? hnorm : 1.0);
    for (int k = 0; k < n - 1; ++k) {
        if (std::abs(A(k + 1, k)) > std::abs(A(k, k))) {
            for (int j = k; j < n; ++j) std::swap(A(k, j), A(k + 1, j));
            std::swap(b[k], b[k + 1]);
        }
        if (std::abs(A(k, k)) < tiny) A(k, k) = tiny;
        const cd f = A(k + 1, k) / A(k, k);
        if (f != cd(0)) {
            for (int j = k; j < n; ++j) A(k + 1, j) -= f * A(k, j);
            b[k + 1] -= f * b[k];
        }
    }
    if (std::abs(A(n - 1, n - 1)) < tiny) A(n - 1, n - 1) = tiny;
    for (int i = n - 1; i >= 0; --i) {
        cd s = b[i];
        for (int j = i + 1; j < n; ++j) s -= A(i, j) * b[j];
        b[i] = s / A(i, i);
    }
}

bool host_eig(const std::vector<double>& H, int m, std::vector<double>& wr, std::vector<double>& wi,
              std::vector<double>& vr, std::vector<double>& vi) {
    std::vector<cd> a((size_t)m * m);
    double hnorm = 0.0;
    for (size_t i = 0; i < a.size(); ++i) {
        a[i] = H[i];
        hnorm = std::max(hnorm, std::abs(H[i]));
    }
    std::vector<cd> ev;
    if (!hess_eigenvalues(a, m, ev)) return false;
    wr.resize(m);
    wi.resize(m);
    vr.assign((size_t)m * m, 0.0);
    vi.assign((size_t)m * m, 0.0);
    for (int j = 0; j < m; ++j) {
        // clean near-real values so conjugate pairs and real values are unambiguous
        cd lam = ev[j];
        if (std::abs(lam.imag()) <= 1e-12 * (std::abs(lam) + hnorm * 1e-3)) lam = cd(lam.real(), 0.0);
        wr[j] = lam.real();
        wi[j] = lam.imag();
        std::vector<cd> y(m);
        for (int i = 0; i < m; ++i) y[i] = cd(1.0 + 0.01 * ((i * 7919) % 101), 0.0);
        const cd sigma = lam + cd(1e-13 * (hnorm > 0 ? hnorm : 1.0), 0.0);
        for (int sweep = 0; sweep < 3; ++sweep) {
            hess_shifted_solve(H, m, sigma, y, hnorm);
            double nrm = 0.0;
            int imax = 0;
            for (int i = 0; i < m; ++i) {
                nrm += std::norm(y[i]);
                if (std::abs(y[i]) > std::abs(y[imax])) imax = i;
            }
            nrm = std::sqrt(nrm);
            if (!(nrm > 0) || !std::isfinite(nrm)) return false;
            // unit norm, largest component real and positive
            const cd ph = std::abs(y[imax]) > 0 ? std::conj(y[imax]) / std::abs(y[imax]) : cd(1, 0);
            for (int i = 0; i < m; ++i) y[i] *= ph / nrm;
        }
        for (int i = 0; i < m; ++i) {
            vr[(size_t)i * m + j] = y[i].real();
            vi[(size_t)i * m + j] = (wi[j] == 0.0) ? 0.0 : y[i].imag();
        }
    }
    return true;
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
    // inv = L^-T L^-1, column by column
    inv.assign((size_t)n * n, 0.0);
    std::vector<double> y(n);
    for (int c = 0; c < n; ++c) {
        for (int i = 0; i < n; ++i) {
            double s = (i == c) ? 1.0 : 0.0;
            for (int k = 0; k < i; ++k) s -= L[(size_t)i * n + k] * y[k];
            y[i] = s / L[(size_t)i * n + i];
        }
        for (int i = n - 1; i >= 0; --i) {
            double s = y[i];
            for (int k = i + 1; k < n; ++k) s -= L[(size_t)k * n + i] * inv[(size_t)k * n + c];
            inv[(size_t)i * n + c] = s / L[(size_t)i * n + i];
        }
    }
}

void host_upper_inverse(const std::vector<double>& R, int n, std::vector<double>& Rinv) {
    Rinv.assign((size_t)n * n, 0.0);
    for (int c = 0; c < n; ++c) {
        for (int i = n - 1; i >= 0; --i) {
            double s = (i == c) ? 1.0 : 0.0;
            for (int k = i + 1; k < n; ++k) s -= R[(size_t)i * n + k] * Rinv[(size_t)k * n + c];
            Rinv[(size_t)i * n + c] = s / R[(size_t)i * n + i];
        }
    }
}

}  // namespace mm
