// Host numerics of klecgc_setup (offline part of Algorithm 3).
//
//  - KL eigenpairs of sigma^2 exp(-|x-y|/ell) on [0,1]: on the centred interval
//    [-1/2, 1/2] with c = 1/ell the eigenvalues are 2 c sigma^2 / (w^2 + c^2),
//    w the roots of c - w tan(w/2) = 0 (cosine modes) and w + c tan(w/2) = 0
//    (sine modes), one root per half period; found here by bisection.
//  - Total-degree multi-indices of the Hermite gPC basis (eq. complete),
//    ordered by degree, then decreasing lexicographically.
//  - Symmetric eigensolver for the snapshot covariance C (Section 2.1):
//    Householder reduction to tridiagonal form, then implicit QL iterations
//    with a shift from the leading 2x2 block, eigenvectors accumulated.
//  - Least squares h = argmin ||B h - D||_2 (eq. least square problem) by
//    Householder QR.
#include "setup_host.h"

#include <algorithm>
#include <cmath>
#include <numeric>

namespace klecgc {

static double bisect(double (*f)(double, double), double c, double lo, double hi) {
    double flo = f(lo, c);
    for (int it = 0; it < 400; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        double fm = f(mid, c);
        if ((fm < 0) == (flo < 0)) {
            lo = mid;
            flo = fm;
        } else {
            hi = mid;
        }
    }
    return 0.5 * (lo + hi);
}

static double even_eq(double w, double c) { return c - w * std::tan(0.5 * w); }
static double odd_eq(double w, double c) { return w + c * std::tan(0.5 * w); }

void kl_modes_1d(double corr_len, double sigma, int count, std::vector<double>& lam,
                 std::vector<double>& omega, std::vector<int>& parity) {
    const double c = 1.0 / corr_len, pi = 3.14159265358979323846;
    lam.clear();
    omega.clear();
    parity.clear();
    for (int k = 0; (int)omega.size() < count; ++k) {
        // cosine mode: w in (2k pi, 2k pi + pi); sine mode: w in (2k pi + pi, 2k pi + 2 pi)
        double lo = 2 * k * pi, hi = lo + pi;
        double off = 1e-10 * std::max(1.0, hi);
        omega.push_back(bisect(even_eq, c, k == 0 ? 0.0 : lo + off, hi - off));
        parity.push_back(0);
        if ((int)omega.size() == count) break;
        lo = hi;
        hi = lo + pi;
        off = 1e-10 * std::max(1.0, hi);
        omega.push_back(bisect(odd_eq, c, lo + off, hi - off));
        parity.push_back(1);
    }
    for (double w : omega) lam.push_back(2.0 * c * sigma * sigma / (w * w + c * c));
}

void kl_modes_2d(double corr_len, double sigma, int count, std::vector<double>& lam,
                 std::vector<int>& mi, std::vector<int>& mj, std::vector<double>& mu,
                 std::vector<double>& omega, std::vector<int>& parity) {
    // The separable kernel sigma^2 exp(-|x1-y1|/l) exp(-|x2-y2|/l) has the
    // eigenpairs (sigma^2 mu_i mu_j, phi_i(x1) phi_j(x2)) of the unit-variance
    // 1D pairs.  A pair among the top `count` has both indices below count.
    const int n1 = count + 2;
    kl_modes_1d(corr_len, 1.0, n1, mu, omega, parity);
    struct Pair {
        double lam;
        int i, j;
    };
    std::vector<Pair> all;
    for (int i = 0; i < n1; ++i)
        for (int j = 0; j < n1; ++j) all.push_back({sigma * sigma * (mu[i] * mu[j]), i, j});
    // descending eigenvalue; (i, j) and (j, i) tie exactly: smaller i + j, then smaller i
    std::stable_sort(all.begin(), all.end(), [](const Pair& a, const Pair& b) {
        if (a.lam != b.lam) return a.lam > b.lam;
        if (a.i + a.j != b.i + b.j) return a.i + a.j < b.i + b.j;
        return a.i < b.i;
    });
    lam.clear();
    mi.clear();
    mj.clear();
    for (int m = 0; m < count; ++m) {
        lam.push_back(all[m].lam);
        mi.push_back(all[m].i);
        mj.push_back(all[m].j);
    }
}

double kl_phi_1d(double x, double w, int parity) {
    double t = x - 0.5;
    if (parity == 0) return std::cos(w * t) / std::sqrt(0.5 + std::sin(w) / (2.0 * w));
    return std::sin(w * t) / std::sqrt(0.5 - std::sin(w) / (2.0 * w));
}

static void degree_level(int M, int d, std::vector<int>& cur, std::vector<int>& out) {
    if ((int)cur.size() == M - 1) {
        cur.push_back(d);
        out.insert(out.end(), cur.begin(), cur.end());
        cur.pop_back();
        return;
    }
    for (int first = d; first >= 0; --first) {
        cur.push_back(first);
        degree_level(M, d - first, cur, out);
        cur.pop_back();
    }
}

std::vector<int> gpc_multi_indices(int M, int p) {
    std::vector<int> out, cur;
    for (int d = 0; d <= p; ++d) degree_level(M, d, cur, out);
    return out;
}

// A (n x n, row-major, symmetric) -> eigenvalues ev (descending) and
// eigenvectors as the columns of V (row-major n x n).  Returns false if the
// QL iteration did not converge.
bool sym_eig(int n, std::vector<double> A, std::vector<double>& ev, std::vector<double>& V) {
    auto a = [&](int i, int j) -> double& { return A[(size_t)i * n + j]; };
    std::vector<double> Q((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) Q[(size_t)i * n + i] = 1.0;
    std::vector<double> v(n), p(n), q(n);
    // Householder: zero column k below the sub-diagonal, A <- H A H, Q <- Q H.
    for (int k = 0; k + 2 < n; ++k) {
        double nrm = 0.0;
        for (int i = k + 1; i < n; ++i) nrm += a(i, k) * a(i, k);
        nrm = std::sqrt(nrm);
        if (nrm == 0.0) continue;
        double alpha = a(k + 1, k) > 0 ? -nrm : nrm;
        double vn = 0.0;
        for (int i = k + 1; i < n; ++i) {
            v[i] = a(i, k) - (i == k + 1 ? alpha : 0.0);
            vn += v[i] * v[i];
        }
        vn = std::sqrt(vn);
        if (vn == 0.0) continue;
        for (int i = k + 1; i < n; ++i) v[i] /= vn;
        // p = A v on the trailing block (rows/cols k..n-1 touched by H on k+1..)
        for (int i = k; i < n; ++i) {
            double s = 0.0;
            for (int j = k + 1; j < n; ++j) s += a(i, j) * v[j];
            p[i] = s;
        }
        double K = 0.0;
        for (int i = k + 1; i < n; ++i) K += v[i] * p[i];
        for (int i = k + 1; i < n; ++i) q[i] = p[i] - K * v[i];
        for (int i = k + 1; i < n; ++i)
            for (int j = k + 1; j < n; ++j) a(i, j) -= 2.0 * (v[i] * q[j] + q[i] * v[j]);
        a(k + 1, k) = alpha;
        a(k, k + 1) = alpha;
        for (int i = k + 2; i < n; ++i) a(i, k) = a(k, i) = 0.0;
        for (int r = 0; r < n; ++r) {
            double s = 0.0;
            for (int j = k + 1; j < n; ++j) s += Q[(size_t)r * n + j] * v[j];
            for (int j = k + 1; j < n; ++j) Q[(size_t)r * n + j] -= 2.0 * s * v[j];
        }
    }
    std::vector<double> d(n), e(n, 0.0);
    for (int i = 0; i < n; ++i) d[i] = a(i, i);
    for (int i = 0; i + 1 < n; ++i) e[i] = a(i + 1, i);
    // Implicit QL: e[i] couples i and i+1.  Each sweep chases a rotation from
    // the bottom of the unreduced block [l, m] up to l.
    const double eps = 2.220446049250313e-16;
    for (int l = 0; l < n; ++l) {
        for (int iter = 0;; ++iter) {
            int m = l;
            for (; m + 1 < n; ++m)
                if (std::fabs(e[m]) <= eps * (std::fabs(d[m]) + std::fabs(d[m + 1]))) break;
            if (m == l) break;
            if (iter > 200) return false;
            double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
            double r = std::hypot(g, 1.0);
            g = d[m] - d[l] + e[l] / (g + (g >= 0 ? r : -r));
            double s = 1.0, c = 1.0, pp = 0.0;
            bool early = false;
            for (int i = m - 1; i >= l; --i) {
                double f = s * e[i], b = c * e[i];
                r = std::hypot(f, g);
                e[i + 1] = r;
                if (r == 0.0) {
                    d[i + 1] -= pp;
                    e[m] = 0.0;
                    early = true;
                    break;
                }
                s = f / r;
                c = g / r;
                g = d[i + 1] - pp;
                r = (d[i] - g) * s + 2.0 * c * b;
                pp = s * r;
                d[i + 1] = g + pp;
                g = c * r - b;
                for (int row = 0; row < n; ++row) {
                    double* qr = &Q[(size_t)row * n];
                    double t1 = qr[i + 1];
                    qr[i + 1] = s * qr[i] + c * t1;
                    qr[i] = c * qr[i] - s * t1;
                }
            }
            if (early) continue;
            d[l] -= pp;
            e[l] = g;
            e[m] = 0.0;
        }
    }
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(), [&](int x, int y) { return d[x] > d[y]; });
    ev.resize(n);
    V.assign((size_t)n * n, 0.0);
    for (int c = 0; c < n; ++c) {
        ev[c] = d[order[c]];
        for (int r = 0; r < n; ++r) V[(size_t)r * n + c] = Q[(size_t)r * n + order[c]];
    }
    return true;
}

// Householder QR least squares: B (m x n, row-major, m >= n), D (m x r).
// Returns X (n x r) minimizing ||B X - D||_F column by column.
bool lstsq(int m, int n, int r, std::vector<double> B, std::vector<double> D,
           std::vector<double>& X) {
    if (m < n) return false;
    auto b = [&](int i, int j) -> double& { return B[(size_t)i * n + j]; };
    auto dd = [&](int i, int j) -> double& { return D[(size_t)i * r + j]; };
    std::vector<double> v(m);
    for (int k = 0; k < n; ++k) {
        double nrm = 0.0;
        for (int i = k; i < m; ++i) nrm += b(i, k) * b(i, k);
        nrm = std::sqrt(nrm);
        if (nrm == 0.0) return false;
        double alpha = b(k, k) > 0 ? -nrm : nrm;
        double vn = 0.0;
        for (int i = k; i < m; ++i) {
            v[i] = b(i, k) - (i == k ? alpha : 0.0);
            vn += v[i] * v[i];
        }
        if (vn == 0.0) continue;
        // apply H = I - 2 v v^T / (v^T v) to the remaining columns of B and to D
        for (int j = k; j < n; ++j) {
            double s = 0.0;
            for (int i = k; i < m; ++i) s += v[i] * b(i, j);
            s *= 2.0 / vn;
            for (int i = k; i < m; ++i) b(i, j) -= s * v[i];
        }
        for (int j = 0; j < r; ++j) {
            double s = 0.0;
            for (int i = k; i < m; ++i) s += v[i] * dd(i, j);
            s *= 2.0 / vn;
            for (int i = k; i < m; ++i) dd(i, j) -= s * v[i];
        }
    }
    X.assign((size_t)n * r, 0.0);
    for (int j = 0; j < r; ++j)
        for (int i = n - 1; i >= 0; --i) {
            double s = dd(i, j);
            for (int t = i + 1; t < n; ++t) s -= b(i, t) * X[(size_t)t * r + j];
            if (b(i, i) == 0.0) return false;
            X[(size_t)i * r + j] = s / b(i, i);
        }
    return true;
}

}  // namespace klecgc
