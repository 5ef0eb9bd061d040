// Host numerics of klecgc_setup (offline part of Algorithm 3).
//
//  - KL eigenpairs of sigma^2 exp(-|x-y|/ell) on [0,1]: on the centred interval
//    [-1/2, 1/2] with c = 1/ell the eigenvalues are 2 c sigma^2 / (w^2 + c^2),
//    w the roots of c - w tan(w/2) = 0 (cosine modes) and w + c tan(w/2) = 0
//    (sine modes), one root per half period; found here by bisection.
//  - Total-degree multi-indices of the Hermite gPC basis (eq. complete),
//    ordered by degree, then decreasing lexicographically.
// The snapshot eigenproblem and the least-squares fit run on the device
// (k_offline.cu).
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

}  // namespace klecgc
