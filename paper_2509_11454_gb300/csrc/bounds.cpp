// Sample-size bound of Algorithm 1 (host code; four scalars in, one integer
// out).  Follows Propositions 2-3 for rho^ and v^, x^ as in Algorithm 1, and
// Theorem 1 for l with the confidence split of Proposition 4
// (ln(4 d^ rho^ / (x delta))).
#include <cmath>
#include <cstdint>
#include <vector>

#include "internal.h"

namespace percis {

int64_t ell1_default(double eps, double delta) {
    const double v = std::ceil(std::log(1.0 / delta) / eps);
    return v > 1000.0 ? (int64_t)v : 1000;
}

namespace {

// Theorem 1's objective: d^2 ln(4 d rho / (x delta)) / (g(x) h(eps d / g(x))),
// g(x) = x (d - x), h(y) = (1 + y) ln(1 + y) - y.
double objective(double x, double eps, double delta, double dhat, double rho_h) {
    const double gx = x * (dhat - x);
    const double y = eps * dhat / gx;
    const double hy = (1.0 + y) * std::log(1.0 + y) - y;
    return dhat * dhat * std::log(4.0 * dhat * rho_h / (x * delta)) / (gx * hy);
}

// sup over (0, x^]: the paper gives no method.  Maximum over the geometric
// grid x_k = x^ 10^(-12 + 12 k / 4096), k = 0..4096, then 100 golden-section
// steps on [x_{k*-1}, x_{k*+1}] around the best grid point.
constexpr int kGrid = 4096;

// the grid factors 10^(-12 + 12 k / 4096), computed once (the same values each call)
const double *grid_factors() {
    static const std::vector<double> f = [] {
        std::vector<double> v(kGrid + 1);
        for (int k = 0; k <= kGrid; ++k) v[k] = std::pow(10.0, -12.0 + 12.0 * k / kGrid);
        return v;
    }();
    return f.data();
}

double sup_objective(double eps, double delta, double dhat, double rho_h, double xh) {
    const int K = kGrid;
    const double *gf = grid_factors();
    double best = -INFINITY;
    int best_k = 0;
    for (int k = 0; k <= K; ++k) {
        const double xk = xh * gf[k];
        const double fv = objective(xk, eps, delta, dhat, rho_h);
        if (fv > best) {
            best = fv;
            best_k = k;
        }
    }
    const int klo = best_k - 1 < 0 ? 0 : best_k - 1;
    const int khi = best_k + 1 > K ? K : best_k + 1;
    double a = xh * gf[klo];
    double b = xh * gf[khi];
    const double gr = (std::sqrt(5.0) - 1.0) / 2.0;
    double c1 = b - gr * (b - a);
    double c2 = a + gr * (b - a);
    double f1 = objective(c1, eps, delta, dhat, rho_h);
    double f2 = objective(c2, eps, delta, dhat, rho_h);
    for (int it = 0; it < 100; ++it) {
        if (f1 > best) best = f1;
        if (f2 > best) best = f2;
        if (f1 >= f2) {
            const double nb = c2, nc2 = c1, nf2 = f1;
            b = nb;
            c2 = nc2;
            f2 = nf2;
            c1 = b - gr * (b - a);
            f1 = objective(c1, eps, delta, dhat, rho_h);
        } else {
            const double na = c1, nc1 = c2, nf1 = f2;
            a = na;
            c1 = nc1;
            f1 = nf1;
            c2 = a + gr * (b - a);
            f2 = objective(c2, eps, delta, dhat, rho_h);
        }
    }
    if (f1 > best) best = f1;
    if (f2 > best) best = f2;
    return best;
}

}  // namespace

Bounds compute_bounds(double eps, double delta, double dhat, int64_t D, int64_t ell1, int64_t sum_ilen,
                      int64_t sum_ilen2, double p1_max, int data_independent) {
    Bounds b{};
    if (data_independent) {
        // PercIS-DI (Section IV-B): rho^ = D, v^ = d^2 / 4, no first phase.
        b.rho_hat = (double)D;
        b.v_hat = dhat * dhat / 4.0;
    } else {
        const double l1 = (double)ell1;
        b.rho_tilde = (double)sum_ilen / l1;
        // Lambda = (1/(l(l-1))) sum_{i<j} (a_i - a_j)^2 = (l sum a^2 - (sum a)^2) / (l(l-1)), exact in integers
        const int64_t num = ell1 * sum_ilen2 - sum_ilen * sum_ilen;
        b.Lambda = (double)num / ((double)ell1 * (double)(ell1 - 1));
        const double lg8 = std::log(8.0 / delta);
        b.rho_hat = b.rho_tilde + std::sqrt(2.0 * b.Lambda * lg8 / l1) + 7.0 * (double)D * lg8 / (3.0 * (l1 - 1.0));
        const double lg4 = std::log(4.0 / delta);
        b.v_hat = dhat * dhat * (p1_max + std::sqrt(2.0 * p1_max * lg4 / l1) + lg4 / (3.0 * l1));
    }
    const double q = dhat * dhat / 4.0;
    b.x_hat = dhat / 2.0 - std::sqrt(q - (q < b.v_hat ? q : b.v_hat));
    b.ell = (int64_t)std::ceil(sup_objective(eps, delta, dhat, b.rho_hat, b.x_hat));
    return b;
}

}  // namespace percis
