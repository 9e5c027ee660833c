// Host-side check of the library's reference tables (compiled by tests/test_tables_cpu.py).
// Prints, per rule, the worst relative error over all monomials up to its degree, and
// for the basis the worst deviation of the Gram matrix from the identity.
#include <cmath>
#include <cstdio>
#include <vector>

#include "internal.h"

using namespace festung;

static double fact(int n) { return std::tgamma(n + 1.0); }

int main() {
    for (int q = 1; q <= 10; ++q) {
        Rule2D R = triangle_rule(q);
        const int eff = (q == 3) ? 4 : q;
        double worst = 0.0;
        for (int a = 0; a <= eff; ++a)
            for (int b = 0; a + b <= eff; ++b) {
                const double ex = fact(a) * fact(b) / fact(a + b + 2);
                double s = 0.0;
                for (size_t r = 0; r < R.w.size(); ++r) s += R.w[r] * std::pow(R.x1[r], a) * std::pow(R.x2[r], b);
                worst = std::fmax(worst, std::fabs(s - ex) / ex);
            }
        double minw = 1e300, minx = 1e300;
        for (size_t r = 0; r < R.w.size(); ++r) {
            minw = std::fmin(minw, R.w[r]);
            minx = std::fmin(minx, std::fmin(std::fmin(R.x1[r], R.x2[r]), 1.0 - R.x1[r] - R.x2[r]));
        }
        std::printf("tri %d %zu %.3e %.3e %.3e\n", q, R.w.size(), worst, minw, minx);
    }
    for (int n = 1; n <= 9; ++n) {
        Rule1D G = gauss_legendre01(n);
        double worst = 0.0, sym = 0.0;
        for (int k = 0; k < 2 * n; ++k) {
            double s = 0.0;
            for (int r = 0; r < n; ++r) s += G.w[r] * std::pow(G.s[r], k);
            worst = std::fmax(worst, std::fabs(s - 1.0 / (k + 1)) * (k + 1));
        }
        for (int r = 0; r < n; ++r) sym = std::fmax(sym, std::fabs(G.s[r] + G.s[n - 1 - r] - 1.0));
        std::printf("gauss %d %.3e %.3e\n", n, worst, sym);
    }
    // orthonormality with the degree-10 rule; gradient vs central differences
    Rule2D R = triangle_rule(10);
    std::vector<double> P(R.w.size() * 15);
    for (size_t r = 0; r < R.w.size(); ++r) basis_eval(15, R.x1[r], R.x2[r], &P[r * 15], nullptr, nullptr);
    double gram = 0.0;
    for (int i = 0; i < 15; ++i)
        for (int j = 0; j < 15; ++j) {
            double s = 0.0;
            for (size_t r = 0; r < R.w.size(); ++r) s += R.w[r] * P[r * 15 + i] * P[r * 15 + j];
            gram = std::fmax(gram, std::fabs(s - (i == j ? 1.0 : 0.0)));
        }
    double gerr = 0.0;
    const double h = 1e-6;
    for (int t = 0; t < 20; ++t) {
        const double x = 0.05 + 0.04 * t, y = 0.03 + 0.02 * (t % 7);
        double v[15], d1[15], d2[15], vp[15], vm[15];
        basis_eval(15, x, y, v, d1, d2);
        basis_eval(15, x + h, y, vp, nullptr, nullptr);
        basis_eval(15, x - h, y, vm, nullptr, nullptr);
        for (int i = 0; i < 15; ++i) gerr = std::fmax(gerr, std::fabs((vp[i] - vm[i]) / (2 * h) - d1[i]) / (1 + std::fabs(d1[i])));
        basis_eval(15, x, y + h, vp, nullptr, nullptr);
        basis_eval(15, x, y - h, vm, nullptr, nullptr);
        for (int i = 0; i < 15; ++i) gerr = std::fmax(gerr, std::fabs((vp[i] - vm[i]) / (2 * h) - d2[i]) / (1 + std::fabs(d2[i])));
    }
    double v0[15];
    basis_eval(15, 0.0, 0.0, v0, nullptr, nullptr);
    std::printf("basis %.3e %.3e", gram, gerr);
    for (int i = 0; i < 15; ++i) std::printf(" %d", v0[i] > 0 ? 1 : -1);
    std::printf("\n");
    return 0;
}
