// Reference-element tables: modal basis (Sec. 2.4.1) and quadrature rules (Sec. 3.3).
//
// The basis phi_1..phi_15 is the paper's orthonormal basis on T^ = {x, y >= 0,
// x + y <= 1}.  Here each function is written in a factored form (products of
// low-degree polynomials in x and u = x + 2y - 1); gradients come from evaluating
// the same expressions on first-order dual numbers, so values and gradients cannot
// disagree.
#include "internal.h"

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <stdexcept>

namespace festung {

namespace {

struct Dual {
    double v, dx, dy;
};
inline Dual cst(double c) { return {c, 0.0, 0.0}; }
inline Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.dx + b.dx, a.dy + b.dy}; }
inline Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.dx - b.dx, a.dy - b.dy}; }
inline Dual operator*(Dual a, Dual b) {
    return {a.v * b.v, a.dx * b.v + a.v * b.dx, a.dy * b.v + a.v * b.dy};
}
inline Dual operator*(double c, Dual a) { return {c * a.v, c * a.dx, c * a.dy}; }
inline Dual operator+(Dual a, double c) { return {a.v + c, a.dx, a.dy}; }

// polynomial in x alone by Horner, coefficients from the highest degree down
Dual horner(Dual x, std::initializer_list<double> c) {
    Dual r = cst(0.0);
    for (double ci : c) r = r * x + ci;
    return r;
}

Dual basis_fn(int i, Dual x, Dual y) {
    const Dual u = x + 2.0 * y + (-1.0);                                      // x + 2y - 1
    const Dual q2 = x * x + 6.0 * (x * y) - 2.0 * x + 6.0 * (y * y) - 6.0 * y + 1.0;
    const Dual q3 = x * x + 10.0 * (x * y) - 2.0 * x + 10.0 * (y * y) - 10.0 * y + 1.0;
    switch (i) {
        case 0: return cst(std::sqrt(2.0));
        case 1: return 2.0 * (cst(1.0) - 3.0 * x);
        case 2: return (-2.0 * std::sqrt(3.0)) * u;
        case 3: return std::sqrt(6.0) * horner(x, {10.0, -8.0, 1.0});
        case 4: return std::sqrt(3.0) * (horner(x, {5.0, -4.0, -1.0}) + horner(y, {-15.0, 12.0, 0.0}));
        case 5: return (3.0 * std::sqrt(5.0)) *
                       (3.0 * (x * x) + 8.0 * (x * y) - 4.0 * x + 3.0 * (y * y) - 4.0 * y + 1.0);
        case 6: return (2.0 * std::sqrt(2.0)) * horner(x, {35.0, -45.0, 15.0, -1.0});
        case 7: return (2.0 * std::sqrt(6.0)) * (u * horner(x, {21.0, -12.0, 1.0}));
        case 8: return (2.0 * std::sqrt(10.0)) * (horner(x, {7.0, -1.0}) * q2);
        case 9: return (2.0 * std::sqrt(14.0)) * (u * q3);
        case 10: return std::sqrt(10.0) * horner(x, {126.0, -224.0, 126.0, -24.0, 1.0});
        case 11: return std::sqrt(30.0) * (u * horner(x, {84.0, -84.0, 21.0, -1.0}));
        case 12: return (5.0 * std::sqrt(2.0)) * (horner(x, {36.0, -16.0, 1.0}) * q2);
        case 13: return std::sqrt(70.0) * (horner(x, {9.0, -1.0}) * (u * q3));
        case 14: {
            // sum over the monomials x^a y^b of degree <= 4, coefficients c[a][b]
            const double c[5][5] = {{1.0, -20.0, 90.0, -140.0, 70.0},
                                    {-4.0, 60.0, -180.0, 140.0, 0.0},
                                    {6.0, -60.0, 90.0, 0.0, 0.0},
                                    {-4.0, 20.0, 0.0, 0.0, 0.0},
                                    {1.0, 0.0, 0.0, 0.0, 0.0}};
            Dual r = cst(0.0), xa = cst(1.0);
            for (int a = 0; a <= 4; ++a) {
                Dual yb = cst(1.0);
                for (int b = 0; b + a <= 4; ++b) {
                    r = r + c[a][b] * (xa * yb);
                    yb = yb * y;
                }
                xa = xa * x;
            }
            return (3.0 * std::sqrt(10.0)) * r;
        }
    }
    throw std::logic_error("basis index");
}

}  // namespace

int num_dofs(int p) { return (p + 1) * (p + 2) / 2; }

void basis_eval(int N, double x1, double x2, double *phi, double *d1, double *d2) {
    const Dual x{x1, 1.0, 0.0}, y{x2, 0.0, 1.0};
    for (int i = 0; i < N; ++i) {
        Dual r = basis_fn(i, x, y);
        if (phi) phi[i] = r.v;
        if (d1) d1[i] = r.dx;
        if (d2) d2[i] = r.dy;
    }
}

// ---------------------------------------------------------------------------
// Gauss rules from the three-term recurrences (Newton on bracketed roots)
// ---------------------------------------------------------------------------
namespace {

// Jacobi polynomial P_n^{(a,b)}(x) and its derivative
void jacobi(int n, double a, double b, double x, double *p, double *dp) {
    double p0 = 1.0, p1 = 0.5 * (a - b + (a + b + 2.0) * x);
    if (n == 0) {
        *p = 1.0;
        *dp = 0.0;
        return;
    }
    for (int k = 2; k <= n; ++k) {
        const double c = 2.0 * k + a + b;
        const double a1 = 2.0 * k * (k + a + b) * (c - 2.0);
        const double a2 = (c - 1.0) * (c * (c - 2.0) * x + a * a - b * b);
        const double a3 = 2.0 * (k + a - 1.0) * (k + b - 1.0) * c;
        const double p2 = (a2 * p1 - a3 * p0) / a1;
        p0 = p1;
        p1 = p2;
    }
    *p = p1;
    // (2n + a + b)(1 - x^2) P_n' = n[(a - b) - (2n + a + b) x] P_n + 2(n + a)(n + b) P_{n-1}
    const double c = 2.0 * n + a + b;
    *dp = (n * ((a - b) - c * x) * p1 + 2.0 * (n + a) * (n + b) * p0) / (c * (1.0 - x * x));
}

// roots of P_n^{(a,b)} on (-1, 1), ascending, with Gauss-Jacobi weights
void gauss_jacobi(int n, double a, double b, std::vector<double> &x, std::vector<double> &w) {
    x.clear();
    w.clear();
    const int M = 4000;
    double xl = -1.0 + 1e-14, pl, dpl;
    jacobi(n, a, b, xl, &pl, &dpl);
    for (int s = 1; s <= M && (int)x.size() < n; ++s) {
        double xr = -1.0 + 2.0 * s / M;
        if (s == M) xr = 1.0 - 1e-14;
        double pr, dpr;
        jacobi(n, a, b, xr, &pr, &dpr);
        if (pr == 0.0) {
            x.push_back(xr);  // grid point is a root
        } else if (pl != 0.0 && (pl < 0) != (pr < 0)) {
            // bisect the bracket down to 1e-6, then Newton to machine precision
            double lo = xl, hi = xr, plo = pl;
            while (hi - lo > 1e-6) {
                const double m = 0.5 * (lo + hi);
                double pm, dm;
                jacobi(n, a, b, m, &pm, &dm);
                if (pm == 0.0) { lo = hi = m; break; }
                if ((pm < 0) == (plo < 0)) { lo = m; plo = pm; } else { hi = m; }
            }
            double r = 0.5 * (lo + hi);
            for (int it = 0; it < 60; ++it) {
                double pv, dv;
                jacobi(n, a, b, r, &pv, &dv);
                if (pv == 0.0) break;
                const double dx = pv / dv;
                r -= dx;
                if (std::fabs(dx) <= 1e-17 * (1.0 + std::fabs(r))) break;
            }
            x.push_back(r);
        }
        xl = xr;
        pl = pr;
    }
    if ((int)x.size() != n) throw std::runtime_error("gauss_jacobi: root count");
    // w_i = 2^{a+b+1} Gamma(n+a+1) Gamma(n+b+1) / (Gamma(n+a+b+1) n!) / ((1 - x_i^2) P_n'(x_i)^2)
    const double g = std::exp(std::lgamma(n + a + 1.0) + std::lgamma(n + b + 1.0) -
                              std::lgamma(n + a + b + 1.0) - std::lgamma(n + 1.0)) *
                     std::pow(2.0, a + b + 1.0);
    for (int i = 0; i < n; ++i) {
        double pv, dv;
        jacobi(n, a, b, x[i], &pv, &dv);
        w.push_back(g / ((1.0 - x[i] * x[i]) * dv * dv));
    }
}

void push_orbit3(Rule2D &R, double a, double w) {
    const double b = 1.0 - 2.0 * a;
    const double pts[3][2] = {{a, a}, {b, a}, {a, b}};
    for (auto &p : pts) {
        R.x1.push_back(p[0]);
        R.x2.push_back(p[1]);
        R.w.push_back(w);
    }
}

void push_orbit6(Rule2D &R, double a, double b, double w) {
    const double c = 1.0 - a - b;
    const double pts[6][2] = {{a, b}, {b, a}, {a, c}, {c, a}, {b, c}, {c, b}};
    for (auto &p : pts) {
        R.x1.push_back(p[0]);
        R.x2.push_back(p[1]);
        R.w.push_back(w);
    }
}

}  // namespace

Rule1D gauss_legendre01(int n) {
    Rule1D R;
    std::vector<double> x, w;
    gauss_jacobi(n, 0.0, 0.0, x, w);
    for (int i = 0; i < n; ++i) {
        R.s.push_back(0.5 * (x[i] + 1.0));
        R.w.push_back(0.5 * w[i]);
    }
    // enforce the exact mirror symmetry s_r + s_{n-1-r} = 1 used for neighbour traces
    for (int i = 0; i < n / 2; ++i) {
        const double s = 0.5 * (R.s[i] + (1.0 - R.s[n - 1 - i]));
        const double ww = 0.5 * (R.w[i] + R.w[n - 1 - i]);
        R.s[i] = s;
        R.s[n - 1 - i] = 1.0 - s;
        R.w[i] = R.w[n - 1 - i] = ww;
    }
    if (n % 2 == 1) R.s[n / 2] = 0.5;
    return R;
}

int edge_points_for_degree(int q) { return std::max(1, (q + 2) / 2); }

Rule2D triangle_rule(int q) {
    Rule2D R;
    if (q < 1) q = 1;
    if (q == 1) {
        R.x1 = {1.0 / 3.0};
        R.x2 = {1.0 / 3.0};
        R.w = {0.5};
    } else if (q == 2) {
        R.x1 = {1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0};
        R.x2 = {1.0 / 6.0, 1.0 / 6.0, 2.0 / 3.0};
        R.w = {1.0 / 6.0, 1.0 / 6.0, 1.0 / 6.0};
    } else if (q == 3 || q == 4) {
        // degree 4, two 3-point orbits (Strang-Fix/Cowper constants as printed, Sec. 4)
        push_orbit3(R, 0.445948490915965, 0.111690794839005);
        push_orbit3(R, 0.091576213509771, 0.054975871827661);
    } else if (q == 5) {
        const double r = std::sqrt(15.0);
        R.x1 = {1.0 / 3.0};
        R.x2 = {1.0 / 3.0};
        R.w = {9.0 / 80.0};
        push_orbit3(R, (6.0 - r) / 21.0, (155.0 - r) / 2400.0);
        push_orbit3(R, (6.0 + r) / 21.0, (155.0 + r) / 2400.0);
    } else if (q == 6) {
        push_orbit3(R, 0.063089014491502, 0.025422453185103);
        push_orbit3(R, 0.249286745170910, 0.058393137863189);
        push_orbit6(R, 0.053145049844816, 0.310352451033785, 0.041425537809187);
    } else {
        // collapsed square: x1 = u, x2 = (1 - u) v; Gauss-Jacobi(1, 0) in u, Gauss-Legendre in v
        const int n = edge_points_for_degree(q);
        std::vector<double> t, wt;
        gauss_jacobi(n, 1.0, 0.0, t, wt);
        Rule1D v = gauss_legendre01(n);
        for (int i = 0; i < n; ++i) {
            const double u = 0.5 * (t[i] + 1.0), wu = 0.25 * wt[i];
            for (int j = 0; j < n; ++j) {
                R.x1.push_back(u);
                R.x2.push_back((1.0 - u) * v.s[j]);
                R.w.push_back(wu * v.w[j]);
            }
        }
    }
    return R;
}

void build_tables(int p, int qT, HostTables &T) {
    const int N = num_dofs(p);
    const int qE = std::max(qT, 2 * p + 1);
    Rule2D tri = triangle_rule(qT);
    Rule1D edg = gauss_legendre01(edge_points_for_degree(qE));
    const int R2 = (int)tri.w.size(), R1 = (int)edg.w.size();
    T.p = p;
    T.N = N;
    T.R2 = R2;
    T.R1 = R1;
    T.qT = qT;
    T.tri = tri;
    T.edge = edg;
    T.phiQ.assign(R2 * N, 0.0);
    T.wphiQ.assign(R2 * N, 0.0);
    T.gw1.assign(R2 * N, 0.0);
    T.gw2.assign(R2 * N, 0.0);
    std::vector<double> ph(N), g1(N), g2(N);
    for (int r = 0; r < R2; ++r) {
        basis_eval(N, tri.x1[r], tri.x2[r], ph.data(), g1.data(), g2.data());
        for (int j = 0; j < N; ++j) {
            T.phiQ[r * N + j] = ph[j];
            T.wphiQ[r * N + j] = tri.w[r] * ph[j];
            T.gw1[r * N + j] = tri.w[r] * g1[j];
            T.gw2[r * N + j] = tri.w[r] * g2[j];
        }
    }
    // H^[i][j][m] = int d_m phi_i phi_j (exact: degree 2p - 1 <= qT)
    T.H1.assign(N * N, 0.0);
    T.H2.assign(N * N, 0.0);
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) {
            double s1 = 0.0, s2 = 0.0;
            for (int r = 0; r < R2; ++r) {
                s1 += T.gw1[r * N + i] * T.phiQ[r * N + j];
                s2 += T.gw2[r * N + i] * T.phiQ[r * N + j];
            }
            T.H1[i * N + j] = s1;
            T.H2[i * N + j] = s2;
        }
    // d_m phi_i has degree deg(i) - 1 and the basis is orthonormal and ordered by degree,
    // so H^[i][j] vanishes for every phi_j of degree >= deg(i); the kernels skip these
    // entries, so they are checked here and stored as exact zeros
    auto degree = [](int i) { return i < 1 ? 0 : i < 3 ? 1 : i < 6 ? 2 : i < 10 ? 3 : 4; };
    for (int i = 0; i < N; ++i)
        for (int j = degree(i) * (degree(i) + 1) / 2; j < N; ++j) {
            if (std::abs(T.H1[i * N + j]) > 1e-12 || std::abs(T.H2[i * N + j]) > 1e-12)
                throw std::runtime_error("H^ is not strictly lower block-triangular by degree");
            T.H1[i * N + j] = 0.0;
            T.H2[i * N + j] = 0.0;
        }
    // edge traces: phi_j(gamma_n(s_r)), gamma_1(s) = (1-s, s), gamma_2 = (0, 1-s), gamma_3 = (s, 0)
    T.phiE.assign(3 * R1 * N, 0.0);
    T.wphiE.assign(3 * R1 * N, 0.0);
    for (int n = 0; n < 3; ++n)
        for (int r = 0; r < R1; ++r) {
            const double s = edg.s[r];
            double x1 = 0, x2 = 0;
            if (n == 0) { x1 = 1.0 - s; x2 = s; }
            if (n == 1) { x1 = 0.0; x2 = 1.0 - s; }
            if (n == 2) { x1 = s; x2 = 0.0; }
            basis_eval(N, x1, x2, ph.data(), nullptr, nullptr);
            for (int j = 0; j < N; ++j) {
                T.phiE[(n * R1 + r) * N + j] = ph[j];
                T.wphiE[(n * R1 + r) * N + j] = edg.w[r] * ph[j];
            }
        }
}

float round_to_bf16(double v) {
    // keep the top 16 bits of the IEEE single, rounding the low 16 away (ties to even)
    const float f = (float)v;
    uint32_t u;
    std::memcpy(&u, &f, sizeof(u));
    if ((u & 0x7f800000u) == 0x7f800000u) return f;  // Inf or NaN: unchanged
    const uint32_t lsb = (u >> 16) & 1u;
    u = (u + 0x7fffu + lsb) & 0xffff0000u;
    float r;
    std::memcpy(&r, &u, sizeof(r));
    return r;
}

}  // namespace festung
