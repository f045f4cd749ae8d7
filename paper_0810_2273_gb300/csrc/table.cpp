// Host FP64 construction of the vdW-DF kernel table (paper section 2: phi
// "calculated according to formula (14) in Ref. [Dion et al.], which requires a
// double integration"; section 7: table limits and divisions fixed by
// refinement) and of its bicubic B-spline coefficients.
//
// Quadrature of Dion eq. (14):
//   phi(d1, d2) = 2/pi^2 int_0^inf a^2 da int_0^inf b^2 db W(a,b) T(nu1(a), nu1(b), nu2(a), nu2(b))
//   W(a,b) = 2 [j0(a) u(b) + j0(b) u(a) - 3 u(a) u(b)],  j0(a) = sin a / a,
//            u(a) = (sin a - a cos a)/a^3   (Dion's printed W, bracket collected),
//   T(w,x,y,z) = 1/2 [1/(w+x) + 1/(y+z)] [1/((w+y)(x+z)) + 1/((w+z)(y+x))],
//   nu_d(y) = y^2 / (2 h(y/d)),  h(x) = 1 - exp(-4 pi x^2 / 9).
// The integrand is symmetric in (a, b), so the tensor grid is folded to
// i <= j.  Both axes share one node set on (0, A], A = (M + 1/2) pi:
//   octave panels 2^-p (p < 24) below 1, then panels of pi/4 up to 4 pi,
//   pi/2 up to 16 pi and pi beyond, with n GL points each.
// The part a > A (and b > A) is added by integration by parts: writing the
// a-integrand for fixed b as S(a) sin a + C(a) cos a with smooth S, C,
//   int_A^inf = sigma [-S'(A) - C(A) + S'''(A) + C''(A)] + ...,  sigma = sin A,
// since cos A = 0; derivatives of S and C by central differences.  The corner
// a, b > A is of order A^-8 and dropped.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "table.h"

namespace vdwdf {

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kGamma = 4.0 * kPi / 9.0;

// Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on P_n (Golub-Welsch
// would also do; the recurrence is enough for n <= 32).
void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (p0 - z * p1) / (1.0 - z * z);
            double step = p1 / dp;
            z -= step;
            if (std::fabs(step) < 1e-16) break;
        }
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (p0 - z * p1) / (1.0 - z * z);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

struct Quad {
    int M;      // A = (M + 1/2) pi
    int n_log;  // points per octave panel
    int n_osc;  // points per panel above 1
};

Quad quad_for_level(int level) {
    switch (level) {
        case 0: return {15, 5, 6};
        case 2: return {127, 8, 10};
        default: return {63, 7, 8};
    }
}

void build_nodes(const Quad &q, std::vector<double> &a, std::vector<double> &w) {
    std::vector<double> gx, gw;
    a.clear();
    w.clear();
    auto panel = [&](double lo, double hi, int n) {
        gauss_legendre(n, gx, gw);
        for (int i = 0; i < n; ++i) {
            a.push_back(0.5 * (lo + hi) + 0.5 * (hi - lo) * gx[i]);
            w.push_back(0.5 * (hi - lo) * gw[i]);
        }
    };
    for (int p = 23; p >= 0; --p) panel(std::ldexp(1.0, -p - 1), std::ldexp(1.0, -p), q.n_log);
    // boundaries at integer multiples of pi/4: quarter counts 2 (pi/2) .. 4M + 2 (A)
    const int qA = 4 * q.M + 2;
    double lo = 1.0;
    for (int qb = 2; qb <= qA;) {
        const double hi = qb * (kPi / 4.0);
        panel(lo, hi, q.n_osc);
        lo = hi;
        const int step = (qb < 16) ? 1 : ((qb < 64) ? 2 : 4);
        qb = (qb + step > qA && qb < qA) ? qA : qb + step;
    }
}

inline double j0(double a) { return std::sin(a) / a; }

inline double ufun(double a) {
    if (a < 0.1) {
        // j1(a)/a = 1/3 - a^2/30 + a^4/840 - a^6/45360 + a^8/3991680
        double a2 = a * a;
        return 1.0 / 3.0 + a2 * (-1.0 / 30.0 + a2 * (1.0 / 840.0 + a2 * (-1.0 / 45360.0 + a2 / 3991680.0)));
    }
    return (std::sin(a) - a * std::cos(a)) / (a * a * a);
}

inline double nu(double y, double d) {
    double x = y / d;
    return 0.5 * y * y / (-std::expm1(-kGamma * x * x));
}

inline double Tfun(double w, double x, double y, double z) {
    return 0.5 * (1.0 / (w + x) + 1.0 / (y + z)) * (1.0 / ((w + y) * (x + z)) + 1.0 / ((w + z) * (y + x)));
}

struct Integrator {
    Quad q;
    std::vector<double> a, w;      // nodes, weights
    std::vector<double> WW;        // w_i w_j a_i^2 a_j^2 W(a_i, a_j), upper triangle used
    std::vector<double> ub, kb;    // u(b), j0(b) - 3 u(b) at nodes
    double A, sigma;

    explicit Integrator(const Quad &qq) : q(qq) {
        build_nodes(q, a, w);
        const int N = static_cast<int>(a.size());
        std::vector<double> s(N), u(N);
        for (int i = 0; i < N; ++i) {
            s[i] = j0(a[i]);
            u[i] = ufun(a[i]);
        }
        WW.assign(static_cast<size_t>(N) * N, 0.0);
        for (int i = 0; i < N; ++i)
            for (int j = i; j < N; ++j) {
                double Wij = 2.0 * (s[i] * u[j] + s[j] * u[i] - 3.0 * u[i] * u[j]);
                double v = w[i] * w[j] * a[i] * a[i] * a[j] * a[j] * Wij;
                WW[static_cast<size_t>(i) * N + j] = (i == j) ? v : 2.0 * v;
            }
        ub = u;
        kb.resize(N);
        for (int i = 0; i < N; ++i) kb[i] = s[i] - 3.0 * u[i];
        A = (q.M + 0.5) * kPi;
        sigma = (q.M % 2 == 0) ? 1.0 : -1.0;  // sin((M + 1/2) pi)
    }

    // phi(d1, d2); scratch of 2N doubles.
    double phi(double d1, double d2, double *scratch) const {
        const int N = static_cast<int>(a.size());
        double *n1 = scratch, *n2 = scratch + N;
        for (int i = 0; i < N; ++i) {
            n1[i] = nu(a[i], d1);
            n2[i] = nu(a[i], d2);
        }
        double sum = 0.0;
        for (int i = 0; i < N; ++i) {
            const double wi = n1[i], yi = n2[i];
            const double *row = &WW[static_cast<size_t>(i) * N];
            double acc = 0.0;
            for (int j = i; j < N; ++j) {
                const double xj = n1[j], zj = n2[j];
                acc += row[j] * Tfun(wi, xj, yi, zj);
            }
            sum += acc;
        }
        // tail a > A at every b node (twice: the b > A tail is its mirror)
        double tail = 0.0;
        const double e = 0.5;
        const double nuA1[5] = {nu(A - 2 * e, d1), nu(A - e, d1), nu(A, d1), nu(A + e, d1), nu(A + 2 * e, d1)};
        const double nuA2[5] = {nu(A - 2 * e, d2), nu(A - e, d2), nu(A, d2), nu(A + e, d2), nu(A + 2 * e, d2)};
        for (int j = 0; j < N; ++j) {
            const double b = a[j], xj = n1[j], zj = n2[j];
            double S[5], Cc[5];
            for (int t = 0; t < 5; ++t) {
                const double at = A + (t - 2) * e;
                const double T = Tfun(nuA1[t], xj, nuA2[t], zj);
                S[t] = 2.0 * b * b * T * (at * ub[j] + kb[j] / at);
                Cc[t] = -2.0 * b * b * T * kb[j];
            }
            const double S1 = (S[3] - S[1]) / (2 * e);
            const double S3 = (S[4] - 2 * S[3] + 2 * S[1] - S[0]) / (2 * e * e * e);
            const double C2 = (Cc[3] - 2 * Cc[2] + Cc[1]) / (e * e);
            tail += w[j] * sigma * (-S1 - Cc[2] + S3 + C2);
        }
        return 2.0 / (kPi * kPi) * (sum + 2.0 * tail);
    }
};

// 1-D interpolating cubic B-spline coefficients on a uniform grid of N nodes with
// zero slope at node 0 and zero curvature at node N-1.  Input f (stride fs);
// output c_{-1} .. c_N (N + 2 values, stride cs).
void bspline_1d(int N, const double *f, int fs, double *c, int cs, std::vector<double> &cp,
                std::vector<double> &dp) {
    // unknowns c_0 .. c_{N-2}; c_{N-1} = f_{N-1}; rows:
    //   4 c_0 + 2 c_1 = 6 f_0
    //   c_{i-1} + 4 c_i + c_{i+1} = 6 f_i         (i = 1 .. N-2, c_{N-1} on the right)
    const int n = N - 1;
    cp.assign(n, 0.0);
    dp.assign(n, 0.0);
    const double cl = f[fs * (N - 1)];
    for (int i = 0; i < n; ++i) {
        double sub = (i == 0) ? 0.0 : 1.0;
        double diag = 4.0;
        double sup = (i == 0) ? 2.0 : ((i == n - 1) ? 0.0 : 1.0);
        double rhs = 6.0 * f[fs * i] - ((i == n - 1 && i > 0) ? cl : 0.0);
        if (i == 0 && n == 1) {  // N == 2: 4 c0 + 2 c1 = 6 f0 with c1 known
            sup = 0.0;
            rhs = 6.0 * f[0] - 2.0 * cl;
        }
        if (i == 0) {
            cp[0] = sup / diag;
            dp[0] = rhs / diag;
        } else {
            double den = diag - sub * cp[i - 1];
            cp[i] = sup / den;
            dp[i] = (rhs - sub * dp[i - 1]) / den;
        }
    }
    std::vector<double> x(N);
    x[N - 1] = cl;
    x[n - 1] = dp[n - 1];
    for (int i = n - 2; i >= 0; --i) x[i] = dp[i] - cp[i] * x[i + 1];
    // ghosts: c_{-1} = c_1 (zero slope), c_N = 2 c_{N-1} - c_{N-2} (zero curvature)
    c[0] = x[1];
    for (int i = 0; i < N; ++i) c[cs * (i + 1)] = x[i];
    c[cs * (N + 1)] = 2.0 * x[N - 1] - x[N - 2];
}

}  // namespace

int quadrature_node_count(int level) {
    std::vector<double> a, w;
    build_nodes(quad_for_level(level), a, w);
    return static_cast<int>(a.size());
}

int build_phi_nodes(int nD, double Dmax, int ndelta, int level, double *nodes) {
    Integrator *I = nullptr;
    try {
        I = new Integrator(quad_for_level(level));
    } catch (const std::bad_alloc &) {
        return -1;
    }
    const int N = static_cast<int>(I->a.size());
    const int npts = (nD - 1) * ndelta;
    int fail = 0;
#pragma omp parallel
    {
        std::vector<double> scratch;
        try {
            scratch.resize(2 * static_cast<size_t>(N));
        } catch (const std::bad_alloc &) {
#pragma omp atomic write
            fail = 1;
        }
        if (!scratch.empty()) {
#pragma omp for schedule(dynamic, 4)
            for (int p = 0; p < npts; ++p) {
                const int k = 1 + p / ndelta, l = p % ndelta;
                const double D = Dmax * k / (nD - 1), dl = static_cast<double>(l) / ndelta;
                nodes[static_cast<size_t>(k) * ndelta + l] = I->phi(D * (1.0 + dl), D * (1.0 - dl), scratch.data());
            }
        }
    }
    delete I;
    if (fail) return -1;
    // D = 0: eq. (14) diverges like -(2/pi) ln D; take the even quadratic through D_1, D_2.
    for (int l = 0; l < ndelta; ++l)
        nodes[l] = (4.0 * nodes[ndelta + l] - nodes[2 * static_cast<size_t>(ndelta) + l]) / 3.0;
    return 0;
}

void rho_coefficients(int nD, double Dmax, int nd, const double *nodes, double *coef) {
    // rho(delta_l) = phi(Dmax, delta_l) / phi17(Dmax, delta_l).  Past Dmax the kernel is
    // eq. (17) times g = rho(delta*) + (1 - rho(0)) (1 - (Dmax/D)^2) with the cubic
    // spline of rho, so that it is continuous with the table at Dmax.
    const double C = 12.0 * std::pow(4.0 * kPi / 9.0, 3);
    std::vector<double> r(nd), cp, dp;
    for (int l = 0; l < nd; ++l) {
        const double dl = static_cast<double>(l) / nd;
        const double d1 = Dmax * (1.0 + dl), d2 = Dmax * (1.0 - dl);
        r[l] = nodes[static_cast<size_t>(nD - 1) * nd + l] / (-C / (d1 * d1 * d2 * d2 * (d1 * d1 + d2 * d2)));
    }
    bspline_1d(nd, r.data(), 1, coef, 1, cp, dp);
}

void spline_coefficients(int nD, int nd, const double *nodes, double *coef) {
    // coef: (nD + 2) x (nd + 2), D outer.  First along D for every delta node, then
    // along delta for every (ghost-extended) D row.
    const int S = nd + 2;
    std::vector<double> tmp(static_cast<size_t>(nD + 2) * nd);
    std::vector<double> cp, dp;
    for (int l = 0; l < nd; ++l) bspline_1d(nD, nodes + l, nd, tmp.data() + l, nd, cp, dp);
    for (int k = 0; k < nD + 2; ++k)
        bspline_1d(nd, tmp.data() + static_cast<size_t>(k) * nd, 1, coef + static_cast<size_t>(k) * S, 1, cp, dp);
}

}  // namespace vdwdf
