/*
 * oracle.c -- plain, slow, FP64 CPU oracle for the vdW-DF nonlocal correlation
 * hot path of JuNoLo (Lazic et al., arXiv 0810.2273).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library (paper_0810_2273_gb300/)
 * may include, link, load or call this file.  Only tests/, the smoke() check in
 * __graft_entry__.py and the cpu_baseline / reference arm of bench.py use it.
 * It shares no code, header, table or constant generator with the CUDA path.
 *
 * What it computes (paper section 2, eqs. (1)-(2)):
 *     E_c^nl = 1/2 sum_i sum_j n_i phi(q0_i r_ij, q0_j r_ij) n_j  dV^2
 * over grid points with n >= n_cut (section 3, density trimming), including
 * periodic images (section 3, "the charge density from the 0th cell must be
 * repeated in space"), with the kernel phi of Dion et al. (PRL 92, 246401,
 * eq. 14) tabulated in (D, delta) (section 2: "redefined to depend on two
 * quantities, D >= 0 and 0 <= delta < 1") and its large-D asymptote (Dion
 * eq. 17, section 2).  It also gives the adjoint potential v = dE/dn / dV.
 *
 * Every function below is written straight from its definition, with no
 * blocking, fusion or reordering beyond what the definition states.  Where the
 * paper is silent the reading used is stated at the function.
 *
 * Parity status of each function (pins live in tests/test_oracle_*.py):
 *   orc_W, orc_phi, orc_phi_table  pinned: symmetry, zero integral, large-D
 *                                   asymptote, small-D logarithm, printed-W
 *                                   formula at high precision
 *   kernel_pair (orc_kernel_many)   pinned: continuity at Dmax, the eq. (17)
 *                                   limit at large D for any delta < 1,
 *                                   direct quadrature of eq. (14) at D = 60,
 *                                   120 past the table, r dphi/dd1 against
 *                                   central differences in both branches
 *   orc_spline_*                    pinned: node reproduction, exact cubic
 *                                   reproduction, 1-D library spline
 *   orc_eps_c, orc_q0               pinned: k_F and gradient-term hand values,
 *                                   high-density limit, partials vs FD
 *   orc_gradient, orc_gradient_T    pinned: Fourier symbol, adjoint identity
 *   orc_pair_AU                     pinned: brute force with direct
 *                                   quadrature, translation invariance,
 *                                   far-fragment asymptotic sum
 *   orc_semilocal, orc_fx_many,     pinned: exact uniform scaling of the
 *   orc_pbe_H_many                  exchange energies on the grid, uniform
 *                                   density (GGA = LDA), enhancement-factor
 *                                   and gradient-correction limits
 *   orc_pair_AU_cell,               pinned: equals the orthogonal code on
 *   orc_gradient_cell,              diagonal cells, lattice-basis and rotation
 *   orc_gradient_T_cell             invariance of E, exact Fourier symbol of
 *                                   the skewed gradient, adjoint identity,
 *                                   brute-force pair counts
 *   orc_far_tail                    pinned: the radial integrals of the
 *                                   lattice continuum by adaptive quadrature
 *                                   (one, two and three periodic axes, skewed
 *                                   cells), the exact lattice sum of eq. (17)
 *                                   beyond r_cut (for one axis: averaged over
 *                                   the offset along it), convergence of
 *                                   E + T with r_cut against direct sums
 *   orc_line_tail_integral          pinned: adaptive quadrature of its
 *                                   integral on both of its branches
 *   orc_far_tail_AB                 pinned: the far field's potential against
 *                                   central differences of orc_far_tail
 *   orc_phi0_many                   pinned: small-voxel logarithmic law,
 *                                   scale duality phi0(s q; v) = phi0(q; s v),
 *                                   Monte Carlo voxel average, quadrature
 *                                   convergence
 *   gradient_spectral(_T)           pinned: band-limited plane-wave sums on
 *   (numpy, in __init__.py)         orthorhombic and skewed cells, Nyquist
 *                                   mode, textbook circulant matrix, adjoint
 *                                   identity, spectral accuracy
 *   paper-level energies            parity unpinned: the paper's Xe density
 *                                   file is not available
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ---------------------------------------------------------------------- */
/* Gauss-Legendre rule on [-1, 1]: roots of P_n by Newton's method on the   */
/* three-term recurrence (textbook; Abramowitz & Stegun 25.4.29).           */
/* ---------------------------------------------------------------------- */
static void gl_rule(int n, double *x, double *w)
{
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = cos(M_PI * (i + 0.75) / (n + 0.5));
        double pn = 0.0, dpn = 1.0;
        for (int it = 0; it < 200; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            pn = (n == 1) ? z : p1;
            double pm = (n == 1) ? 1.0 : p0;
            dpn = n * (z * pn - pm) / (z * z - 1.0);
            double dz = pn / dpn;
            z -= dz;
            if (fabs(dz) < 1e-15) {
                /* one more evaluation of P'_n at the converged root */
                p0 = 1.0; p1 = z;
                for (int k = 2; k <= n; ++k) {
                    double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                    p0 = p1;
                    p1 = p2;
                }
                pn = (n == 1) ? z : p1;
                pm = (n == 1) ? 1.0 : p0;
                dpn = n * (z * pn - pm) / (z * z - 1.0);
                break;
            }
        }
        x[i] = -z;
        x[n - 1 - i] = z;
        w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dpn * dpn);
    }
}

/* ---------------------------------------------------------------------- */
/* Quadrature grid on (0, A], A = (m + 1/2) pi.                             */
/*  - (0, a_min) is dropped: the integrand vanishes like a^2 there.          */
/*  - [a_min, 1]: panels of equal ratio (about log_ratio), n_log GL points.  */
/*  - [1, A]: [1, 3pi/2] then unit-pi panels [(k-1/2)pi, (k+1/2)pi]; a panel */
/*    starting at a_lo is cut into ceil(width / max(a_lo/4, pi/4)) equal     */
/*    pieces (the switch of h(a/d) near a ~ d needs them for d of order 1),  */
/*    n_osc GL points each.  Ending at cos(A) = 0 removes the leading 1/A^3  */
/*    term of the truncated oscillatory tail (left error ~ 4/A^4).           */
/* When a is NULL only the node count is returned.                          */
/* ---------------------------------------------------------------------- */
static int grid_fill(double a_min, double log_ratio, int n_log, int m_half, int n_osc,
                     double *a, double *w)
{
    if (a_min <= 0.0 || a_min >= 1.0 || log_ratio <= 1.0 || n_log < 1 ||
        m_half < 1 || n_osc < 1 || n_log > 64 || n_osc > 64)
        return -1;
    double xl[64], wl[64], xo[64], wo[64];
    gl_rule(n_log, xl, wl);
    gl_rule(n_osc, xo, wo);
    int nlp = (int)ceil(log(1.0 / a_min) / log(log_ratio) - 1e-12);
    if (nlp < 1) nlp = 1;
    double rho = pow(1.0 / a_min, 1.0 / nlp);
    int c = 0;
    for (int p = 0; p < nlp; ++p) {
        double lo = a_min * pow(rho, p);
        double hi = (p == nlp - 1) ? 1.0 : a_min * pow(rho, p + 1);
        for (int i = 0; i < n_log; ++i) {
            if (a) {
                a[c] = 0.5 * (lo + hi) + 0.5 * (hi - lo) * xl[i];
                w[c] = 0.5 * (hi - lo) * wl[i];
            }
            ++c;
        }
    }
    for (int k = 1; k <= m_half; ++k) {
        double lo = (k == 1) ? 1.0 : (k - 0.5) * M_PI;
        double hi = (k + 0.5) * M_PI;
        double wmax = 0.25 * lo > 0.25 * M_PI ? 0.25 * lo : 0.25 * M_PI;
        int sub = (int)ceil((hi - lo) / wmax - 1e-12);
        if (sub < 1) sub = 1;
        for (int q = 0; q < sub; ++q) {
            double l2 = lo + (hi - lo) * q / sub, h2 = lo + (hi - lo) * (q + 1) / sub;
            for (int i = 0; i < n_osc; ++i) {
                if (a) {
                    a[c] = 0.5 * (l2 + h2) + 0.5 * (h2 - l2) * xo[i];
                    w[c] = 0.5 * (h2 - l2) * wo[i];
                }
                ++c;
            }
        }
    }
    return c;
}

int orc_grid_size(double a_min, double log_ratio, int n_log, int m_half, int n_osc)
{
    return grid_fill(a_min, log_ratio, n_log, m_half, n_osc, NULL, NULL);
}

int orc_grid(double a_min, double log_ratio, int n_log, int m_half, int n_osc,
             double *a, double *w)
{
    return grid_fill(a_min, log_ratio, n_log, m_half, n_osc, a, w);
}

/* ---------------------------------------------------------------------- */
/* Dion eq. (14) ingredients.                                              */
/*   W(a,b) = 2[(3-a^2) b cos b sin a + (3-b^2) a cos a sin b               */
/*             + (a^2+b^2-3) sin a sin b - 3 a b cos a cos b] / (a^3 b^3)  */
/* Collecting the bracket gives                                             */
/*   a^2 sin a (sin b - b cos b) + b^2 sin b (sin a - a cos a)              */
/*   - 3 (sin a - a cos a)(sin b - b cos b),                                */
/* so with s(a) = sin a / a and u(a) = (sin a - a cos a)/a^3,               */
/*   W = 2 [ s(a) u(b) + s(b) u(a) - 3 u(a) u(b) ].                         */
/* u(a) is evaluated by its Maclaurin series for small a, where the printed */
/* form cancels: u(a) = sum_k (-1)^k (2k+2) a^(2k) / (2k+3)!.               */
/* ---------------------------------------------------------------------- */
static double orc_s(double a) { return sin(a) / a; }

static double orc_u(double a)
{
    if (a < 0.25) {
        double a2 = a * a, term = 1.0, sum = 0.0, fact = 6.0; /* (2k+3)! at k=0 */
        for (int k = 0; k < 10; ++k) {
            sum += ((k & 1) ? -1.0 : 1.0) * (2.0 * k + 2.0) * term / fact;
            term *= a2;
            fact *= (2.0 * k + 4.0) * (2.0 * k + 5.0);
        }
        return sum;
    }
    return (sin(a) - a * cos(a)) / (a * a * a);
}

double orc_W(double a, double b)
{
    double sa = orc_s(a), sb = orc_s(b), ua = orc_u(a), ub = orc_u(b);
    return 2.0 * (sa * ub + sb * ua - 3.0 * ua * ub);
}

/* h(y) = 1 - exp(-gamma y^2), gamma = 4 pi / 9 (Dion eq. 16);
 * nu(y) = y^2 / (2 h(y/d)) (Dion eq. 15).  d = 0 gives h = 1. */
static double orc_nu(double y, double d)
{
    if (d <= 0.0) return 0.5 * y * y;
    const double gam = 4.0 * M_PI / 9.0;
    double x = y / d;
    double h = -expm1(-gam * x * x);
    return 0.5 * y * y / h;
}

/* T(w,x,y,z) = 1/2 [1/(w+x) + 1/(y+z)] [1/((w+y)(x+z)) + 1/((w+z)(y+x))] */
static double orc_T(double w, double x, double y, double z)
{
    return 0.5 * (1.0 / (w + x) + 1.0 / (y + z)) *
           (1.0 / ((w + y) * (x + z)) + 1.0 / ((w + z) * (y + x)));
}

/* phi(d1, d2) = 2/pi^2 int_0^inf a^2 da int_0^inf b^2 db W(a,b)
 *               T(nu(a), nu(b), nu'(a), nu'(b)),  nu uses d1, nu' uses d2.
 * Full tensor-product double loop (no symmetry folding). */
static double phi_on_grid(int N, const double *a, const double *WW,
                          double d1, double d2, double *nu1, double *nu2)
{
    for (int i = 0; i < N; ++i) {
        nu1[i] = orc_nu(a[i], d1);
        nu2[i] = orc_nu(a[i], d2);
    }
    double total = 0.0;
    for (int i = 0; i < N; ++i) {
        double row = 0.0;
        const double *Wi = WW + (size_t)i * N;
        for (int j = 0; j < N; ++j)
            row += Wi[j] * orc_T(nu1[i], nu1[j], nu2[i], nu2[j]);
        total += row;
    }
    return 2.0 / (M_PI * M_PI) * total;
}

static double *make_WW(int N, const double *a, const double *w)
{
    double *WW = (double *)malloc(sizeof(double) * (size_t)N * N);
    if (!WW) return NULL;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j)
            WW[(size_t)i * N + j] = w[i] * w[j] * a[i] * a[i] * a[j] * a[j] * orc_W(a[i], a[j]);
    return WW;
}

/* phi at a list of (d1, d2) points. */
int orc_phi_many(int npts, const double *d1, const double *d2, double *out,
                 double a_min, double log_ratio, int n_log, int m_half, int n_osc)
{
    int N = orc_grid_size(a_min, log_ratio, n_log, m_half, n_osc);
    double *a = (double *)malloc(sizeof(double) * N);
    double *w = (double *)malloc(sizeof(double) * N);
    if (!a || !w) { free(a); free(w); return -2; }
    if (orc_grid(a_min, log_ratio, n_log, m_half, n_osc, a, w) != N) { free(a); free(w); return -1; }
    double *WW = make_WW(N, a, w);
    if (!WW) { free(a); free(w); return -2; }
    int err = 0;
#pragma omp parallel
    {
        double *nu1 = (double *)malloc(sizeof(double) * N);
        double *nu2 = (double *)malloc(sizeof(double) * N);
        if (!nu1 || !nu2) {
#pragma omp atomic write
            err = -2;
        } else {
#pragma omp for schedule(dynamic, 1)
            for (int p = 0; p < npts; ++p)
                out[p] = phi_on_grid(N, a, WW, d1[p], d2[p], nu1, nu2);
        }
        free(nu1);
        free(nu2);
    }
    free(WW); free(a); free(w);
    return err;
}

/* Node table phi(D_k, delta_l), D_k = Dmax k/(nD-1), delta_l = l/ndelta
 * (section 2: phi tabulated in D and delta; section 7: grid limits fixed by
 * refinement).  Row k = 0 (D = 0): eq. (14) diverges like -(2/pi) ln D there,
 * so the row holds the value at D = 0 of the even quadratic c0 + c2 D^2
 * through the nodes D_1 and D_2:  phi(0, delta) = (4 phi(D_1) - phi(D_2))/3. */
int orc_phi_table(int nD, double Dmax, int ndelta, double *nodes,
                  double a_min, double log_ratio, int n_log, int m_half, int n_osc)
{
    if (nD < 3 || ndelta < 2 || Dmax <= 0.0) return -1;
    int npts = (nD - 1) * ndelta;
    double *d1 = (double *)malloc(sizeof(double) * npts);
    double *d2 = (double *)malloc(sizeof(double) * npts);
    double *v = (double *)malloc(sizeof(double) * npts);
    if (!d1 || !d2 || !v) { free(d1); free(d2); free(v); return -2; }
    for (int k = 1; k < nD; ++k)
        for (int l = 0; l < ndelta; ++l) {
            double D = Dmax * k / (nD - 1), dl = (double)l / ndelta;
            d1[(k - 1) * ndelta + l] = D * (1.0 + dl);
            d2[(k - 1) * ndelta + l] = D * (1.0 - dl);
        }
    int rc = orc_phi_many(npts, d1, d2, v, a_min, log_ratio, n_log, m_half, n_osc);
    if (rc == 0) {
        for (int k = 1; k < nD; ++k)
            for (int l = 0; l < ndelta; ++l)
                nodes[(size_t)k * ndelta + l] = v[(k - 1) * ndelta + l];
        for (int l = 0; l < ndelta; ++l)
            nodes[l] = (4.0 * nodes[ndelta + l] - nodes[2 * ndelta + l]) / 3.0;
    }
    free(d1); free(d2); free(v);
    return rc;
}

/* ---------------------------------------------------------------------- */
/* Tensor-product cubic interpolating spline on the uniform (D, delta)      */
/* node grid, written with second derivatives (the "M" form).  Boundary     */
/* conditions (reading; the paper only says "lookup table", section 7):     */
/* zero slope at D = 0 and delta = 0 (phi is even in r and in delta),       */
/* zero second derivative at the last node of each axis.                    */
/* ---------------------------------------------------------------------- */
/* Solve for M_0..M_{N-1} of the 1-D spline through f (stride fs) with
 * S'(x_0) = 0 and M_{N-1} = 0; result to M (stride ms). */
static void spline_M_1d(int N, double h, const double *f, int fs, double *M, int ms,
                        double *cp, double *dp)
{
    /* rows: 0: 2 M0 + M1 = 6 (f1 - f0)/h^2
     *       i: M_{i-1} + 4 M_i + M_{i+1} = 6 (f_{i+1} - 2 f_i + f_{i-1})/h^2
     *       N-1: M_{N-1} = 0                                                 */
    double h2 = h * h;
    /* Thomas algorithm on rows 0..N-2 with M_{N-1} = 0 substituted. */
    int n = N - 1;
    for (int i = 0; i < n; ++i) {
        double diag, sup, rhs, sub;
        if (i == 0) {
            sub = 0.0; diag = 2.0; sup = 1.0;
            rhs = 6.0 * (f[fs * 1] - f[0]) / h2;
        } else {
            sub = 1.0; diag = 4.0; sup = (i == n - 1) ? 0.0 : 1.0;
            rhs = 6.0 * (f[fs * (i + 1)] - 2.0 * f[fs * i] + f[fs * (i - 1)]) / h2;
        }
        if (i == 0) {
            cp[i] = sup / diag;
            dp[i] = rhs / diag;
        } else {
            double den = diag - sub * cp[i - 1];
            cp[i] = sup / den;
            dp[i] = (rhs - sub * dp[i - 1]) / den;
        }
    }
    M[ms * (N - 1)] = 0.0;
    M[ms * (n - 1)] = dp[n - 1];
    for (int i = n - 2; i >= 0; --i) M[ms * i] = dp[i] - cp[i] * M[ms * (i + 1)];
}

/* f: nD x nd nodes (row-major, D outer).  Outputs fDD, fdd, fDDdd same shape,
 * and rho, rhoM (nd): the ratio of the last row to eq. (17) at D = Dmax and its
 * second derivatives along delta (see kernel_pair). */
int orc_spline_prepare(int nD, double hD, int nd, double hd, const double *f,
                       double *fDD, double *fdd, double *fDDdd, double *rho, double *rhoM)
{
    if (nD < 3 || nd < 3) return -1;
    int nmax = nD > nd ? nD : nd;
    double *cp = (double *)malloc(sizeof(double) * nmax);
    double *dp = (double *)malloc(sizeof(double) * nmax);
    if (!cp || !dp) { free(cp); free(dp); return -2; }
    for (int l = 0; l < nd; ++l) spline_M_1d(nD, hD, f + l, nd, fDD + l, nd, cp, dp);
    for (int k = 0; k < nD; ++k) spline_M_1d(nd, hd, f + (size_t)k * nd, 1, fdd + (size_t)k * nd, 1, cp, dp);
    for (int k = 0; k < nD; ++k) spline_M_1d(nd, hd, fDD + (size_t)k * nd, 1, fDDdd + (size_t)k * nd, 1, cp, dp);
    const double C = 12.0 * pow(4.0 * M_PI / 9.0, 3);
    const double Dmax = (nD - 1) * hD;
    for (int l = 0; l < nd; ++l) {
        double d1 = Dmax * (1.0 + l * hd), d2 = Dmax * (1.0 - l * hd);
        double a17 = -C / (d1 * d1 * d2 * d2 * (d1 * d1 + d2 * d2));
        rho[l] = f[(size_t)(nD - 1) * nd + l] / a17;
    }
    spline_M_1d(nd, hd, rho, 1, rhoM, 1, cp, dp);
    free(cp); free(dp);
    return 0;
}

typedef struct {
    int nD, nd;
    double hD, hd;
    const double *f, *fDD, *fdd, *fDDdd;
    const double *rho, *rhoM;  /* beyond-table normalisation (see kernel_pair) */
} orc_spline;

/* 1-D cubic spline in delta (M form) through y at the delta nodes: value and slope. */
static void spline1_eval(int nd, double hd, const double *y, const double *M, double dl,
                         double *v, double *dv)
{
    double td = dl / hd;
    int l = (int)floor(td);
    if (l > nd - 2) l = nd - 2;
    if (l < 0) l = 0;
    double u = td - l, A = 1.0 - u, B = u;
    *v = A * y[l] + B * y[l + 1] + ((A * A * A - A) * M[l] + (B * B * B - B) * M[l + 1]) * hd * hd / 6.0;
    *dv = (y[l + 1] - y[l]) / hd + (-(3.0 * A * A - 1.0) * M[l] + (3.0 * B * B - 1.0) * M[l + 1]) * hd / 6.0;
}

/* S(D, delta), its partials and the mixed partial, D in [0, (nD-1) hD],
 * delta in [0, (nd-1) hd]. */
static void spline_eval2(const orc_spline *s, double D, double dl,
                         double *phi, double *phiD, double *phid, double *phiDd)
{
    double tD = D / s->hD, td = dl / s->hd;
    int k = (int)floor(tD), l = (int)floor(td);
    if (k > s->nD - 2) k = s->nD - 2;
    if (k < 0) k = 0;
    if (l > s->nd - 2) l = s->nd - 2;
    if (l < 0) l = 0;
    double t = tD - k, u = td - l;
    double hD = s->hD, hd = s->hd;
    /* 1-D cubic spline basis in the M form, and their derivatives. */
    double al[2] = {1.0 - t, t};
    double ga[2] = {((1.0 - t) * (1.0 - t) * (1.0 - t) - (1.0 - t)) * hD * hD / 6.0,
                    (t * t * t - t) * hD * hD / 6.0};
    double dal[2] = {-1.0 / hD, 1.0 / hD};
    double dga[2] = {-(3.0 * (1.0 - t) * (1.0 - t) - 1.0) * hD / 6.0,
                     (3.0 * t * t - 1.0) * hD / 6.0};
    double be[2] = {1.0 - u, u};
    double et[2] = {((1.0 - u) * (1.0 - u) * (1.0 - u) - (1.0 - u)) * hd * hd / 6.0,
                    (u * u * u - u) * hd * hd / 6.0};
    double dbe[2] = {-1.0 / hd, 1.0 / hd};
    double det[2] = {-(3.0 * (1.0 - u) * (1.0 - u) - 1.0) * hd / 6.0,
                     (3.0 * u * u - 1.0) * hd / 6.0};
    double p = 0.0, pD = 0.0, pd = 0.0, pDd = 0.0;
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            size_t o = (size_t)(k + i) * s->nd + (l + j);
            double F = s->f[o], FDD = s->fDD[o], Fdd = s->fdd[o], FDDdd = s->fDDdd[o];
            p += al[i] * be[j] * F + ga[i] * be[j] * FDD + al[i] * et[j] * Fdd + ga[i] * et[j] * FDDdd;
            pD += dal[i] * be[j] * F + dga[i] * be[j] * FDD + dal[i] * et[j] * Fdd + dga[i] * et[j] * FDDdd;
            pd += al[i] * dbe[j] * F + ga[i] * dbe[j] * FDD + al[i] * det[j] * Fdd + ga[i] * det[j] * FDDdd;
            pDd += dal[i] * dbe[j] * F + dga[i] * dbe[j] * FDD + dal[i] * det[j] * Fdd + dga[i] * det[j] * FDDdd;
        }
    *phi = p;
    *phiD = pD;
    *phid = pd;
    if (phiDd) *phiDd = pDd;
}

static void spline_eval(const orc_spline *s, double D, double dl,
                        double *phi, double *phiD, double *phid)
{
    spline_eval2(s, D, dl, phi, phiD, phid, NULL);
}

int orc_spline_eval_many(int nD, double hD, int nd, double hd, const double *f,
                         const double *fDD, const double *fdd, const double *fDDdd,
                         int npts, const double *D, const double *dl,
                         double *phi, double *phiD, double *phid)
{
    orc_spline s = {nD, nd, hD, hd, f, fDD, fdd, fDDdd, NULL, NULL};
    for (int p = 0; p < npts; ++p) spline_eval(&s, D[p], dl[p], &phi[p], &phiD[p], &phid[p]);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* The kernel as the double sum uses it (section 2):                        */
/*   D <= Dmax: the spline of the node table; above the last delta node   */
/*              (delta > 0.995 for 200 nodes) its natural continuation,     */
/*              linear in delta with the end slope (zero curvature there),  */
/*              so phi stays twice differentiable in delta;                */
/*   D >  Dmax: Dion eq. (17), phi17 = -C / (d1^2 d2^2 (d1^2 + d2^2)),      */
/*              C = 12 (4 pi / 9)^3, d1 = D (1 + delta), d2 = D (1 - delta),*/
/*              times g = rho(delta*) + (1 - rho(0)) (1 - (Dmax / D)^2),    */
/*              rho the cubic spline (same end conditions as the table)     */
/*              through phi(Dmax, delta_l) / phi17(Dmax, delta_l), and      */
/*              delta* = max(0, 1 - min(d1, d2) / Dmax): the delta at which */
/*              the last table row has the same smaller argument.          */
/* Reading: eq. (17) is the limit where both d1 and d2 are large; with d1   */
/* large, phi / phi17 depends on the smaller argument alone (by quadrature */
/* of eq. (14): at min(d1, d2) = 1.8 the ratio is 0.3614 at D = 30 and     */
/* 0.3629 at D = 120).  So the ratio the table shows at D = Dmax is carried */
/* to larger D along constant min(d1, d2), and it tends to 1 as that grows. */
/* The second term takes out the table's own error at delta* = 0 (where    */
/* eq. (17) is exact to 1e-8 at D = 30) over growing D.  At D = Dmax,      */
/* g = rho(delta): phi is continuous there, so E is a continuous function   */
/* of n.                                                                    */
/* Returns phi, and r * dphi/dd1 for the pair (d1 = q_i r, d2 = q_j r),     */
/* with signed ds = (q_i - q_j)/(q_i + q_j), dds/dd1 = (1 - ds)/(2 D):      */
/*   dphi/dd1 = 1/2 phi_D + (1 - ds)/(2 D) phi_ds;                          */
/* beyond Dmax, r dg/dd1 = -rho'(delta*) r / Dmax (only when d1 is the     */
/* smaller argument and delta* > 0) + (1 - rho(0)) Dmax^2 r / D^3.          */
/* ---------------------------------------------------------------------- */
static void kernel_pair(const orc_spline *s, double Dmax, double r, double qi, double qj,
                        double *phi, double *rdphi1, int *clamped)
{
    const double C = 12.0 * pow(4.0 * M_PI / 9.0, 3);
    double sq = qi + qj;
    double D = 0.5 * r * sq;
    double ds = (qi - qj) / sq;
    double dl = fabs(ds);
    double sgn = (ds > 0.0) ? 1.0 : ((ds < 0.0) ? -1.0 : 0.0);
    double dlast = (s->nd - 1) * s->hd;
    double ext = 0.0;   /* distance beyond the last delta node */
    if (dl > dlast) { ext = dl - dlast; dl = dlast; *clamped += 1; }
    if (D > Dmax) {
        double d1 = qi * r, d2 = qj * r;
        double d12 = d1 * d1, d22 = d2 * d2;
        double p17 = -C / (d12 * d22 * (d12 + d22));
        double dp17 = -p17 * (2.0 / d1 + 2.0 * d1 / (d12 + d22));
        double dsmall = (d1 < d2) ? d1 : d2;
        double dstar = 1.0 - dsmall / Dmax;
        double rho, drho;
        if (dstar > 0.0) {
            double e = 0.0;   /* past the last delta node: linear continuation */
            double dc = dstar;
            if (dc > dlast) { e = dc - dlast; dc = dlast; }
            spline1_eval(s->nd, s->hd, s->rho, s->rhoM, dc, &rho, &drho);
            rho += drho * e;
        } else {
            rho = s->rho[0];  /* the spline through the nodes takes rho_0 at delta = 0 */
            drho = 0.0;       /* and has zero slope there (end condition) */
        }
        double rho0 = s->rho[0];
        double Dr = Dmax / D;
        double g = rho + (1.0 - rho0) * (1.0 - Dr * Dr);
        double rdg = (1.0 - rho0) * Dr * Dr * r / D;
        if (d1 < d2 && dstar > 0.0) rdg -= drho * r / Dmax;
        *phi = g * p17;
        *rdphi1 = r * g * dp17 + p17 * rdg;
        return;
    }
    double p, pD, pd, pDd;
    spline_eval2(s, D, dl, &p, &pD, &pd, &pDd);
    p += pd * ext;      /* the continuation: S(D, last) + S_delta(D, last) ext */
    pD += pDd * ext;
    *phi = p;
    if (D > 0.0)
        *rdphi1 = r * (0.5 * pD + (1.0 - ds) / (2.0 * D) * sgn * pd);
    else
        *rdphi1 = 0.0;
}

int orc_kernel_many(int nD, double hD, int nd, double hd, const double *f,
                    const double *fDD, const double *fdd, const double *fDDdd,
                    const double *rho, const double *rhoM,
                    int npts, const double *r, const double *qi, const double *qj,
                    double *phi, double *rdphi1)
{
    orc_spline s = {nD, nd, hD, hd, f, fDD, fdd, fDDdd, rho, rhoM};
    double Dmax = (nD - 1) * hD;
    int cl = 0;
    for (int p = 0; p < npts; ++p) kernel_pair(&s, Dmax, r[p], qi[p], qj[p], &phi[p], &rdphi1[p], &cl);
    return cl;
}

/* ---------------------------------------------------------------------- */
/* Pair sums (section 2 eq. (2), section 3: trimming, 0th cell + images).   */
/* Active points p = 0..Na-1 at integer grid indices (i0,i1,i2) of an       */
/* orthorhombic cell L0 x L1 x L2 on an n0 x n1 x n2 grid: r = (i0 L0/n0,    */
/* i1 L1/n1, i2 L2/n2).  Periodic axes add images m L (|m| <= M); pairs with */
/* |r_i - r_j + L|^2 > rc^2 (1 + 1e-12) are dropped when rc > 0 (spherical  */
/* cutoff, inclusive, with distances that equal rc up to rounding counted    */
/* inside; the paper repeats cells until convergence, sections 3 and 6.2).  */
/* The self                                                                  */
/* term i = j, L = 0 is n_i phi(0,0) and always included.                   */
/*   A_i = sum_{j,L} n_j phi_ijL,  U_i = n_i sum_{j,L} n_j r dphi/dd1.       */
/* Also returns, per query, the number of (j, L) terms other than the self  */
/* term (the ordered pair count) and how many had delta clamped.            */
/* ---------------------------------------------------------------------- */
int orc_pair_AU(int Na, const int32_t *i0, const int32_t *i1, const int32_t *i2,
                const double *n, const double *q,
                int n0, int n1, int n2, double L0, double L1, double L2,
                int per0, int per1, int per2, double rc,
                int nD, double hD, int nd, double hd, const double *f,
                const double *fDD, const double *fdd, const double *fDDdd,
                const double *rho, const double *rhoM,
                int nq, const int32_t *qidx, double *A, double *U,
                int64_t *npairs, int64_t *nclamp)
{
    if ((per0 || per1 || per2) && !(rc > 0.0)) return -1;
    orc_spline s = {nD, nd, hD, hd, f, fDD, fdd, fDDdd, rho, rhoM};
    double Dmax = (nD - 1) * hD;
    int M0 = per0 ? (int)ceil(rc / L0) + 1 : 0;
    int M1 = per1 ? (int)ceil(rc / L1) + 1 : 0;
    int M2 = per2 ? (int)ceil(rc / L2) + 1 : 0;
    double h0 = L0 / n0, h1 = L1 / n1, h2 = L2 / n2;
    double phi00 = f[0];
#pragma omp parallel for schedule(dynamic, 4)
    for (int t = 0; t < nq; ++t) {
        int i = qidx[t];
        double xi = i0[i] * h0, yi = i1[i] * h1, zi = i2[i] * h2;
        double a = 0.0, u = 0.0;
        int64_t cnt = 0;
        int cl = 0;
        for (int j = 0; j < Na; ++j) {
            double xj = i0[j] * h0, yj = i1[j] * h1, zj = i2[j] * h2;
            for (int m0 = -M0; m0 <= M0; ++m0)
                for (int m1 = -M1; m1 <= M1; ++m1)
                    for (int m2 = -M2; m2 <= M2; ++m2) {
                        if (j == i && m0 == 0 && m1 == 0 && m2 == 0) {
                            a += n[i] * phi00;
                            continue;
                        }
                        double dx = xi - xj + m0 * L0, dy = yi - yj + m1 * L1, dz = zi - zj + m2 * L2;
                        double r2 = dx * dx + dy * dy + dz * dz;
                        if (rc > 0.0 && r2 > rc * rc * (1.0 + 1e-12)) continue;
                        double r = sqrt(r2);
                        double p, rd;
                        kernel_pair(&s, Dmax, r, q[i], q[j], &p, &rd, &cl);
                        a += n[j] * p;
                        u += n[j] * rd;
                        ++cnt;
                    }
        }
        A[t] = a;
        U[t] = n[i] * u;
        if (npairs) npairs[t] = cnt;
        if (nclamp) nclamp[t] = cl;
    }
    return 0;
}

/* Brute force of the same sum with phi from direct quadrature of eq. (14)
 * at every pair (no table, no spline, no asymptote); the self term uses phi00
 * given by the caller.  Returns sum_i n_i A_i. */
int orc_pair_brute(int Na, const int32_t *i0, const int32_t *i1, const int32_t *i2,
                   const double *n, const double *q,
                   int n0, int n1, int n2, double L0, double L1, double L2,
                   int per0, int per1, int per2, double rc, double Dmax, double phi00,
                   double a_min, double log_ratio, int n_log, int m_half, int n_osc,
                   double *sum_out)
{
    if ((per0 || per1 || per2) && !(rc > 0.0)) return -1;
    (void)Dmax;
    int M0 = per0 ? (int)ceil(rc / L0) + 1 : 0;
    int M1 = per1 ? (int)ceil(rc / L1) + 1 : 0;
    int M2 = per2 ? (int)ceil(rc / L2) + 1 : 0;
    double h0 = L0 / n0, h1 = L1 / n1, h2 = L2 / n2;
    /* gather every ordered non-self term within the cutoff */
    size_t cap = 1024, cnt = 0;
    double *d1 = (double *)malloc(sizeof(double) * cap);
    double *d2 = (double *)malloc(sizeof(double) * cap);
    double *wt = (double *)malloc(sizeof(double) * cap);
    if (!d1 || !d2 || !wt) { free(d1); free(d2); free(wt); return -2; }
    double self = 0.0;
    for (int i = 0; i < Na; ++i) {
        self += n[i] * n[i] * phi00;
        for (int j = 0; j < Na; ++j)
            for (int m0 = -M0; m0 <= M0; ++m0)
                for (int m1 = -M1; m1 <= M1; ++m1)
                    for (int m2 = -M2; m2 <= M2; ++m2) {
                        if (j == i && m0 == 0 && m1 == 0 && m2 == 0) continue;
                        double dx = i0[i] * h0 - i0[j] * h0 + m0 * L0;
                        double dy = i1[i] * h1 - i1[j] * h1 + m1 * L1;
                        double dz = i2[i] * h2 - i2[j] * h2 + m2 * L2;
                        double r2 = dx * dx + dy * dy + dz * dz;
                        if (rc > 0.0 && r2 > rc * rc * (1.0 + 1e-12)) continue;
                        double r = sqrt(r2);
                        if (cnt == cap) {
                            cap *= 2;
                            double *t1 = (double *)realloc(d1, sizeof(double) * cap);
                            double *t2 = (double *)realloc(d2, sizeof(double) * cap);
                            double *t3 = (double *)realloc(wt, sizeof(double) * cap);
                            if (!t1 || !t2 || !t3) {
                                free(t1 ? t1 : d1); free(t2 ? t2 : d2); free(t3 ? t3 : wt);
                                return -2;
                            }
                            d1 = t1; d2 = t2; wt = t3;
                        }
                        d1[cnt] = q[i] * r;
                        d2[cnt] = q[j] * r;
                        wt[cnt] = n[i] * n[j];
                        ++cnt;
                    }
    }
    double *ph = (double *)malloc(sizeof(double) * (cnt ? cnt : 1));
    if (!ph) { free(d1); free(d2); free(wt); return -2; }
    int rc2 = orc_phi_many((int)cnt, d1, d2, ph, a_min, log_ratio, n_log, m_half, n_osc);
    double tab = 0.0;
    for (size_t p = 0; p < cnt; ++p) tab += wt[p] * ph[p];
    *sum_out = self + tab;
    free(d1); free(d2); free(wt); free(ph);
    return rc2;
}

/* ---------------------------------------------------------------------- */
/* Gradient by real-space finite differences along the (orthogonal) axes    */
/* (section 3: "real space finite differences ... perpendicular axes only"),*/
/* 4th order central, periodic wrap on every axis:                          */
/*   (D_h f)_m = (f_{m-2} - 8 f_{m-1} + 8 f_{m+1} - f_{m+2}) / (12 h).      */
/* Grid row-major [n0][n1][n2]; g is [3][N].                                */
/* ---------------------------------------------------------------------- */
static const double orc_fd_c[5] = {1.0 / 12.0, -8.0 / 12.0, 0.0, 8.0 / 12.0, -1.0 / 12.0};

int orc_gradient(int n0, int n1, int n2, double h0, double h1, double h2,
                 const double *f, double *g)
{
    size_t N = (size_t)n0 * n1 * n2;
    int dims[3] = {n0, n1, n2};
    double hs[3] = {h0, h1, h2};
#pragma omp parallel for collapse(2) schedule(static)
    for (int a = 0; a < n0; ++a)
        for (int b = 0; b < n1; ++b)
            for (int c = 0; c < n2; ++c) {
                int idx[3] = {a, b, c};
                size_t m = ((size_t)a * n1 + b) * n2 + c;
                for (int ax = 0; ax < 3; ++ax) {
                    double s = 0.0;
                    for (int o = -2; o <= 2; ++o) {
                        int jj[3] = {idx[0], idx[1], idx[2]};
                        jj[ax] = ((idx[ax] + o) % dims[ax] + dims[ax]) % dims[ax];
                        s += orc_fd_c[o + 2] * f[((size_t)jj[0] * n1 + jj[1]) * n2 + jj[2]];
                    }
                    g[ax * N + m] = s / hs[ax];
                }
            }
    return 0;
}

/* out = sum_axes D_h^T w_ax, the transpose of the stencil above written out
 * directly: (D_h^T w)_m = sum_o c_o w_{m-o} / h. */
int orc_gradient_T(int n0, int n1, int n2, double h0, double h1, double h2,
                   const double *w, double *out)
{
    size_t N = (size_t)n0 * n1 * n2;
    int dims[3] = {n0, n1, n2};
    double hs[3] = {h0, h1, h2};
#pragma omp parallel for collapse(2) schedule(static)
    for (int a = 0; a < n0; ++a)
        for (int b = 0; b < n1; ++b)
            for (int c = 0; c < n2; ++c) {
                int idx[3] = {a, b, c};
                size_t m = ((size_t)a * n1 + b) * n2 + c;
                double s = 0.0;
                for (int ax = 0; ax < 3; ++ax)
                    for (int o = -2; o <= 2; ++o) {
                        int jj[3] = {idx[0], idx[1], idx[2]};
                        jj[ax] = ((idx[ax] - o) % dims[ax] + dims[ax]) % dims[ax];
                        s += orc_fd_c[o + 2] * w[ax * N + ((size_t)jj[0] * n1 + jj[1]) * n2 + jj[2]] / hs[ax];
                    }
                out[m] = s;
            }
    return 0;
}

/* ---------------------------------------------------------------------- */
/* LDA correlation: Perdew & Wang, PRB 45, 13244 (1992), spin-unpolarised   */
/* (the paper names only "LDA", section 2 eq. (3)); Hartree units.          */
/*   eps_c(rs) = -2A (1 + a1 rs) ln[1 + 1/(2A (b1 rs^1/2 + b2 rs            */
/*                                          + b3 rs^3/2 + b4 rs^2))]        */
/* ---------------------------------------------------------------------- */
static const double PW_A = 0.031091, PW_a1 = 0.21370;
static const double PW_b1 = 7.5957, PW_b2 = 3.5876, PW_b3 = 1.6382, PW_b4 = 0.49294;

static void pw92(double rs, double *e, double *de_drs)
{
    double sr = sqrt(rs);
    double Q0 = -2.0 * PW_A * (1.0 + PW_a1 * rs);
    double Q1 = 2.0 * PW_A * (PW_b1 * sr + PW_b2 * rs + PW_b3 * rs * sr + PW_b4 * rs * rs);
    double Q1p = PW_A * (PW_b1 / sr + 2.0 * PW_b2 + 3.0 * PW_b3 * sr + 4.0 * PW_b4 * rs);
    double L = log(1.0 + 1.0 / Q1);
    *e = Q0 * L;
    *de_drs = -2.0 * PW_A * PW_a1 * L - Q0 * Q1p / (Q1 * Q1 + Q1);
}

int orc_eps_c(int N, const double *rs, double *e, double *de)
{
    for (int p = 0; p < N; ++p) pw92(rs[p], &e[p], &de[p]);
    return 0;
}

/* q0 (Dion eqs. 11-12):  q0 = -(4 pi / 3) eps_xc^0 with
 *   eps_xc^0 = eps_c^LDA + eps_x^LDA [1 - (Zab/9) s^2],
 *   eps_x^LDA = -3 k_F / (4 pi),  k_F = (3 pi^2 n)^(1/3),
 *   s = |grad n| / (2 k_F n),  Zab = -0.8491.
 * Partials (closed form):
 *   dq0/dn    = k_F/(3n) + (7 Zab/108) |g|^2/(k_F n^3) - (4 pi/3) d eps_c/dn
 *   dq0/dgrad = -(Zab/18) g / (k_F n^2)
 * Points with n <= 0 get zeros. */
int orc_q0(int N, const double *n, const double *g, double *q0, double *dq0dn, double *dq0dg)
{
    const double Zab = -0.8491;
#pragma omp parallel for schedule(static)
    for (int m = 0; m < N; ++m) {
        double nn = n[m];
        if (!(nn > 0.0)) {
            q0[m] = 0.0;
            if (dq0dn) dq0dn[m] = 0.0;
            if (dq0dg) { dq0dg[m] = 0.0; dq0dg[(size_t)N + m] = 0.0; dq0dg[2 * (size_t)N + m] = 0.0; }
            continue;
        }
        double gx = g[m], gy = g[(size_t)N + m], gz = g[2 * (size_t)N + m];
        double g2 = gx * gx + gy * gy + gz * gz;
        double kF = cbrt(3.0 * M_PI * M_PI * nn);
        double s = sqrt(g2) / (2.0 * kF * nn);
        double rs = cbrt(3.0 / (4.0 * M_PI * nn));
        double ec, dec_drs;
        pw92(rs, &ec, &dec_drs);
        double ex = -3.0 * kF / (4.0 * M_PI);
        double exc0 = ec + ex * (1.0 - (Zab / 9.0) * s * s);
        q0[m] = -(4.0 * M_PI / 3.0) * exc0;
        if (dq0dn) {
            double dec_dn = dec_drs * (-rs / (3.0 * nn));
            dq0dn[m] = kF / (3.0 * nn) + (7.0 * Zab / 108.0) * g2 / (kF * nn * nn * nn) -
                       (4.0 * M_PI / 3.0) * dec_dn;
        }
        if (dq0dg) {
            double c = -(Zab / 18.0) / (kF * nn * nn);
            dq0dg[m] = c * gx;
            dq0dg[(size_t)N + m] = c * gy;
            dq0dg[2 * (size_t)N + m] = c * gz;
        }
    }
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Semilocal energies of eq. (3).  Section 2 has JuNoLo evaluate E_x^LDA,   */
/* E_c^LDA, E_x^PBE, E_c^PBE and E_x^revPBE from the density itself, since */
/* the DFT code may not report them.  Spin-unpolarised, Hartree units,     */
/* written from the published definitions:                                 */
/*   eps_x^LDA = -3 k_F / (4 pi),  k_F = (3 pi^2 n)^(1/3)                  */
/*   eps_x^GGA = eps_x^LDA F_x(s),  s = |grad n| / (2 k_F n),              */
/*     F_x(s) = 1 + kappa - kappa / (1 + mu s^2 / kappa)                   */
/*     PBE (Perdew, Burke, Ernzerhof, PRL 77, 3865 (1996)): kappa = 0.804, */
/*     revPBE (Zhang and Yang, PRL 80, 890 (1998)): kappa = 1.245,         */
/*     mu = beta pi^2 / 3 in both                                          */
/*   eps_c^PBE = eps_c^PW92(rs) + H(rs, t),  t = |grad n| / (2 k_s n),     */
/*     k_s = (4 k_F / pi)^(1/2),                                           */
/*     H = gamma ln[1 + (beta/gamma) t^2 (1 + A t^2) / (1 + A t^2 + A^2 t^4)], */
/*     A = (beta/gamma) / (exp(-eps_c^PW92 / gamma) - 1),                  */
/*     beta = 0.06672455060314922, gamma = (1 - ln 2) / pi^2               */
/*   E = dV sum over points with n > 0 of n eps.                           */
/* ---------------------------------------------------------------------- */
static const double PBE_beta = 0.06672455060314922;

static double pbe_gamma(void) { return (1.0 - log(2.0)) / (M_PI * M_PI); }

static double pbe_mu(void) { return PBE_beta * M_PI * M_PI / 3.0; }

/* exchange enhancement factor F_x(s) for a given kappa */
static double fx(double s, double kappa)
{
    return 1.0 + kappa - kappa / (1.0 + pbe_mu() * s * s / kappa);
}

/* gradient correction H(rs, t) of the PBE correlation, given eps_c^PW92(rs) */
static double pbe_H(double ec, double t)
{
    double g = pbe_gamma();
    double A = (PBE_beta / g) / expm1(-ec / g);
    double t2 = t * t;
    double num = 1.0 + A * t2;
    double den = 1.0 + A * t2 + A * A * t2 * t2;
    return g * log(1.0 + (PBE_beta / g) * t2 * num / den);
}

int orc_fx_many(int N, const double *s, double kappa, double *out)
{
    for (int p = 0; p < N; ++p) out[p] = fx(s[p], kappa);
    return 0;
}

int orc_pbe_H_many(int N, const double *rs, const double *t, double *out)
{
    for (int p = 0; p < N; ++p) {
        double ec, de;
        pw92(rs[p], &ec, &de);
        out[p] = pbe_H(ec, t[p]);
    }
    return 0;
}

/* sums[0..4] = sum n eps for x^LDA, c^LDA (PW92), x^PBE, c^PBE, x^revPBE over
 * the N points with n > 0 (g: [3][N] gradient); *count = number of such points */
int orc_semilocal(int N, const double *n, const double *g, double *sums, int64_t *count)
{
    double S[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    int64_t c = 0;
    for (int m = 0; m < N; ++m) {
        double nn = n[m];
        if (!(nn > 0.0)) continue;
        double gx = g[m], gy = g[(size_t)N + m], gz = g[2 * (size_t)N + m];
        double ag = sqrt(gx * gx + gy * gy + gz * gz);
        double kF = cbrt(3.0 * M_PI * M_PI * nn);
        double ks = sqrt(4.0 * kF / M_PI);
        double s = ag / (2.0 * kF * nn);
        double t = ag / (2.0 * ks * nn);
        double rs = cbrt(3.0 / (4.0 * M_PI * nn));
        double ec, de;
        pw92(rs, &ec, &de);
        double ex = -3.0 * kF / (4.0 * M_PI);
        S[0] += nn * ex;
        S[1] += nn * ec;
        S[2] += nn * ex * fx(s, 0.804);
        S[3] += nn * (ec + pbe_H(ec, t));
        S[4] += nn * ex * fx(s, 1.245);
        ++c;
    }
    for (int k = 0; k < 5; ++k) sums[k] = S[k];
    *count = c;
    return 0;
}

/* ---------------------------------------------------------------------- */
/* General cells (section 2: the grid axes need not be orthogonal; the     */
/* paper's Xe monolayer cell is hexagonal).  Rows of cell[9] are the       */
/* lattice vectors M_0, M_1, M_2 (bohr); grid point (i_0, i_1, i_2) sits at */
/* r = sum_a (i_a / N_a) M_a, images are L = sum_a m_a M_a over the        */
/* periodic axes.  Reciprocal rows B_a with B_a . M_b = delta_ab.          */
/* ---------------------------------------------------------------------- */
static int cell_recip(const double *M, double *B)
{
    /* B = (M^{-1})^T: B_a = (M_b x M_c) / det, (a, b, c) cyclic */
    double det = M[0] * (M[4] * M[8] - M[5] * M[7]) - M[1] * (M[3] * M[8] - M[5] * M[6]) +
                 M[2] * (M[3] * M[7] - M[4] * M[6]);
    if (!(fabs(det) > 0.0)) return -1;
    for (int a = 0; a < 3; ++a) {
        const double *u = M + 3 * ((a + 1) % 3), *v = M + 3 * ((a + 2) % 3);
        B[3 * a + 0] = (u[1] * v[2] - u[2] * v[1]) / det;
        B[3 * a + 1] = (u[2] * v[0] - u[0] * v[2]) / det;
        B[3 * a + 2] = (u[0] * v[1] - u[1] * v[0]) / det;
    }
    return 0;
}

/* The pair sum of orc_pair_AU for a general cell.  Image range per periodic
 * axis: every L with |r_i - r_j + L| <= rc has |m_a| <= rc |B_a| + 1, since
 * the fractional coordinate of a vector r along a is r . B_a and that of
 * r_i - r_j lies in (-1, 1). */
int orc_pair_AU_cell(int Na, const int32_t *i0, const int32_t *i1, const int32_t *i2,
                     const double *n, const double *q, int n0, int n1, int n2, const double *cell,
                     int per0, int per1, int per2, double rc,
                     int nD, double hD, int nd, double hd, const double *f,
                     const double *fDD, const double *fdd, const double *fDDdd,
                     const double *rho, const double *rhoM,
                     int nq, const int32_t *qidx, double *A, double *U,
                     int64_t *npairs, int64_t *nclamp)
{
    if ((per0 || per1 || per2) && !(rc > 0.0)) return -1;
    double B[9];
    if (cell_recip(cell, B)) return -1;
    orc_spline s = {nD, nd, hD, hd, f, fDD, fdd, fDDdd, rho, rhoM};
    double Dmax = (nD - 1) * hD;
    int per[3] = {per0, per1, per2};
    int Mx[3];
    for (int a = 0; a < 3; ++a) {
        double bl = sqrt(B[3 * a] * B[3 * a] + B[3 * a + 1] * B[3 * a + 1] + B[3 * a + 2] * B[3 * a + 2]);
        Mx[a] = per[a] ? (int)ceil(rc * bl) + 1 : 0;
    }
    int N[3] = {n0, n1, n2};
    double phi00 = f[0];
#pragma omp parallel for schedule(dynamic, 4)
    for (int t = 0; t < nq; ++t) {
        int i = qidx[t];
        double ri[3], a_ = 0.0, u_ = 0.0;
        int64_t cnt = 0;
        int cl = 0;
        int ii[3] = {i0[i], i1[i], i2[i]};
        for (int c = 0; c < 3; ++c)
            ri[c] = ii[0] / (double)N[0] * cell[c] + ii[1] / (double)N[1] * cell[3 + c] +
                    ii[2] / (double)N[2] * cell[6 + c];
        for (int j = 0; j < Na; ++j) {
            int jj[3] = {i0[j], i1[j], i2[j]};
            double rj[3];
            for (int c = 0; c < 3; ++c)
                rj[c] = jj[0] / (double)N[0] * cell[c] + jj[1] / (double)N[1] * cell[3 + c] +
                        jj[2] / (double)N[2] * cell[6 + c];
            for (int m0 = -Mx[0]; m0 <= Mx[0]; ++m0)
                for (int m1 = -Mx[1]; m1 <= Mx[1]; ++m1)
                    for (int m2 = -Mx[2]; m2 <= Mx[2]; ++m2) {
                        if (j == i && m0 == 0 && m1 == 0 && m2 == 0) {
                            a_ += n[i] * phi00;
                            continue;
                        }
                        double d[3];
                        for (int c = 0; c < 3; ++c)
                            d[c] = ri[c] - rj[c] + m0 * cell[c] + m1 * cell[3 + c] + m2 * cell[6 + c];
                        double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                        if (rc > 0.0 && r2 > rc * rc * (1.0 + 1e-12)) continue;
                        double p, rd;
                        kernel_pair(&s, Dmax, sqrt(r2), q[i], q[j], &p, &rd, &cl);
                        a_ += n[j] * p;
                        u_ += n[j] * rd;
                        ++cnt;
                    }
        }
        A[t] = a_;
        U[t] = n[i] * u_;
        if (npairs) npairs[t] = cnt;
        if (nclamp) nclamp[t] = cl;
    }
    return 0;
}

/* Gradient on a general cell: the 4th-order central difference along grid
 * axis a gives df/du_a (u_a = i_a / N_a, the fractional coordinate), and
 * grad f = sum_a (df/du_a) B_a.  g is [3][N], Cartesian. */
int orc_gradient_cell(int n0, int n1, int n2, const double *cell, const double *f, double *g)
{
    double B[9];
    if (cell_recip(cell, B)) return -1;
    size_t N = (size_t)n0 * n1 * n2;
    int dims[3] = {n0, n1, n2};
#pragma omp parallel for collapse(2) schedule(static)
    for (int a = 0; a < n0; ++a)
        for (int b = 0; b < n1; ++b)
            for (int c = 0; c < n2; ++c) {
                int idx[3] = {a, b, c};
                size_t m = ((size_t)a * n1 + b) * n2 + c;
                double du[3];
                for (int ax = 0; ax < 3; ++ax) {
                    double s = 0.0;
                    for (int o = -2; o <= 2; ++o) {
                        int jj[3] = {idx[0], idx[1], idx[2]};
                        jj[ax] = ((idx[ax] + o) % dims[ax] + dims[ax]) % dims[ax];
                        s += orc_fd_c[o + 2] * f[((size_t)jj[0] * n1 + jj[1]) * n2 + jj[2]];
                    }
                    du[ax] = s * dims[ax];
                }
                for (int k = 0; k < 3; ++k) g[k * N + m] = du[0] * B[k] + du[1] * B[3 + k] + du[2] * B[6 + k];
            }
    return 0;
}

/* The transpose of orc_gradient_cell: out = sum_a D_a^T (sum_k B_a[k] w_k),
 * D_a the index stencil times N_a; w is [3][N], Cartesian. */
int orc_gradient_T_cell(int n0, int n1, int n2, const double *cell, const double *w, double *out)
{
    double B[9];
    if (cell_recip(cell, B)) return -1;
    size_t N = (size_t)n0 * n1 * n2;
    int dims[3] = {n0, n1, n2};
#pragma omp parallel for collapse(2) schedule(static)
    for (int a = 0; a < n0; ++a)
        for (int b = 0; b < n1; ++b)
            for (int c = 0; c < n2; ++c) {
                int idx[3] = {a, b, c};
                size_t m = ((size_t)a * n1 + b) * n2 + c;
                double s = 0.0;
                for (int ax = 0; ax < 3; ++ax)
                    for (int o = -2; o <= 2; ++o) {
                        int jj[3] = {idx[0], idx[1], idx[2]};
                        jj[ax] = ((idx[ax] - o) % dims[ax] + dims[ax]) % dims[ax];
                        size_t mm = ((size_t)jj[0] * n1 + jj[1]) * n2 + jj[2];
                        double wa = B[3 * ax] * w[mm] + B[3 * ax + 1] * w[N + mm] + B[3 * ax + 2] * w[2 * N + mm];
                        s += orc_fd_c[o + 2] * dims[ax] * wa;
                    }
                out[m] = s;
            }
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Voxel-averaged diagonal ("phi0").  The paper's Appendix A output shows   */
/* a separate diagonal step (nphi0, E_DIAG_nlc) but the paper does not     */
/* describe it.  Reading: with n and q0 constant over voxel i, the i = j,  */
/* L = 0 term of eq. (1) is 1/2 n_i^2 dV^2 phi0(q_i) with                 */
/*   phi0(q) = int_{[-1,1]^3} prod_a (1 - |t_a|) phi_0(q |sum_a t_a v_a|) d^3t, */
/* the kernel at delta = 0 averaged over pairs of points of one voxel      */
/* (v_a = M_a / N_a: r - r' = sum_a t_a v_a with t_a the difference of two */
/* uniform variables, density 1 - |t_a|).  phi_0(D) is the kernel of       */
/* orc_kernel_many at delta = 0 for D >= D_1 (first table node after 0);    */
/* below D_1, where eq. (14) diverges like -(2/pi) ln D and the table's row */
/* 0 is softened, phi_0 = -(2/pi) ln D + psi0 + c2 D^2 with psi = phi +     */
/* (2/pi) ln D fitted at the nodes D_1, D_2 (psi0 = (4 psi1 - psi2)/3,      */
/* c2 = (psi1 - psi0) / D_1^2).  The singularity is integrable.            */
/* Quadrature: the eight sign octants of t, in each a tensor Gauss-Legendre */
/* rule on geometric panels [0, 2^-(P-1)], ..., [1/4, 1/2], [1/2, 1] per     */
/* axis (np points per panel), graded towards the singular corner t = 0.   */
/* ---------------------------------------------------------------------- */
static double phi_delta0(const orc_spline *s, double Dmax, double D, double D1, double psi0, double c2)
{
    if (D < D1) return -(2.0 / M_PI) * log(D) + psi0 + c2 * D * D;
    double p, rd;
    int cl = 0;
    kernel_pair(s, Dmax, D, 1.0, 1.0, &p, &rd, &cl);
    return p;
}

int orc_phi0_many(int nD, double hD, int nd, double hd, const double *f,
                  const double *fDD, const double *fdd, const double *fDDdd,
                  const double *rho, const double *rhoM, const double *vox,
                  int nq, const double *q, double *out, int panels, int np)
{
    if (panels < 1 || np < 1 || np > 64 || nD < 3) return -1;
    orc_spline s = {nD, nd, hD, hd, f, fDD, fdd, fDDdd, rho, rhoM};
    double Dmax = (nD - 1) * hD;
    double D1 = hD, D2 = 2.0 * hD;
    double psi1 = f[(size_t)1 * nd] + (2.0 / M_PI) * log(D1);
    double psi2 = f[(size_t)2 * nd] + (2.0 / M_PI) * log(D2);
    double psi0 = (4.0 * psi1 - psi2) / 3.0;
    double c2 = (psi1 - psi0) / (D1 * D1);
    /* 1-D composite rule on [0, 1] */
    double gx[64], gw[64];
    gl_rule(np, gx, gw);
    int nn = panels * np;
    double *x = (double *)malloc(sizeof(double) * nn), *w = (double *)malloc(sizeof(double) * nn);
    if (!x || !w) { free(x); free(w); return -2; }
    for (int p = 0; p < panels; ++p) {
        double a = (p == 0) ? 0.0 : ldexp(1.0, p - panels);
        double b = ldexp(1.0, p + 1 - panels);
        for (int k = 0; k < np; ++k) {
            /* gl_rule gives nodes and weights on [-1, 1] */
            x[p * np + k] = 0.5 * (a + b) + 0.5 * (b - a) * gx[k];
            w[p * np + k] = 0.5 * (b - a) * gw[k];
        }
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int t = 0; t < nq; ++t) {
        double acc = 0.0;
        for (int sg = 0; sg < 8; ++sg) {
            double s0 = (sg & 1) ? -1.0 : 1.0, s1 = (sg & 2) ? -1.0 : 1.0, s2 = (sg & 4) ? -1.0 : 1.0;
            for (int i = 0; i < nn; ++i)
                for (int j = 0; j < nn; ++j)
                    for (int k = 0; k < nn; ++k) {
                        double t0 = s0 * x[i], t1 = s1 * x[j], t2 = s2 * x[k];
                        double r[3];
                        for (int c = 0; c < 3; ++c) r[c] = t0 * vox[c] + t1 * vox[3 + c] + t2 * vox[6 + c];
                        double D = q[t] * sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
                        double wt = w[i] * w[j] * w[k] * (1.0 - x[i]) * (1.0 - x[j]) * (1.0 - x[k]);
                        acc += wt * phi_delta0(&s, Dmax, D, D1, psi0, c2);
                    }
        }
        out[t] = acc;
    }
    free(x);
    free(w);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* I(rho, x0) = int_{x0}^inf dx / (rho^2 + x^2)^3, rho >= 0, x0 >= 0, not   */
/* both 0: the continuum of one periodic axis (orc_far_tail).               */
/*  - x0 = 0: 3 pi / (16 rho^5).                                            */
/*  - rho / x0 = e < 1/2: with x = x0 t, (t^2 + e^2)^-3 = t^-6 (1 + e^2 / t^2)^-3 */
/*    expands by the binomial series into sum_k (-1)^k C(k+2, 2) e^2k t^-(6+2k), */
/*    and term by term over [1, inf): I = x0^-5 sum_k (-1)^k C(k+2, 2) e^2k / (2k + 5). */
/*  - otherwise the antiderivative of (rho^2 + x^2)^-3 (two steps of the     */
/*    reduction formula for int dx / (x^2 + a^2)^n),                         */
/*      x / (4 rho^2 (rho^2 + x^2)^2) + 3 x / (8 rho^4 (rho^2 + x^2))         */
/*      + 3 / (8 rho^5) atan(x / rho),                                       */
/*    taken from x0 to infinity.  The series avoids its cancellation when    */
/*    rho is small beside x0.                                               */
/* ---------------------------------------------------------------------- */
double orc_line_tail_integral(double rho, double x0)
{
    if (!(x0 > 0.0)) return 3.0 * M_PI / (16.0 * pow(rho, 5));
    double e = rho / x0;
    if (e < 0.5) {
        double sum = 0.0, p = 1.0;
        for (int k = 0; k < 80; ++k) {
            double term = 0.5 * (k + 1.0) * (k + 2.0) * p / (2.0 * k + 5.0);
            sum += (k % 2) ? -term : term;
            if (term < 1e-19) break;
            p *= e * e;
        }
        return sum / pow(x0, 5);
    }
    double r2 = rho * rho, s2 = r2 + x0 * x0;
    return 3.0 / (8.0 * pow(rho, 5)) * atan(rho / x0) - x0 / (4.0 * r2 * s2 * s2) -
           3.0 * x0 / (8.0 * r2 * r2 * s2);
}

/* The continuum factor K_ij of the far field (orc_far_tail) for the pair of  */
/* points at ri, rj; geometry from far_geometry.                             */
typedef struct {
    int np;          /* periodic axes: 1, 2 or 3                               */
    double V;        /* cell volume                                            */
    double A;        /* two axes: |a x b|                                      */
    double alen;     /* one axis: |a|                                          */
    double e[3];     /* two axes: unit normal of the periodic plane; one axis:  */
                     /* unit vector along the periodic lattice vector         */
} far_geom;

static int far_geometry(const double *cell, const int per[3], far_geom *g)
{
    const double *M0 = cell, *M1 = cell + 3, *M2 = cell + 6;
    const double *P[3] = {M0, M1, M2};
    g->np = (per[0] != 0) + (per[1] != 0) + (per[2] != 0);
    double x01[3] = {M0[1] * M1[2] - M0[2] * M1[1], M0[2] * M1[0] - M0[0] * M1[2], M0[0] * M1[1] - M0[1] * M1[0]};
    g->V = fabs(x01[0] * M2[0] + x01[1] * M2[1] + x01[2] * M2[2]);
    if (!(g->V > 0.0) || g->np < 1) return -1;
    g->A = 0.0;
    g->alen = 0.0;
    g->e[0] = g->e[1] = g->e[2] = 0.0;
    if (g->np == 2) {
        const double *a = NULL, *b = NULL;
        for (int k = 0; k < 3; ++k)
            if (per[k]) { if (!a) a = P[k]; else b = P[k]; }
        double x[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
        g->A = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
        for (int c = 0; c < 3; ++c) g->e[c] = x[c] / g->A;
    } else if (g->np == 1) {
        const double *a = per[0] ? M0 : (per[1] ? M1 : M2);
        g->alen = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
        for (int c = 0; c < 3; ++c) g->e[c] = a[c] / g->alen;
    }
    return 0;
}

static double far_K(const far_geom *g, const double ri[3], const double rj[3], double rc)
{
    if (g->np == 3) return (4.0 * M_PI / g->V) / (3.0 * rc * rc * rc);
    double d[3] = {ri[0] - rj[0], ri[1] - rj[1], ri[2] - rj[2]};
    double z = d[0] * g->e[0] + d[1] * g->e[1] + d[2] * g->e[2];
    if (g->np == 2) {
        double R = fabs(z) > rc ? fabs(z) : rc;
        return (2.0 * M_PI / g->A) / (4.0 * R * R * R * R);
    }
    /* one axis: rho the distance from the line through rj along the axis.  x0 has  */
    /* a square-root singularity at rho = rc, where many grid pairs sit exactly;   */
    /* as the pair sum's inclusive cutoff does, rc^2 - rho^2 within 1e-12 rc^2 of   */
    /* zero counts as zero, so that rounding does not decide those pairs.          */
    double p2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] - z * z;
    double rho = p2 > 0.0 ? sqrt(p2) : 0.0;
    double t = rc * rc - p2;
    double x0 = t > 1e-12 * rc * rc ? sqrt(t) : 0.0;
    return (2.0 / g->alen) * orc_line_tail_integral(rho, x0);
}

/* ---------------------------------------------------------------------- */
/* Far field past the cutoff from the asymptote alone.  Section 7 names      */
/* image sums sped up by the kernel's asymptotic form as future work;       */
/* sections 3 and 6.2 repeat the cell until the energy converges.           */
/* Reading: every pair beyond r_cut takes eq. (17),                          */
/*   phi17 = -C / (q_i^2 q_j^2 (q_i^2 + q_j^2) r^6),                          */
/* and the lattice images beyond r_cut are replaced by the lattice's        */
/* continuum (images per unit area or volume):                              */
/*   two periodic axes a, b (area A = |a x b|, unit normal e):              */
/*     sum_{L : |d + L| > rc} g(|d + L|)                                    */
/*       -> (1/A) int_{rho^2 + z^2 > rc^2} g(sqrt(rho^2 + z^2)) d^2 rho      */
/*        = (2 pi / A) int_{R}^inf g(r) r dr,  z = d . e,  R = max(rc, |z|), */
/*     which for g = r^-6 is (2 pi / A) / (4 R^4);                           */
/*   three periodic axes (volume V): (4 pi / V) int_rc^inf g(r) r^2 dr       */
/*     = (4 pi / V) / (3 rc^3);                                             */
/*   one periodic axis a (length |a|): with rho the distance of d from the  */
/*   axis direction and x the coordinate along it,                          */
/*     sum_{m : |d + m a| > rc} g(|d + m a|)                                */
/*       -> (1/|a|) int_{rho^2 + x^2 > rc^2} g(sqrt(rho^2 + x^2)) dx         */
/*        = (2 / |a|) I(rho, x0),  x0 = sqrt(max(0, rc^2 - rho^2)),          */
/*     I from orc_line_tail_integral for g = r^-6 (rc^2 - rho^2 below       */
/*     1e-12 rc^2 counts as 0, see far_K).                                  */
/* So the tail is                                                           */
/*   T = 1/2 dV^2 sum_i sum_j n_i n_j (-C / (q_i^2 q_j^2 (q_i^2 + q_j^2))) K_ij */
/* over all ordered pairs of active points, i = j included (the self term's */
/* own images), and E(r_cut -> inf) is read as E(r_cut) + T.  Open cells    */
/* have no lattice images: returns -1.                                      */
/* Points i at fractional index (i0/n0, i1/n1, i2/n2) of the cell (rows of  */
/* `cell` are the lattice vectors).                                          */
/* ---------------------------------------------------------------------- */
int orc_far_tail(int Na, const int32_t *i0, const int32_t *i1, const int32_t *i2,
                 const double *n, const double *q, int n0, int n1, int n2, const double *cell,
                 int per0, int per1, int per2, double rc, double *out)
{
    int per[3] = {per0, per1, per2};
    far_geom g;
    if (far_geometry(cell, per, &g) != 0 || !(rc > 0.0)) return -1;
    const double C = 12.0 * pow(4.0 * M_PI / 9.0, 3);
    const double *M0 = cell, *M1 = cell + 3, *M2 = cell + 6;
    int N[3] = {n0, n1, n2};
    double dV = g.V / ((double)n0 * n1 * n2);
    double sum = 0.0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : sum)
    for (int i = 0; i < Na; ++i) {
        double ri[3];
        for (int c = 0; c < 3; ++c)
            ri[c] = i0[i] / (double)N[0] * M0[c] + i1[i] / (double)N[1] * M1[c] + i2[i] / (double)N[2] * M2[c];
        double ui = q[i] * q[i];
        double acc = 0.0;
        for (int j = 0; j < Na; ++j) {
            double rj[3];
            for (int c = 0; c < 3; ++c)
                rj[c] = i0[j] / (double)N[0] * M0[c] + i1[j] / (double)N[1] * M1[c] + i2[j] / (double)N[2] * M2[c];
            double uj = q[j] * q[j];
            double K = far_K(&g, ri, rj, rc);
            acc += n[j] * (-C / (ui * uj * (ui + uj))) * K;
        }
        sum += n[i] * acc;
    }
    *out = 0.5 * dV * dV * sum;
    return 0;
}

/* The far field's own potential: with f(a, b) = 1 / (a b (a + b)), u = q0^2,
 *   T = -1/2 dV^2 C sum_i sum_j n_i n_j f(u_i, u_j) K_ij   (orc_far_tail),
 * so, for query points m,
 *   AT_m = sum_j n_j f(u_m, u_j) K_mj         (dT/dn_m = -dV^2 C AT_m),
 *   BT_m = sum_j n_j df/da(u_m, u_j) K_mj,    df/da = -f (1/a + 1/(a + b))
 *                                             (dT/du_m = -dV^2 C n_m BT_m).
 * Same points, cell and K_ij as orc_far_tail; returns -1 likewise. */
int orc_far_tail_AB(int Na, const int32_t *i0, const int32_t *i1, const int32_t *i2,
                    const double *n, const double *q, int n0, int n1, int n2, const double *cell,
                    int per0, int per1, int per2, double rc, int nq, const int32_t *qidx,
                    double *AT, double *BT)
{
    int per[3] = {per0, per1, per2};
    far_geom g;
    if (far_geometry(cell, per, &g) != 0 || !(rc > 0.0)) return -1;
    const double *M0 = cell, *M1 = cell + 3, *M2 = cell + 6;
    int N[3] = {n0, n1, n2};
#pragma omp parallel for schedule(dynamic, 4)
    for (int t = 0; t < nq; ++t) {
        int i = qidx[t];
        double ri[3];
        for (int c = 0; c < 3; ++c)
            ri[c] = i0[i] / (double)N[0] * M0[c] + i1[i] / (double)N[1] * M1[c] + i2[i] / (double)N[2] * M2[c];
        double ui = q[i] * q[i];
        double sa = 0.0, sb = 0.0;
        for (int j = 0; j < Na; ++j) {
            double rj[3];
            for (int c = 0; c < 3; ++c)
                rj[c] = i0[j] / (double)N[0] * M0[c] + i1[j] / (double)N[1] * M1[c] + i2[j] / (double)N[2] * M2[c];
            double uj = q[j] * q[j];
            double K = far_K(&g, ri, rj, rc);
            double f = 1.0 / (ui * uj * (ui + uj));
            sa += n[j] * f * K;
            sb += n[j] * (-f * (1.0 / ui + 1.0 / (ui + uj))) * K;
        }
        AT[t] = sa;
        BT[t] = sb;
    }
    return 0;
}
