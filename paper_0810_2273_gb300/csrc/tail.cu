// Far field past the pair cutoff from the kernel's asymptote alone (the paper's
// section 7 names image sums sped up by the asymptotic form as future work;
// sections 3 and 6.2 repeat the cell until the energy converges).
//
// Every pair beyond r_cut takes eq. (17), phi17 = -C / (u_i u_j (u_i + u_j) r^6)
// with u = q0^2, and the lattice images beyond r_cut are replaced by the
// lattice's continuum.  Per pair of points that gives
//   K_ij = (2 pi / A) / (4 max(r_cut, |z_ij|)^4)   (two periodic axes, area A,
//          z_ij the separation normal to the periodic plane),
//   K    = (4 pi / V) / (3 r_cut^3)                 (three periodic axes),
// and the tail T = 1/2 dV^2 sum_ij n_i n_j (-C / (u_i u_j (u_i + u_j))) K_ij.
//
// On the grid, z depends only on the plane of the non-periodic axis, and
// 1/(u_i + u_j) = int_0^inf exp(-(u_i + u_j) s) ds separates i from j.  With
// s = e^x and the trapezoidal rule in x (step hx = 0.3; the integrand is analytic
// in the strip |Im x| < pi/2, so the error falls like exp(-pi^2 / hx)),
//   T = -1/2 dV^2 C sum_k hx s_k sum_{p, p'} K(p, p') F_k(p) F_k(p'),
//   F_k(p) = sum over active points of plane p of (n / u) exp(-u s_k).
// That is O(N_grid x nodes) work for the planes and O(planes^2 x nodes) for the
// pairs of planes, instead of O(N_active^2): a few milliseconds in FP64.  Its
// potential (the derivative of T with the active mask frozen) comes from the
// same sums, point by point (k_tail_AU), in the pair sum's adjoint form.
//
// One periodic axis a (length |a|): the images of a pair lie on a line, and
// their continuum beyond r_cut gives
//   K_ij = (2 / |a|) I(rho_ij, x0),  I(rho, x0) = int_{x0}^inf dx / (rho^2 + x^2)^3,
// rho_ij the distance of r_i - r_j from the axis direction and
// x0 = sqrt(max(0, r_cut^2 - rho^2)).  rho depends only on the grid lines along
// a that hold i and j, so the lines take the place of the planes: F_k per
// line with an active point, K as a table over the lines' index differences
// (k_tail_line_Ktab), G_k = K F_k as a tiled FP64 product (k_tail_line_G).
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"

namespace vdwdf {

namespace {

constexpr int kTailChunk = 16;     // quadrature nodes per block of k_tail_planes
constexpr int kTailThreads = 256;

constexpr double kTailPi = 3.14159265358979323846;

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Grid index of the t-th point of plane p (the points whose index along axis
// `ax` is p); one plane holding every point when np == 1.
__device__ __forceinline__ long long plane_point(int d0, int d1, int d2, int ax, int np, int p, long long t) {
    if (np == 1) return t;
    if (ax == 0) return static_cast<long long>(p) * d1 * d2 + t;
    if (ax == 1) return (t / d2 * d1 + p) * static_cast<long long>(d2) + t % d2;
    return t * d2 + p;
}

// F[k * np + p] for the kTailChunk nodes k of blockIdx.y; one block per plane p,
// sums in a fixed order (threads stride the plane, then warp and block trees).
__global__ void __launch_bounds__(kTailThreads) k_tail_planes(int d0, int d1, int d2, int ax, int np,
                                                              const double *__restrict__ n,
                                                              const double *__restrict__ q0, double n_cut,
                                                              double x0, double hx, int nodes,
                                                              double *__restrict__ F) {
    __shared__ double s_k[kTailChunk];
    __shared__ double red[kTailThreads / 32][kTailChunk];
    const int p = blockIdx.x;
    const int k0 = blockIdx.y * kTailChunk;
    if (threadIdx.x < kTailChunk) s_k[threadIdx.x] = exp(x0 + hx * (k0 + static_cast<int>(threadIdx.x)));
    __syncthreads();
    const long long per_plane = (np == 1) ? static_cast<long long>(d0) * d1 * d2
                                          : static_cast<long long>(d0) * d1 * d2 / np;
    double acc[kTailChunk];
#pragma unroll
    for (int c = 0; c < kTailChunk; ++c) acc[c] = 0.0;
    for (long long t = threadIdx.x; t < per_plane; t += blockDim.x) {
        const long long m = plane_point(d0, d1, d2, ax, np, p, t);
        const double nm = n[m];
        if (!(nm >= n_cut)) continue;  // inactive (NaN as well)
        const double q = q0[m];
        const double u = q * q;
        const double a = nm / u;
#pragma unroll
        for (int c = 0; c < kTailChunk; ++c) acc[c] += a * exp(-u * s_k[c]);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < kTailChunk; ++c) {
        const double v = warp_sum_d(acc[c]);
        if (lane == 0) red[warp][c] = v;
    }
    __syncthreads();
    if (threadIdx.x < kTailChunk && k0 + static_cast<int>(threadIdx.x) < nodes) {
        double s = 0.0;
        for (int w = 0; w < kTailThreads / 32; ++w) s += red[w][threadIdx.x];
        F[static_cast<long long>(k0 + threadIdx.x) * np + p] = s;
    }
}

// Tk[k] = sum_{p, p'} K(p, p') F_k(p) F_k(p') for node k = blockIdx.x, with
// K(p, p') = c2 / max(rc, |p - p'| dz)^4 (two periodic axes) or c3 (three);
// G (when given) keeps G_k(p) = sum_{p'} K(p, p') F_k(p') for the potential.
__global__ void __launch_bounds__(kTailThreads) k_tail_pairs(int np, const double *__restrict__ F, double dz,
                                                             double rc, double c2, double c3,
                                                             double *__restrict__ Tk, double *__restrict__ G) {
    __shared__ double red[kTailThreads / 32];
    const double *f = F + static_cast<long long>(blockIdx.x) * np;
    double acc = 0.0;
    for (int p = threadIdx.x; p < np; p += blockDim.x) {
        double row = 0.0;
        for (int pp = 0; pp < np; ++pp) {
            double K = c3;
            if (np > 1) {
                const double z = fabs(static_cast<double>(p - pp)) * dz;
                const double R = z > rc ? z : rc;
                const double R2 = R * R;
                K = c2 / (R2 * R2);
            }
            row += K * f[pp];
        }
        if (G) G[static_cast<long long>(blockIdx.x) * np + p] = row;
        acc += f[p] * row;
    }
    acc = warp_sum_d(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kTailThreads / 32; ++w) s += red[w];
        Tk[blockIdx.x] = s;
    }
}

// out = scale * sum_k hx s_k Tk[k], in node order.
__global__ void k_tail_final(int nodes, const double *__restrict__ Tk, double x0, double hx, double scale,
                             double *__restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0.0;
    for (int k = 0; k < nodes; ++k) s += hx * exp(x0 + hx * k) * Tk[k];
    *out = scale * s;
}

// The far field's potential in the pair sum's adjoint form, per grid point m:
// with S0 = sum_k hx s_k e^{-u s_k} G_k(p) and S1 = sum_k hx s_k^2 e^{-u s_k} G_k(p)
// (u = q0_m^2, p the plane of m),
//   sum_j n_j f(u, u_j) K_mj = S0 / u,   sum_j n_j df/du K_mj = -S0 / u^2 - S1 / u,
// f(a, b) = 1 / (a b (a + b)), since 1/(a + b) and 1/(a + b)^2 are the integrals of
// e^{-(a + b) s} and s e^{-(a + b) s}.  A = -C S0 / u and U = -2 C n q (-S0/u^2 - S1/u)
// at active points (slot[m] = m), slot[m] = -1 elsewhere.
__global__ void __launch_bounds__(kTailThreads) k_tail_AU(int d0, int d1, int d2, int ax, int np,
                                                          const int *__restrict__ line_slot,
                                                          const double *__restrict__ n,
                                                          const double *__restrict__ q0, double n_cut, double x0,
                                                          double hx, int nodes, const double *__restrict__ G,
                                                          double C, int *__restrict__ slot,
                                                          double *__restrict__ A, double *__restrict__ U) {
    extern __shared__ double s_nodes[];  // s_k = e^{x0 + k hx}, k < nodes
    for (int k = threadIdx.x; k < nodes; k += blockDim.x) s_nodes[k] = exp(x0 + hx * k);
    __syncthreads();
    const long long N = static_cast<long long>(d0) * d1 * d2;
    for (long long m = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; m < N;
         m += static_cast<long long>(gridDim.x) * blockDim.x) {
        const double nm = n[m];
        if (!(nm >= n_cut)) {
            slot[m] = -1;
            continue;
        }
        int p = 0;
        const long long c2i = m % d2, c1i = (m / d2) % d1, c0i = m / (static_cast<long long>(d1) * d2);
        if (line_slot) {
            // one periodic axis: the active line of m
            const long long ib = ax == 0 ? c1i : c0i, ic = ax == 2 ? c1i : c2i;
            p = line_slot[ib * (ax == 2 ? d1 : d2) + ic];
        } else if (np > 1) {
            p = static_cast<int>(ax == 0 ? c0i : (ax == 1 ? c1i : c2i));
        }
        const double q = q0[m];
        const double u = q * q;
        double S0 = 0.0, S1 = 0.0;
        for (int k = 0; k < nodes; ++k) {
            const double s = s_nodes[k];
            const double t = hx * s * exp(-u * s) * G[static_cast<long long>(k) * np + p];
            S0 += t;
            S1 += s * t;
        }
        slot[m] = static_cast<int>(m);
        A[m] = -C * S0 / u;
        U[m] = -2.0 * C * nm * q * (-S0 / (u * u) - S1 / u);
    }
}

// ---------------------------------------------------------------------------
// one periodic axis: lines along it
// ---------------------------------------------------------------------------

// The grid index of the t-th point of line (ib, ic) along ax.
__device__ __forceinline__ long long line_point(int d1, int d2, int ax, int ib, int ic, long long t) {
    if (ax == 0) return (t * d1 + ib) * static_cast<long long>(d2) + ic;
    if (ax == 1) return (static_cast<long long>(ib) * d1 + t) * d2 + ic;
    return (static_cast<long long>(ib) * d1 + ic) * d2 + t;
}

// The line (ib * N_c + ic) of grid point m.
__device__ __forceinline__ long long line_of(int d1, int d2, int ax, long long m) {
    const long long i2 = m % d2, i1 = (m / d2) % d1, i0 = m / (static_cast<long long>(d1) * d2);
    const long long ib = ax == 0 ? i1 : i0, ic = ax == 2 ? i1 : i2;
    return ib * (ax == 2 ? d1 : d2) + ic;
}

// flags[line] = 1 where the line holds an active point (the line of grid point m
// is ib * Nc + ic).
__global__ void k_tail_line_flags(int d0, int d1, int d2, int ax, const double *__restrict__ n, double n_cut,
                                  int *__restrict__ flags) {
    const long long N = static_cast<long long>(d0) * d1 * d2;
    for (long long m = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; m < N;
         m += static_cast<long long>(gridDim.x) * blockDim.x) {
        if (!(n[m] >= n_cut)) continue;
        flags[line_of(d1, d2, ax, m)] = 1;
    }
}

// F[k * La + a] = sum over active points of line lines[a] of (n / u) exp(-u s_k),
// one warp per line, nodes in chunks of kTailChunk (their s_k shared by the
// block), sums in a fixed order.
__global__ void __launch_bounds__(kTailThreads) k_tail_line_F(int d0, int d1, int d2, int ax, int La,
                                                              const int *__restrict__ lines,
                                                              const double *__restrict__ n,
                                                              const double *__restrict__ q0, double n_cut,
                                                              double x0, double hx, int nodes,
                                                              double *__restrict__ F) {
    __shared__ double s_k[kTailChunk];
    const int lane = threadIdx.x & 31;
    const int a = blockIdx.x * (kTailThreads / 32) + (threadIdx.x >> 5);
    const bool live = a < La;
    const int Nc = ax == 2 ? d1 : d2, len = ax == 0 ? d0 : (ax == 1 ? d1 : d2);
    const int l = live ? lines[a] : 0;
    const int ib = l / Nc, ic = l % Nc;
    for (int k0 = 0; k0 < nodes; k0 += kTailChunk) {
        __syncthreads();  // the previous chunk's s_k are read
        if (threadIdx.x < kTailChunk) s_k[threadIdx.x] = exp(x0 + hx * (k0 + static_cast<int>(threadIdx.x)));
        __syncthreads();
        if (!live) continue;
        double acc[kTailChunk];
#pragma unroll
        for (int u = 0; u < kTailChunk; ++u) acc[u] = 0.0;
        for (int t = lane; t < len; t += 32) {
            const long long m = line_point(d1, d2, ax, ib, ic, t);
            const double nm = n[m];
            if (!(nm >= n_cut)) continue;
            const double q = q0[m];
            const double u2 = q * q;
            const double w = nm / u2;
#pragma unroll
            for (int u = 0; u < kTailChunk; ++u) acc[u] += w * exp(-u2 * s_k[u]);
        }
#pragma unroll
        for (int u = 0; u < kTailChunk; ++u) {
            const double v = warp_sum_d(acc[u]);
            if (lane == 0 && k0 + u < nodes) F[static_cast<long long>(k0 + u) * La + a] = v;
        }
    }
}

// I(rho, x0) = int_{x0}^inf dx / (rho^2 + x^2)^3.  x0 = 0: 3 pi / (16 rho^5).  For
// e = rho / x0 < 1/2, x0^-5 sum_k (-1)^k (k+1)(k+2)/2 e^2k / (2k + 5) (the binomial
// series of (1 + e^2/t^2)^-3 integrated over t >= 1); otherwise the closed form
// 3 atan(rho / x0) / (8 rho^5) - x0 / (4 rho^2 s^2) - 3 x0 / (8 rho^4 s), s = rho^2 + x0^2.
__device__ double line_tail_I(double rho, double x0) {
    if (!(x0 > 0.0)) {
        const double r2 = rho * rho;
        return 3.0 * kTailPi / (16.0 * r2 * r2 * rho);
    }
    const double e = rho / x0;
    if (e < 0.5) {
        const double e2 = e * e;
        double sum = 0.0, p = 1.0;
        for (int k = 0; k < 80; ++k) {
            const double term = 0.5 * (k + 1.0) * (k + 2.0) * p / (2.0 * k + 5.0);
            sum += (k & 1) ? -term : term;
            if (term < 1e-19) break;
            p *= e2;
        }
        const double x2 = x0 * x0;
        return sum / (x2 * x2 * x0);
    }
    const double r2 = rho * rho, s = r2 + x0 * x0;
    return 3.0 * atan(e) / (8.0 * r2 * r2 * rho) - x0 / (4.0 * r2 * s * s) - 3.0 * x0 / (8.0 * r2 * r2 * s);
}

// Kt[db * (2 N_c - 1) + dc + N_c - 1] = K between two lines whose index differences
// are (db, dc), 0 <= db < N_b, |dc| < N_c: the squared distance through the metric
// (gbb, gbc, gcc) of the axis steps with their components along the periodic axis
// removed.  K depends on the lines only through (db, dc), and K(-db, -dc) = K(db, dc).
__global__ void k_tail_line_Ktab(int Nb, int Nc, double gbb, double gbc, double gcc, double rc, double pref,
                                 double *__restrict__ Kt) {
    const int W = 2 * Nc - 1;
    const long long total = static_cast<long long>(Nb) * W;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const double db = static_cast<double>(e / W), dc = static_cast<double>(e % W - (Nc - 1));
        double p2 = gbb * db * db + 2.0 * gbc * db * dc + gcc * dc * dc;
        p2 = p2 > 0.0 ? p2 : 0.0;
        // x0 = sqrt(rc^2 - rho^2) is singular at rho = rc, where lattice-aligned line
        // pairs sit exactly: a difference within 1e-12 rc^2 of zero counts as zero
        // (as the pair sum's inclusive cutoff), so rounding does not decide them
        const double x2 = rc * rc - p2;
        Kt[e] = pref * line_tail_I(sqrt(p2), x2 > 1e-12 * rc * rc ? sqrt(x2) : 0.0);
    }
}

// G[k * La + i] = sum_a K(lines[i], lines[a]) F[k * La + a] for every active line i
// and node k: a 32 x 32 output tile per block of 16 x 16 threads (2 x 2 each), the a
// range in shared-memory tiles of 32, K from the table Kt, summed in a fixed order.
constexpr int kGT = 32;
__global__ void __launch_bounds__(256) k_tail_line_G(int La, int nodes, const int *__restrict__ lines, int Nc,
                                                     const double *__restrict__ Kt, const double *__restrict__ F,
                                                     double *__restrict__ G) {
    __shared__ double sK[kGT][kGT + 1], sF[kGT][kGT + 1];
    __shared__ int rb[kGT], rcl[kGT];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int i0 = blockIdx.x * kGT, k0 = blockIdx.y * kGT;
    const int W = 2 * Nc - 1;
    if (threadIdx.x < kGT) {
        const int l = (i0 + threadIdx.x < La) ? lines[i0 + threadIdx.x] : 0;
        rb[threadIdx.x] = l / Nc;
        rcl[threadIdx.x] = l % Nc;
    }
    double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
    for (int a0 = 0; a0 < La; a0 += kGT) {
        __syncthreads();  // rb, rcl written; the previous tiles read
        for (int e = threadIdx.x; e < kGT * kGT; e += 256) {
            const int r = e / kGT, cc = e % kGT;
            const int i = i0 + r, k = k0 + r, a = a0 + cc;
            double kv = 0.0;
            if (i < La && a < La) {
                const int l2 = lines[a];
                int db = rb[r] - l2 / Nc, dc = rcl[r] - l2 % Nc;
                if (db < 0) {
                    db = -db;
                    dc = -dc;
                }
                kv = Kt[static_cast<long long>(db) * W + dc + Nc - 1];
            }
            sK[r][cc] = kv;
            sF[r][cc] = (k < nodes && a < La) ? F[static_cast<long long>(k) * La + a] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int j = 0; j < kGT; ++j) {
            const double k_0 = sK[ty][j], k_1 = sK[ty + 16][j];
            const double f_0 = sF[tx][j], f_1 = sF[tx + 16][j];
            acc[0][0] += k_0 * f_0;
            acc[0][1] += k_0 * f_1;
            acc[1][0] += k_1 * f_0;
            acc[1][1] += k_1 * f_1;
        }
    }
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 2; ++v) {
            const int i = i0 + ty + 16 * u, k = k0 + tx + 16 * v;
            if (i < La && k < nodes) G[static_cast<long long>(k) * La + i] = acc[u][v];
        }
}

// Tk[k] = sum_a F[k * La + a] G[k * La + a], one block per node, fixed order.
__global__ void __launch_bounds__(kTailThreads) k_tail_line_Tk(int La, const double *__restrict__ F,
                                                               const double *__restrict__ G,
                                                               double *__restrict__ Tk) {
    __shared__ double red[kTailThreads / 32];
    const long long base = static_cast<long long>(blockIdx.x) * La;
    double acc = 0.0;
    for (int a = threadIdx.x; a < La; a += blockDim.x) acc += F[base + a] * G[base + a];
    acc = warp_sum_d(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kTailThreads / 32; ++w) s += red[w];
        Tk[blockIdx.x] = s;
    }
}

}  // namespace

int launch_far_tail_line_flags(const int dims[3], int ax, const double *n, double n_cut, int *flags,
                               cudaStream_t st) {
    const long long N = static_cast<long long>(dims[0]) * dims[1] * dims[2];
    long long nb = (N + kTailThreads - 1) / kTailThreads;
    if (nb > 152 * 16) nb = 152 * 16;
    k_tail_line_flags<<<static_cast<int>(nb), kTailThreads, 0, st>>>(dims[0], dims[1], dims[2], ax, n, n_cut, flags);
    count_launches(1);
    VDWDF_CUDA_TRY(cudaGetLastError());
    return VDWDF_OK;
}

int launch_far_tail_lines(const int dims[3], int ax, int La, const int *lines, const double *n, const double *q0,
                          double n_cut, double x0, double hx, int nodes, double gbb, double gbc, double gcc,
                          double rc, double pref, double scale, double *F, double *Kt, double *G, double *Tk,
                          double *out, cudaStream_t st) {
    // lines are ib * N_c + ic, b < c the other two axes
    const int Nb = ax == 0 ? dims[1] : dims[0], Nc = ax == 2 ? dims[1] : dims[2];
    const int wpb = kTailThreads / 32;
    k_tail_line_F<<<(La + wpb - 1) / wpb, kTailThreads, 0, st>>>(dims[0], dims[1], dims[2], ax, La, lines, n, q0,
                                                                 n_cut, x0, hx, nodes, F);
    const long long kt = static_cast<long long>(Nb) * (2 * Nc - 1);
    k_tail_line_Ktab<<<static_cast<int>(std::min<long long>((kt + kTailThreads - 1) / kTailThreads, 152 * 8)),
                       kTailThreads, 0, st>>>(Nb, Nc, gbb, gbc, gcc, rc, pref, Kt);
    k_tail_line_G<<<dim3((La + kGT - 1) / kGT, (nodes + kGT - 1) / kGT), 256, 0, st>>>(La, nodes, lines, Nc, Kt, F,
                                                                                       G);
    k_tail_line_Tk<<<nodes, kTailThreads, 0, st>>>(La, F, G, Tk);
    k_tail_final<<<1, 32, 0, st>>>(nodes, Tk, x0, hx, scale, out);
    count_launches(5);
    VDWDF_CUDA_TRY(cudaGetLastError());
    return VDWDF_OK;
}

int launch_far_tail_AU(const int dims[3], int ax, int np, const int *line_slot, const double *n, const double *q0,
                       double n_cut, double x0, double hx, int nodes, const double *G, double C, int *slot,
                       double *A, double *U, cudaStream_t st) {
    const long long N = static_cast<long long>(dims[0]) * dims[1] * dims[2];
    long long nb = (N + kTailThreads - 1) / kTailThreads;
    if (nb > 152 * 16) nb = 152 * 16;
    const size_t smem = sizeof(double) * static_cast<size_t>(nodes);  // at most 32 KB (4096 nodes)
    k_tail_AU<<<static_cast<int>(nb), kTailThreads, smem, st>>>(dims[0], dims[1], dims[2], ax, np, line_slot, n, q0,
                                                                n_cut, x0, hx, nodes, G, C, slot, A, U);
    count_launches(1);
    VDWDF_CUDA_TRY(cudaGetLastError());
    return VDWDF_OK;
}

int launch_far_tail(const int dims[3], int ax, int np, const double *n, const double *q0, double n_cut,
                    double x0, double hx, int nodes, double dz, double rc, double c2, double c3, double scale,
                    double *F, double *Tk, double *G, double *out, cudaStream_t st) {
    const int chunks = (nodes + kTailChunk - 1) / kTailChunk;
    k_tail_planes<<<dim3(np, chunks), kTailThreads, 0, st>>>(dims[0], dims[1], dims[2], ax, np, n, q0, n_cut, x0,
                                                             hx, nodes, F);
    k_tail_pairs<<<nodes, kTailThreads, 0, st>>>(np, F, dz, rc, c2, c3, Tk, G);
    k_tail_final<<<1, 32, 0, st>>>(nodes, Tk, x0, hx, scale, out);
    count_launches(3);
    VDWDF_CUDA_TRY(cudaGetLastError());
    return VDWDF_OK;
}

}  // namespace vdwdf
