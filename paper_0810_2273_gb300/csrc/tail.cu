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
// s = e^x and the trapezoidal rule in x (step hx; the integrand is analytic in
// the strip |Im x| < pi/2, so the error falls like exp(-pi^2 / hx)),
//   T = -1/2 dV^2 C sum_k hx s_k sum_{p, p'} K(p, p') F_k(p) F_k(p'),
//   F_k(p) = sum over active points of plane p of (n / u) exp(-u s_k).
// That is O(N_grid x nodes) work for the planes and O(planes^2 x nodes) for the
// pairs of planes, instead of O(N_active^2): a few milliseconds in FP64.  Its
// potential (the derivative of T with the active mask frozen) comes from the
// same sums, point by point (k_tail_AU), in the pair sum's adjoint form.
#include <cuda_runtime.h>

#include "common.cuh"

namespace vdwdf {

namespace {

constexpr int kTailChunk = 16;     // quadrature nodes per block of k_tail_planes
constexpr int kTailThreads = 256;

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
        if (np > 1) {
            const long long c2i = m % d2, c1i = (m / d2) % d1, c0i = m / (static_cast<long long>(d1) * d2);
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

}  // namespace

int launch_far_tail_AU(const int dims[3], int ax, int np, const double *n, const double *q0, double n_cut,
                       double x0, double hx, int nodes, const double *G, double C, int *slot, double *A,
                       double *U, cudaStream_t st) {
    const long long N = static_cast<long long>(dims[0]) * dims[1] * dims[2];
    long long nb = (N + kTailThreads - 1) / kTailThreads;
    if (nb > 152 * 16) nb = 152 * 16;
    const size_t smem = sizeof(double) * static_cast<size_t>(nodes);  // at most 32 KB (4096 nodes)
    k_tail_AU<<<static_cast<int>(nb), kTailThreads, smem, st>>>(dims[0], dims[1], dims[2], ax, np, n, q0, n_cut,
                                                                x0, hx, nodes, G, C, slot, A, U);
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
