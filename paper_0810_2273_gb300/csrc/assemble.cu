// Assembly of the nonlocal potential on the grid from the per-point pair sums
// (the adjoint of the double sum of paper section 2 with the active mask of
// section 3 frozen):
//   dE/dn_m = dV^2 [chi_m (A_m + U_m dq0/dn_m) + sum_a (G_a^T w_a)_m],
//   w_a = chi U dq0/dg_a,
// where G_a is the periodic 4th-order central-difference stencil along grid
// axis a mapped to Cartesian components (on a general cell the gradient is
// sum_a (d/du_a) B_a, so w_a becomes sum_c S[3a + c] w_c).  The stencil is
// antisymmetric, so G_a^T w = -G_a w and
//   v_m = dE/dn_m / dV = dV [chi_m (A_m + U_m dq0/dn_m) - sum_a (G_a w_a)_m].
// Also E = 1/2 dV^2 sum_i n_i A_i.
#include <cuda_runtime.h>

#include "common.cuh"

namespace vdwdf {

namespace {

__device__ __forceinline__ int wrap(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}

__global__ void k_assemble(int n0, int n1, int n2, const AxisMap am, double dV,
                           const int *__restrict__ slot, const double *__restrict__ A,
                           const double *__restrict__ U, const double *__restrict__ qn,
                           const double *__restrict__ qg, const double *__restrict__ div_pre,
                           double *__restrict__ v, double *__restrict__ Ag, double *__restrict__ Ug) {
    const long long N = static_cast<long long>(n0) * n1 * n2;
    for (long long m = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; m < N;
         m += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int c = static_cast<int>(m % n2);
        const int b = static_cast<int>((m / n2) % n1);
        const int a = static_cast<int>(m / (static_cast<long long>(n1) * n2));
        const long long sa = static_cast<long long>(n1) * n2;
        // w along grid axis ax at a neighbour index (0 at inactive points): on a
        // diagonal cell U dq0/dg_ax, scaled below; on a general cell the
        // transpose of the axis map, sum_c S[3 ax + c] U dq0/dg_c
        auto w = [&](long long mm, int ax) {
            const int s = slot[mm];
            if (s < 0) return 0.0;
            if (!am.general) return U[s] * qg[ax * N + mm];
            return U[s] * (am.S[3 * ax] * qg[mm] + am.S[3 * ax + 1] * qg[N + mm] + am.S[3 * ax + 2] * qg[2 * N + mm]);
        };
        const double f0 = am.general ? 1.0 : am.S[0], f1 = am.general ? 1.0 : am.S[4],
                     f2 = am.general ? 1.0 : am.S[8];
        auto ia = [&](int aa) { return static_cast<long long>(wrap(aa, n0)) * sa + static_cast<long long>(b) * n2 + c; };
        auto ib = [&](int bb) { return static_cast<long long>(a) * sa + static_cast<long long>(wrap(bb, n1)) * n2 + c; };
        auto ic = [&](int cc) { return static_cast<long long>(a) * sa + static_cast<long long>(b) * n2 + wrap(cc, n2); };
        const double div = div_pre ? div_pre[m] :
            (8.0 * (w(ia(a + 1), 0) - w(ia(a - 1), 0)) - (w(ia(a + 2), 0) - w(ia(a - 2), 0))) * f0 +
            (8.0 * (w(ib(b + 1), 1) - w(ib(b - 1), 1)) - (w(ib(b + 2), 1) - w(ib(b - 2), 1))) * f1 +
            (8.0 * (w(ic(c + 1), 2) - w(ic(c - 1), 2)) - (w(ic(c + 2), 2) - w(ic(c - 2), 2))) * f2;
        const int s = slot[m];
        double loc = 0.0, av = 0.0, uv = 0.0;
        if (s >= 0) {
            av = A[s];
            uv = U[s];
            loc = av + uv * qn[m];
        }
        if (v) v[m] = dV * (loc - div);
        if (Ag) Ag[m] = av;
        if (Ug) Ug[m] = uv;
    }
}

__global__ void k_energy_from_A(int n_max, const double *__restrict__ A, const double *__restrict__ n64,
                                Stats *stats) {
    const int na = min(stats->n_active, n_max);
    double s = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < na; i += gridDim.x * blockDim.x)
        s += n64[i] * A[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ double ws[32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < static_cast<int>(blockDim.x >> 5); ++k) t += ws[k];
        atomicAdd(&stats->E_pair, t);
    }
}

// ---------------------------------------------------------------------------
// Voxel-averaged diagonal: grid passes over the points with n >= n_cut.
// ---------------------------------------------------------------------------
constexpr int kDiagBlocks = 608;
constexpr int kDiagThreads = 256;

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w < v ? w : v;
    }
    return v;
}
__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    return v;
}

// q0 > 0 at active points, so the bit patterns of the doubles order like the values
__global__ void k_diag_range(long long N, const double *__restrict__ n, const double *__restrict__ q0,
                             double n_cut, unsigned long long *mm) {
    unsigned long long lo = ~0ull, hi = 0ull, cnt = 0ull;
    for (long long m = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; m < N;
         m += static_cast<long long>(gridDim.x) * blockDim.x) {
        if (n[m] >= n_cut) {
            const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(q0[m]));
            lo = b < lo ? b : lo;
            hi = b > hi ? b : hi;
            ++cnt;
        }
    }
    lo = warp_min_u64(lo);
    hi = warp_max_u64(hi);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) {
        atomicMin(&mm[0], lo);
        atomicMax(&mm[1], hi);
        atomicAdd(&mm[2], cnt);
    }
}

__global__ void __launch_bounds__(kDiagThreads) k_diag_sum(long long N, const double *__restrict__ n,
                                                           const double *__restrict__ q0, double n_cut,
                                                           const double *__restrict__ tab, int nq,
                                                           double lnq0, double dlnq, double *__restrict__ part) {
    double s0 = 0.0, s1 = 0.0;
    for (long long m = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; m < N;
         m += static_cast<long long>(gridDim.x) * blockDim.x) {
        const double nn = n[m];
        if (!(nn >= n_cut)) continue;
        // 4-point Lagrange interpolation in ln q on the uniform table
        const double x = (log(q0[m]) - lnq0) / dlnq;
        int k = static_cast<int>(floor(x));
        k = max(1, min(nq - 3, k));
        const double u = x - k;
        const double lm = -u * (u - 1.0) * (u - 2.0) / 6.0, l0 = (u + 1.0) * (u - 1.0) * (u - 2.0) / 2.0,
                     l1 = -(u + 1.0) * u * (u - 2.0) / 2.0, l2 = (u + 1.0) * u * (u - 1.0) / 6.0;
        const double p0 = lm * tab[k - 1] + l0 * tab[k] + l1 * tab[k + 1] + l2 * tab[k + 2];
        s0 += nn * nn * p0;
        s1 += nn * nn;
    }
    __shared__ double r0[kDiagThreads], r1[kDiagThreads];
    r0[threadIdx.x] = s0;
    r1[threadIdx.x] = s1;
    __syncthreads();
    for (int o = kDiagThreads / 2; o > 0; o >>= 1) {
        if (static_cast<int>(threadIdx.x) < o) {
            r0[threadIdx.x] += r0[threadIdx.x + o];
            r1[threadIdx.x] += r1[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = r0[0];
        part[2 * blockIdx.x + 1] = r1[0];
    }
}

// Per grid point, for the potential of the voxel diagonal: with the active mask
// frozen, d/dn of 1/2 dV^2 sum_i n_i^2 (phi0(q_i) - phi(0,0)) has the form of the
// pair sum's adjoint with A_m = n_m (phi0(q_m) - phi00) and U_m = 1/2 n_m^2
// phi0'(q_m), so k_assemble turns these into the change of v.  phi0 and its
// derivative come from the 4-point Lagrange interpolant in ln q; slot[m] = m on
// active points, -1 elsewhere.
__global__ void k_diag_AU(long long N, const double *__restrict__ n, const double *__restrict__ q0,
                          double n_cut, const double *__restrict__ tab, int nq, double lnq0, double dlnq,
                          double phi00, int *__restrict__ slot, double *__restrict__ A, double *__restrict__ U) {
    for (long long m = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; m < N;
         m += static_cast<long long>(gridDim.x) * blockDim.x) {
        const double nn = n[m];
        if (!(nn >= n_cut)) {
            slot[m] = -1;
            A[m] = 0.0;
            U[m] = 0.0;
            continue;
        }
        const double q = q0[m];
        const double x = (log(q) - lnq0) / dlnq;
        int k = static_cast<int>(floor(x));
        k = max(1, min(nq - 3, k));
        const double u = x - k;
        const double lm = -u * (u - 1.0) * (u - 2.0) / 6.0, l0 = (u + 1.0) * (u - 1.0) * (u - 2.0) / 2.0,
                     l1 = -(u + 1.0) * u * (u - 2.0) / 2.0, l2 = (u + 1.0) * u * (u - 1.0) / 6.0;
        // d/du of the four Lagrange weights
        const double dm = -(3.0 * u * u - 6.0 * u + 2.0) / 6.0, d0 = (3.0 * u * u - 4.0 * u - 1.0) / 2.0,
                     d1 = -(3.0 * u * u - 2.0 * u - 2.0) / 2.0, d2 = (3.0 * u * u - 1.0) / 6.0;
        const double p0 = lm * tab[k - 1] + l0 * tab[k] + l1 * tab[k + 1] + l2 * tab[k + 2];
        const double dpdu = dm * tab[k - 1] + d0 * tab[k] + d1 * tab[k + 1] + d2 * tab[k + 2];
        const double dpdq = dpdu / (dlnq * q);  // du/dq = 1 / (q dlnq)
        slot[m] = static_cast<int>(m);
        A[m] = nn * (p0 - phi00);
        U[m] = 0.5 * nn * nn * dpdq;
    }
}

__global__ void k_diag_final(const double *__restrict__ part, int nb, double *__restrict__ sums) {
    if (threadIdx.x < 2) {
        double v = 0.0;
        for (int b = 0; b < nb; ++b) v += part[2 * b + threadIdx.x];
        sums[threadIdx.x] = v;
    }
}

}  // namespace

int launch_diag_range(long long N, const double *n, const double *q0, double n_cut, unsigned long long *mm,
                      cudaStream_t st) {
    k_diag_range<<<kDiagBlocks, kDiagThreads, 0, st>>>(N, n, q0, n_cut, mm);
    count_launches(1);
    VDWDF_CUDA_TRY(cudaGetLastError());
    return VDWDF_OK;
}

// part: 2 kDiagBlocks doubles of scratch
int launch_diag_sum(long long N, const double *n, const double *q0, double n_cut, const double *tab, int nq,
                    double lnq0, double dlnq, double *part, double *sums, cudaStream_t st) {
    k_diag_sum<<<kDiagBlocks, kDiagThreads, 0, st>>>(N, n, q0, n_cut, tab, nq, lnq0, dlnq, part);
    k_diag_final<<<1, 32, 0, st>>>(part, kDiagBlocks, sums);
    count_launches(2);
    VDWDF_CUDA_TRY(cudaGetLastError());
    return VDWDF_OK;
}

int launch_diag_AU(long long N, const double *n, const double *q0, double n_cut, const double *tab, int nq,
                   double lnq0, double dlnq, double phi00, int *slot, double *A, double *U, cudaStream_t st) {
    long long nb = (N + 255) / 256;
    if (nb > 1 << 20) nb = 1 << 20;
    k_diag_AU<<<static_cast<int>(nb), 256, 0, st>>>(N, n, q0, n_cut, tab, nq, lnq0, dlnq, phi00, slot, A, U);
    count_launches(1);
    VDWDF_CUDA_TRY(cudaGetLastError());
    return VDWDF_OK;
}

int launch_assemble(const int dims[3], const AxisMap &am, double dV, const int *slot,
                    const double *A, const double *U, const double *dq0dn, const double *dq0dg,
                    const double *div_pre, double *v, double *A_grid, double *U_grid, cudaStream_t st) {
    const long long N = static_cast<long long>(dims[0]) * dims[1] * dims[2];
    const int bs = 256;
    long long nb = (N + bs - 1) / bs;
    if (nb > 1 << 20) nb = 1 << 20;
    k_assemble<<<static_cast<int>(nb), bs, 0, st>>>(dims[0], dims[1], dims[2], am, dV, slot, A, U, dq0dn,
                                                     dq0dg, div_pre, v, A_grid, U_grid);
    count_launches(1);
    VDWDF_CUDA_TRY(cudaGetLastError());
    return VDWDF_OK;
}

int launch_energy_from_A(int n_max, const double *A, const double *n64, Stats *stats,
                         cudaStream_t st) {
    int nb = (n_max + 255) / 256;
    if (nb > 2048) nb = 2048;
    if (nb < 1) nb = 1;
    k_energy_from_A<<<nb, 256, 0, st>>>(n_max, A, n64, stats);
    count_launches(1);
    VDWDF_CUDA_TRY(cudaGetLastError());
    return VDWDF_OK;
}

}  // namespace vdwdf
