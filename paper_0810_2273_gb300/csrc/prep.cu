// Grid-level steps before the pair sum, FP64:
//  - gradient by 4th-order central differences along the grid axes with
//    periodic wrap (section 3 uses finite differences along perpendicular axes;
//    on a general cell the differences along each axis give d/du_a, u_a the
//    fractional coordinate, and grad = sum_a (d/du_a) B_a with the reciprocal
//    rows B_a),
//      along axis a: (n_{-2} - 8 n_{-1} + 8 n_{+1} - n_{+2}) / 12 per index step;
//  - q0 of Dion eqs. 11-12 (section 2 relies on it through D and delta):
//      q0 = k_F - (Zab/36) |g|^2 / (k_F n^2) - (4 pi/3) eps_c(r_s),
//    k_F = (3 pi^2 n)^(1/3), Zab = -0.8491, eps_c of Perdew-Wang 1992, and the
//    partials dq0/dn, dq0/dg used by the adjoint;
//  - trimming (section 3: points below a density cutoff are dropped): active
//    points are listed in the order of 4x4x4 grid bricks taken along a Morton
//    curve, so that consecutive runs of kTile points are compact in space;
//  - bounding boxes of those kTile-point tiles (for image culling).
#include <cuda_runtime.h>

#include "common.cuh"

namespace vdwdf {

namespace {

constexpr double kPi = 3.14159265358979323846;

// Perdew-Wang 1992 unpolarised correlation per electron (Hartree) and d/d rs.
__device__ __forceinline__ void pw92_eps(double rs, double &e, double &dedrs) {
    const double A = 0.031091, a1 = 0.21370;
    const double b1 = 7.5957, b2 = 3.5876, b3 = 1.6382, b4 = 0.49294;
    const double srs = sqrt(rs);
    const double den = 2.0 * A * (srs * (b1 + b3 * rs) + rs * (b2 + b4 * rs));
    const double dden = A * (b1 / srs + 2.0 * b2 + 3.0 * b3 * srs + 4.0 * b4 * rs);
    const double lg = log1p(1.0 / den);
    const double pre = -2.0 * A * (1.0 + a1 * rs);
    e = pre * lg;
    // d/drs of log(1 + 1/den) = -den' / (den (den + 1))
    dedrs = -2.0 * A * a1 * lg - pre * dden / (den * (den + 1.0));
}

__device__ __forceinline__ int wrap(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}

// grad n at point m = (a, b, c): the caller's [3][N] gradient, or the 4th-order
// periodic stencil on n along each grid axis, mapped to Cartesian components
// (general cells: g_c = sum_a S[3a + c] stencil_a).
__device__ __forceinline__ void grad_at(long long m, int n0, int n1, int n2, const AxisMap &am,
                                        const double *__restrict__ n,
                                        const double *__restrict__ gin, double &gx, double &gy,
                                        double &gz) {
    const long long N = static_cast<long long>(n0) * n1 * n2;
    if (gin) {
        gx = gin[m];
        gy = gin[N + m];
        gz = gin[2 * N + m];
        return;
    }
    const int c = static_cast<int>(m % n2);
    const int b = static_cast<int>((m / n2) % n1);
    const int a = static_cast<int>(m / (static_cast<long long>(n1) * n2));
    const long long sa = static_cast<long long>(n1) * n2;
    const long long row = m - static_cast<long long>(a) * sa;  // b * n2 + c
    const long long pl = m - c;                                // (a, b, 0)
    auto at_a = [&](int aa) { return n[static_cast<long long>(wrap(aa, n0)) * sa + row]; };
    auto at_b = [&](int bb) { return n[static_cast<long long>(a) * sa + static_cast<long long>(wrap(bb, n1)) * n2 + c]; };
    auto at_c = [&](int cc) { return n[pl + wrap(cc, n2)]; };
    const double s0 = 8.0 * (at_a(a + 1) - at_a(a - 1)) - (at_a(a + 2) - at_a(a - 2));
    const double s1 = 8.0 * (at_b(b + 1) - at_b(b - 1)) - (at_b(b + 2) - at_b(b - 2));
    const double s2 = 8.0 * (at_c(c + 1) - at_c(c - 1)) - (at_c(c + 2) - at_c(c - 2));
    if (!am.general) {
        gx = s0 * am.S[0];
        gy = s1 * am.S[4];
        gz = s2 * am.S[8];
    } else {
        gx = s0 * am.S[0] + s1 * am.S[3] + s2 * am.S[6];
        gy = s0 * am.S[1] + s1 * am.S[4] + s2 * am.S[7];
        gz = s0 * am.S[2] + s1 * am.S[5] + s2 * am.S[8];
    }
}

__global__ void k_grad_q0(int n0, int n1, int n2, const AxisMap am,
                          const double *__restrict__ n, const double *__restrict__ gin,
                          double *__restrict__ q0, double *__restrict__ qn, double *__restrict__ qg) {
    const long long N = static_cast<long long>(n0) * n1 * n2;
    const double Zab = -0.8491;
    for (long long m = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; m < N;
         m += static_cast<long long>(gridDim.x) * blockDim.x) {
        double gx, gy, gz;
        grad_at(m, n0, n1, n2, am, n, gin, gx, gy, gz);
        const double nn = n[m];
        if (!(nn > 0.0)) {
            q0[m] = 0.0;
            if (qn) qn[m] = 0.0;
            if (qg) {
                qg[m] = 0.0;
                qg[N + m] = 0.0;
                qg[2 * N + m] = 0.0;
            }
            continue;
        }
        const double kF = cbrt(3.0 * kPi * kPi * nn);
        const double g2 = gx * gx + gy * gy + gz * gz;
        const double rs = cbrt(3.0 / (4.0 * kPi * nn));
        double ec, decdrs;
        pw92_eps(rs, ec, decdrs);
        const double inv_kFn2 = 1.0 / (kF * nn * nn);
        q0[m] = kF - (Zab / 36.0) * g2 * inv_kFn2 - (4.0 * kPi / 3.0) * ec;
        if (qn) {
            const double dec_dn = decdrs * (-rs / (3.0 * nn));
            qn[m] = kF / (3.0 * nn) + (7.0 * Zab / 108.0) * g2 * inv_kFn2 / nn - (4.0 * kPi / 3.0) * dec_dn;
        }
        if (qg) {
            const double f = -(Zab / 18.0) * inv_kFn2;
            qg[m] = f * gx;
            qg[N + m] = f * gy;
            qg[2 * N + m] = f * gz;
        }
    }
}

struct BrickGeom {
    int n0, n1, n2, nbz, nby;
};

__device__ __forceinline__ void brick_point(const BrickGeom &g, int brick, int e, int &a, int &b,
                                            int &c, bool &valid) {
    const int bz = brick % g.nbz;
    const int by = (brick / g.nbz) % g.nby;
    const int bx = brick / (g.nbz * g.nby);
    a = bx * kBrick + (e >> 4);
    b = by * kBrick + ((e >> 2) & 3);
    c = bz * kBrick + (e & 3);
    valid = a < g.n0 && b < g.n1 && c < g.n2;
}

// one warp per brick position p: count active points
__global__ void k_brick_count(BrickGeom g, const int *__restrict__ order, int nb,
                              const double *__restrict__ n, double n_cut, int *__restrict__ cnt) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= nb) return;
    const int brick = order[warp];
    int total = 0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        int a, b, c;
        bool valid;
        brick_point(g, brick, lane + 32 * h, a, b, c, valid);
        bool act = false;
        if (valid) act = n[(static_cast<long long>(a) * g.n1 + b) * g.n2 + c] >= n_cut;
        total += __popc(__ballot_sync(0xffffffffu, act));
    }
    if (lane == 0) cnt[warp] = total;
}

// exclusive scan of cnt[0..nb) into off[0..nb], total to stats->n_active (one block)
__global__ void k_scan(const int *__restrict__ cnt, int nb, int *__restrict__ off, Stats *stats) {
    __shared__ int warp_sums[32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int base = 0; base < nb; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const int v = i < nb ? cnt[i] : 0;
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_sums[w] = x;
        __syncthreads();
        if (w == 0) {
            int s = lane < (blockDim.x >> 5) ? warp_sums[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += y;
            }
            warp_sums[lane] = s;  // inclusive over warps
        }
        __syncthreads();
        const int before = (w > 0 ? warp_sums[w - 1] : 0) + carry;
        if (i < nb) off[i] = before + x - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = before + x;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        off[nb] = carry;
        stats->n_active = carry;
    }
}

// one warp per brick: write the active points in brick order, and the slot map
__global__ void k_scatter(BrickGeom g, const int *__restrict__ order, int nb,
                          const double *__restrict__ n, double n_cut, const double *__restrict__ q0,
                          const int *__restrict__ off, int *__restrict__ slot, float4 *__restrict__ p32,
                          float *__restrict__ n32, dvec4 *__restrict__ p64, double *__restrict__ n64) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= nb) return;
    const int brick = order[warp];
    int base = off[warp];
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        int a, b, c;
        bool valid;
        brick_point(g, brick, lane + 32 * h, a, b, c, valid);
        const long long m = (static_cast<long long>(a) * g.n1 + b) * g.n2 + c;
        const double nn = valid ? n[m] : 0.0;
        const bool act = valid && nn >= n_cut;
        const unsigned mask = __ballot_sync(0xffffffffu, act);
        if (act) {
            const int s = base + __popc(mask & lt);
            const double q = q0[m];
            p32[s] = make_float4(static_cast<float>(a), static_cast<float>(b), static_cast<float>(c),
                                 static_cast<float>(q));
            n32[s] = static_cast<float>(nn);
            if (p64) {
                dvec4 v;
                v.x = a;
                v.y = b;
                v.z = c;
                v.w = q;
                p64[s] = v;
            }
            n64[s] = nn;
            if (slot) slot[m] = s;
        } else if (valid && slot) {
            slot[m] = -1;
        }
        base += __popc(mask);
    }
}

// one warp per kTile-point tile: bounding box, q0 range, sum of n^2
__global__ void k_tiles(const float4 *__restrict__ p32, const double *__restrict__ n64,
                        float4 *__restrict__ blo, float4 *__restrict__ bhi, Stats *stats, int ntiles_max) {
    const int na = stats->n_active;
    const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t >= ntiles_max || t * kTile >= na) return;
    const int i = t * kTile + lane;
    const bool in = i < na;
    const float4 p = in ? p32[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    float lo[4] = {in ? p.x : 3e38f, in ? p.y : 3e38f, in ? p.z : 3e38f, in ? p.w : 3e38f};
    float hi[4] = {in ? p.x : -3e38f, in ? p.y : -3e38f, in ? p.z : -3e38f, in ? p.w : -3e38f};
    double n2 = in ? n64[i] * n64[i] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
            hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
        }
        n2 += __shfl_xor_sync(0xffffffffu, n2, o);
    }
    if (lane == 0) {
        blo[t] = make_float4(lo[0], lo[1], lo[2], lo[3]);
        bhi[t] = make_float4(hi[0], hi[1], hi[2], hi[3]);
        atomicAdd(&stats->n2sum, n2);
        // q0 > 0 on active points: float bit patterns order like the values
        atomicMin(&stats->qmin_bits, __float_as_uint(lo[3]));
        atomicMax(&stats->qmax_bits, __float_as_uint(hi[3]));
    }
}

// Cartesian bounding boxes of the kTile-point tiles on a general cell: point
// (i, j, k) sits at i v_0 + j v_1 + k v_2 with v_a = M_a / N_a (rows of vrow).
__global__ void k_tiles_cart(const float4 *__restrict__ p32, const Stats *stats, const CellRows vrow,
                             float4 *__restrict__ clo, float4 *__restrict__ chi, int ntiles_max) {
    const int na = stats->n_active;
    const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t >= ntiles_max || t * kTile >= na) return;
    const int i = t * kTile + lane;
    const bool in = i < na;
    const float4 p = in ? p32[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    float lo[3], hi[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float x = p.x * vrow.v[c] + p.y * vrow.v[3 + c] + p.z * vrow.v[6 + c];
        lo[c] = in ? x : 3e38f;
        hi[c] = in ? x : -3e38f;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            lo[c] = fminf(lo[c], __shfl_xor_sync(0xffffffffu, lo[c], o));
            hi[c] = fmaxf(hi[c], __shfl_xor_sync(0xffffffffu, hi[c], o));
        }
    if (lane == 0) {
        clo[t] = make_float4(lo[0], lo[1], lo[2], 0.f);
        chi[t] = make_float4(hi[0], hi[1], hi[2], 0.f);
    }
}

// ---------------------------------------------------------------------------
// Semilocal energies of eq. (3) (section 2: E_x^LDA, E_c^LDA, E_x^PBE, E_c^PBE
// and E_x^revPBE from the density itself), spin-unpolarised, FP64:
//   eps_x^LDA = -3 k_F/(4 pi);  GGA exchange eps_x^LDA F_x(s),
//   F_x = 1 + kappa - kappa/(1 + mu s^2/kappa), s = |g|/(2 k_F n),
//   kappa = 0.804 (PBE) or 1.245 (revPBE), mu = beta pi^2/3;
//   eps_c^PBE = eps_c^PW92 + gamma ln[1 + (beta/gamma) t^2 (1 + A t^2)/(1 + A t^2 + A^2 t^4)],
//   t = |g|/(2 k_s n), k_s = (4 k_F/pi)^(1/2), A = (beta/gamma)/(exp(-eps_c/gamma) - 1),
//   beta = 0.06672455060314922, gamma = (1 - ln 2)/pi^2.
// Each block sums n eps over its points (fixed grid-stride order, fixed tree);
// a second kernel adds the block sums in order, so the result is reproducible.
// ---------------------------------------------------------------------------
constexpr int kSemiBlocks = 608;  // 4 per SM on 152 SMs
constexpr int kSemiThreads = 256;
constexpr int kSemiVals = 6;      // five energies and the point count

__device__ __forceinline__ double gga_fx(double s2, double kappa, double mu) {
    return 1.0 + kappa - kappa / (1.0 + mu * s2 / kappa);
}

__global__ void __launch_bounds__(kSemiThreads) k_semilocal(int n0, int n1, int n2, const AxisMap am,
                                                            const double *__restrict__ n,
                                                            const double *__restrict__ gin,
                                                            double *__restrict__ part) {
    const long long N = static_cast<long long>(n0) * n1 * n2;
    const double beta = 0.06672455060314922;
    const double gamma = (1.0 - log(2.0)) / (kPi * kPi);
    const double mu = beta * kPi * kPi / 3.0;
    double acc[kSemiVals] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (long long m = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; m < N;
         m += static_cast<long long>(gridDim.x) * blockDim.x) {
        const double nn = n[m];
        if (!(nn > 0.0)) continue;
        double gx, gy, gz;
        grad_at(m, n0, n1, n2, am, n, gin, gx, gy, gz);
        const double g2 = gx * gx + gy * gy + gz * gz;
        const double kF = cbrt(3.0 * kPi * kPi * nn);
        const double rs = cbrt(3.0 / (4.0 * kPi * nn));
        double ec, decdrs;
        pw92_eps(rs, ec, decdrs);
        const double ex = -3.0 * kF / (4.0 * kPi);
        const double s2 = g2 / (4.0 * kF * kF * nn * nn);
        const double ks2 = 4.0 * kF / kPi;
        const double t2 = g2 / (4.0 * ks2 * nn * nn);
        const double A = (beta / gamma) / expm1(-ec / gamma);
        const double At2 = A * t2;
        const double H = gamma * log1p((beta / gamma) * t2 * (1.0 + At2) / (1.0 + At2 + At2 * At2));
        acc[0] += nn * ex;
        acc[1] += nn * ec;
        acc[2] += nn * ex * gga_fx(s2, 0.804, mu);
        acc[3] += nn * (ec + H);
        acc[4] += nn * ex * gga_fx(s2, 1.245, mu);
        acc[5] += 1.0;
    }
    __shared__ double red[kSemiVals][kSemiThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kSemiVals; ++k) {
        double v = acc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[k][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < kSemiVals) {
        double v = 0.0;
        for (int w = 0; w < kSemiThreads / 32; ++w) v += red[threadIdx.x][w];
        part[static_cast<long long>(blockIdx.x) * kSemiVals + threadIdx.x] = v;
    }
}

__global__ void k_semilocal_sum(const double *__restrict__ part, int nblocks, double *__restrict__ out) {
    if (threadIdx.x < kSemiVals) {
        double v = 0.0;
        for (int b = 0; b < nblocks; ++b) v += part[static_cast<long long>(b) * kSemiVals + threadIdx.x];
        out[threadIdx.x] = v;
    }
}

// The finite-difference gradient alone (Cartesian, 3 planes of N).
__global__ void k_gradient_fd(int n0, int n1, int n2, const AxisMap am, const double *__restrict__ n,
                              double *__restrict__ g) {
    const long long N = static_cast<long long>(n0) * n1 * n2;
    for (long long m = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; m < N;
         m += static_cast<long long>(gridDim.x) * blockDim.x) {
        double gx, gy, gz;
        grad_at(m, n0, n1, n2, am, n, nullptr, gx, gy, gz);
        g[m] = gx;
        g[N + m] = gy;
        g[2 * N + m] = gz;
    }
}

}  // namespace

int semilocal_scratch_doubles() { return (kSemiBlocks + 1) * kSemiVals; }

int launch_semilocal(const int dims[3], const AxisMap &am, const double *n, const double *grad_in,
                     double *scratch, cudaStream_t st) {
    k_semilocal<<<kSemiBlocks, kSemiThreads, 0, st>>>(dims[0], dims[1], dims[2], am, n, grad_in, scratch);
    k_semilocal_sum<<<1, 32, 0, st>>>(scratch, kSemiBlocks, scratch + kSemiBlocks * kSemiVals);
    count_launches(2);
    VDWDF_CUDA_TRY(cudaGetLastError());
    return VDWDF_OK;
}

int launch_tiles_cart(const float4 *p32, const Stats *stats, const CellRows &vrow, float4 *clo, float4 *chi,
                      long long n_max, cudaStream_t st) {
    const int tiles = static_cast<int>((n_max + kTile - 1) / kTile);
    k_tiles_cart<<<(tiles + 7) / 8, 256, 0, st>>>(p32, stats, vrow, clo, chi, tiles);
    count_launches(1);
    VDWDF_CUDA_TRY(cudaGetLastError());
    return VDWDF_OK;
}

int launch_gradient_fd(const int dims[3], const AxisMap &am, const double *n, double *grad, cudaStream_t st) {
    const long long N = static_cast<long long>(dims[0]) * dims[1] * dims[2];
    const int bs = 256;
    long long nb = (N + bs - 1) / bs;
    if (nb > 1 << 20) nb = 1 << 20;
    k_gradient_fd<<<static_cast<int>(nb), bs, 0, st>>>(dims[0], dims[1], dims[2], am, n, grad);
    count_launches(1);
    VDWDF_CUDA_TRY(cudaGetLastError());
    return VDWDF_OK;
}

int launch_grad_q0(const int dims[3], const AxisMap &am, const double *n, const double *grad_in,
                   double *q0, double *dq0dn, double *dq0dg, cudaStream_t st) {
    const long long N = static_cast<long long>(dims[0]) * dims[1] * dims[2];
    const int bs = 256;
    long long nb = (N + bs - 1) / bs;
    if (nb > 1 << 20) nb = 1 << 20;
    k_grad_q0<<<static_cast<int>(nb), bs, 0, st>>>(dims[0], dims[1], dims[2], am, n, grad_in, q0, dq0dn, dq0dg);
    count_launches(1);
    VDWDF_CUDA_TRY(cudaGetLastError());
    return VDWDF_OK;
}

int launch_compact(const int dims[3], const double *n, double n_cut, const double *q0,
                   const int *brick_order, int nbricks, int *brick_cnt, int *brick_off, int *slot,
                   float4 *p32, float *n32, dvec4 *p64, double *n64, float4 *blo, float4 *bhi,
                   Stats *stats, cudaStream_t st) {
    BrickGeom g;
    g.n0 = dims[0];
    g.n1 = dims[1];
    g.n2 = dims[2];
    g.nbz = (dims[2] + kBrick - 1) / kBrick;
    g.nby = (dims[1] + kBrick - 1) / kBrick;
    const int wpb = 8;
    const int blocks = (nbricks + wpb - 1) / wpb;
    k_brick_count<<<blocks, 32 * wpb, 0, st>>>(g, brick_order, nbricks, n, n_cut, brick_cnt);
    VDWDF_CUDA_TRY(cudaGetLastError());
    k_scan<<<1, 1024, 0, st>>>(brick_cnt, nbricks, brick_off, stats);
    VDWDF_CUDA_TRY(cudaGetLastError());
    k_scatter<<<blocks, 32 * wpb, 0, st>>>(g, brick_order, nbricks, n, n_cut, q0, brick_off, slot, p32,
                                           n32, p64, n64);
    VDWDF_CUDA_TRY(cudaGetLastError());
    const long long N = static_cast<long long>(dims[0]) * dims[1] * dims[2];
    const int tiles = static_cast<int>((N + kTile - 1) / kTile);
    k_tiles<<<(tiles + 7) / 8, 256, 0, st>>>(p32, n64, blo, bhi, stats, tiles);
    VDWDF_CUDA_TRY(cudaGetLastError());
    count_launches(4);
    return VDWDF_OK;
}

}  // namespace vdwdf
