// Pair kernels of the vdW-DF double sum (paper section 2, eq. (2)) and of its
// adjoint, with periodic images under a spherical cutoff (section 3).
//
// For active points i, j and image vectors L (periodic axes),
//   r = |r_i - r_j + L|,  D = r (q_i + q_j)/2,  delta = |q_i - q_j|/(q_i + q_j),
//   phi = bicubic B-spline of the node table at (D, delta)         if D <= Dmax,
//   phi = -C / (d1^2 d2^2 (d1^2 + d2^2)), d1 = q_i r, d2 = q_j r     otherwise
// (section 2: the kernel "can be redefined to depend on two quantities D and
// delta"; Dion eq. 17 for large D).  Energy mode sums each unordered pair once
// with weight 2 (phi is symmetric in i, j); potential mode gives, per point,
//   A_i = sum_{j,L} n_j phi,   U_i = n_i sum_{j,L} n_j r dphi/dd1,
//   r dphi/dd1 = r/2 phi_D + (1 - ds)/(q_i + q_j) phi_ds,  ds = (q_i - q_j)/(q_i + q_j)
// on the table branch and -2 phi (1/q_i + q_i/(q_i^2 + q_j^2)) on the asymptote.
//
// Work decomposition: persistent CTAs pull work items (instance, i tile,
// range of j tiles) from one queue in global memory; each thread owns one i;
// j tiles of kJT points are staged in shared memory and read as broadcasts;
// the FP32 path keeps a band of B-spline rows resident in shared memory and
// reads it with explicit shared-memory loads, other rows from L2.  Periodic
// images of a j tile are culled against the i tile by bounding boxes.  FP32
// partial sums over one (j tile, image) are folded into FP64 accumulators.
// The work loop is bounded (max_iters); nothing waits on another CTA.
#include <cuda_runtime.h>

#include "common.cuh"

namespace vdwdf {

namespace {

template <typename R>
struct PT;
template <>
struct PT<float> {
    using P = float4;
    static __device__ __forceinline__ const P *pts(const PairParams &pp) { return pp.p32; }
    static __device__ __forceinline__ const float *ns(const PairParams &pp) { return pp.n32; }
    static __device__ __forceinline__ P load(const P *p, int i) { return __ldg(p + i); }
};
template <>
struct PT<double> {
    using P = dvec4;
    static __device__ __forceinline__ const P *pts(const PairParams &pp) { return pp.p64; }
    static __device__ __forceinline__ const double *ns(const PairParams &pp) { return pp.n64; }
    static __device__ __forceinline__ P load(const P *p, int i) {
        const double2 *q = reinterpret_cast<const double2 *>(p + i);
        const double2 a = __ldg(q), b = __ldg(q + 1);
        P r;
        r.x = a.x;
        r.y = a.y;
        r.z = b.x;
        r.w = b.y;
        return r;
    }
};

// floor of a non-negative float below 2^22 without a conversion instruction:
// adding 1.5 * 2^23 rounded toward minus infinity leaves floor(x) in the low
// mantissa bits.
__device__ __forceinline__ int floor_split(float x, float &frac) {
    const float b = __fadd_rd(x, 12582912.0f);
    frac = x - (b - 12582912.0f);
    return __float_as_int(b) - 0x4B400000;
}
__device__ __forceinline__ int floor_split(double x, double &frac) {
    const double f = floor(x);
    frac = x - f;
    return static_cast<int>(f);
}

// Cubic B-spline weights times 6 (the table holds coefficients / 36) and their
// t-derivatives times 6.
template <typename R>
__device__ __forceinline__ void bw(R t, R w[4]) {
    const R t2 = t * t, t3 = t2 * t, s = R(1) - t;
    w[0] = s * s * s;
    w[1] = R(3) * t3 - R(6) * t2 + R(4);
    w[2] = R(-3) * t3 + R(3) * t2 + R(3) * t + R(1);
    w[3] = t3;
}
template <typename R>
__device__ __forceinline__ void bdw(R t, R d[4]) {
    const R t2 = t * t, s = R(1) - t;
    d[0] = R(-3) * s * s;
    d[1] = R(9) * t2 - R(12) * t;
    d[2] = R(-9) * t2 + R(6) * t + R(3);
    d[3] = R(3) * t2;
}

__device__ __forceinline__ float recip(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }
__device__ __forceinline__ float rlen(float r2) { return r2 * rsqrtf(fmaxf(r2, 1e-30f)); }
__device__ __forceinline__ double rlen(double r2) { return sqrt(r2); }

__device__ __forceinline__ float lds32(uint32_t a) {
    float v;
    asm("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
    return v;
}

template <bool POT, typename R>
__device__ __forceinline__ void combine(const R c[4][4], const R wD[4], const R dwD[4],
                                        const R wd[4], const R dwd[4], R &phi, R &pt, R &pu) {
    R p = 0, a = 0, b = 0;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const R row = wd[0] * c[m][0] + wd[1] * c[m][1] + wd[2] * c[m][2] + wd[3] * c[m][3];
        p += wD[m] * row;
        if (POT) {
            const R drow = dwd[0] * c[m][0] + dwd[1] * c[m][1] + dwd[2] * c[m][2] + dwd[3] * c[m][3];
            a += dwD[m] * row;
            b += wD[m] * drow;
        }
    }
    phi = p;
    pt = a;
    pu = b;
}

template <typename R>
struct Consts {
    R cD, cd, tDmax, tDclamp, tdmax, tdclamp, C;
    int kmax, lmax;  // last cell index along D and delta
};

template <typename R>
struct Table {
    const R *g;      // whole coefficient table in global memory, row stride S
    uint32_t s;      // shared-memory address of the resident band (FP32), same stride
    int k0, kn;      // band rows [k0, k0 + kn)
    int S;
};

template <bool POT, typename R>
__device__ __forceinline__ void interp(const Table<R> &tb, int k, int l, const R wD[4],
                                       const R dwD[4], const R wd[4], const R dwd[4], R &p, R &pt,
                                       R &pu) {
    R c[4][4];
    if (sizeof(R) == 4 && k >= tb.k0 && k + 4 <= tb.k0 + tb.kn) {
        const uint32_t a0 = tb.s + 4u * static_cast<uint32_t>((k - tb.k0) * tb.S + l);
        const uint32_t rs = 4u * static_cast<uint32_t>(tb.S);
#pragma unroll
        for (int m = 0; m < 4; ++m)
#pragma unroll
            for (int n = 0; n < 4; ++n) c[m][n] = static_cast<R>(lds32(a0 + m * rs + 4u * n));
    } else {
        const R *g = tb.g + static_cast<size_t>(k) * tb.S + l;
#pragma unroll
        for (int m = 0; m < 4; ++m)
#pragma unroll
            for (int n = 0; n < 4; ++n) c[m][n] = __ldg(g + m * tb.S + n);
    }
    combine<POT, R>(c, wD, dwD, wd, dwd, p, pt, pu);
}

// One pair: phi and (POT) r dphi/dd1; counts a clamped delta.
template <bool POT, typename R>
__device__ __forceinline__ void pair_phi(R r2, R qi, R qj, R inv_qi, R qi2, const Consts<R> &K,
                                         const Table<R> &tb, R &phi, R &rd, unsigned &ncl) {
    const R r = rlen(r2);
    const R sq = qi + qj;
    const R dq = qi - qj;
    const R isq = recip(sq);
    R tD = r * sq * K.cD;
    // the table is read only for 0 <= tD <= nD - 1 (also false for NaN); delta is
    // clamped into [0, last node] so that no index leaves the table
    if (tD >= R(0) && tD <= K.tDmax) {
        tD = fmin(tD, K.tDclamp);
        const R dl = fabs(dq) * isq;
        R td = dl * K.cd;
        const bool cl = td > K.tdmax;
        ncl += cl ? 1u : 0u;
        td = fmin(fmax(td, R(0)), K.tdclamp);
        R t, u;
        int k = floor_split(tD, t);
        int l = floor_split(td, u);
        if (sizeof(R) == 8) {  // FP64 keeps the exact end nodes: last cell at t = 1
            if (k > K.kmax) {
                k = K.kmax;
                t = tD - R(k);
            }
            if (l > K.lmax) {
                l = K.lmax;
                u = td - R(l);
            }
        }
        R wD[4], wd[4], dwD[4], dwd[4];
        bw<R>(t, wD);
        bw<R>(u, wd);
        if (POT) {
            bdw<R>(t, dwD);
            bdw<R>(u, dwd);
        }
        R pt = 0, pu = 0;
        interp<POT, R>(tb, k, l, wD, dwD, wd, dwd, phi, pt, pu);
        if (POT) {
            const R sgn1 = dq > R(0) ? (R(1) - dl) : -(R(1) + dl);
            pu = cl ? R(0) : pu;
            rd = r * K.cD * pt + isq * K.cd * sgn1 * pu;
        }
    } else {
        const R r4 = r2 * r2;
        const R qj2 = qj * qj;
        const R s2 = qi2 + qj2;
        phi = -K.C * recip(r4 * r2 * qi2 * qj2 * s2);
        if (POT) rd = R(-2) * phi * (inv_qi + qi * recip(s2));
    }
}

template <typename R>
__device__ void make_consts(const PairShared &sh, Consts<R> &K) {
    K.cD = static_cast<R>(sh.cD);
    K.cd = static_cast<R>(sh.cd);
    K.C = static_cast<R>(sh.C_asym);
    K.tDmax = static_cast<R>(sh.nD - 1);
    K.tdmax = static_cast<R>(sh.nd - 1);
    if (sizeof(R) == 4) {
        // largest float below nD - 1 (nd - 1): the last cell is reached with t < 1
        K.tDclamp = static_cast<R>(__int_as_float(__float_as_int(static_cast<float>(sh.nD - 1)) - 1));
        K.tdclamp = static_cast<R>(__int_as_float(__float_as_int(static_cast<float>(sh.nd - 1)) - 1));
    } else {
        K.tDclamp = K.tDmax;
        K.tdclamp = K.tdmax;
    }
    K.kmax = sh.nD - 2;
    K.lmax = sh.nd - 2;
}

__device__ __forceinline__ void fold(float &a32, double &a64) {
    a64 += static_cast<double>(a32);
    a32 = 0.0f;
}
__device__ __forceinline__ void fold(double &a, double &a64) {
    a64 += a;
    a = 0.0;
}

// Sum over the block; result valid in thread 0.  All threads must call it.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    T s = T(0);
    if (threadIdx.x < 32) {
        s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : T(0);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    return s;
}

// Squared distance between the i box and the j box shifted by image m.
__device__ __forceinline__ float box_gap2(const float ilo[3], const float ihi[3], const float jl[3],
                                          const float jh[3], const int m[3], const int dims[3],
                                          const float h2[3]) {
    float d2 = 0.0f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float s = static_cast<float>(m[a] * dims[a]);
        const float g = fmaxf(0.0f, fmaxf(ilo[a] - jh[a] + s, jl[a] - ihi[a] - s));
        d2 += h2[a] * g * g;
    }
    return d2;
}

// Spherical cutoff, inclusive: a pair is inside iff r^2 <= rc2 (the host folds a
// 1e-12 relative allowance into rc2 so that distances equal to the cutoff up to
// rounding count as inside in every path).  FP32 decides pairs clearly away from
// the boundary and re-checks the rest in FP64 from the exact index offsets.
struct Cut {
    double rc2d;
    double h2d[3];
    float lo, hi;
};
__device__ __forceinline__ bool beyond(float r2, float dx, float dy, float dz, const Cut &c) {
    if (r2 > c.hi) return true;
    if (r2 <= c.lo) return false;
    const double X = dx, Y = dy, Z = dz;
    return c.h2d[0] * (X * X) + c.h2d[1] * (Y * Y) + c.h2d[2] * (Z * Z) > c.rc2d;
}
__device__ __forceinline__ bool beyond(double r2, double, double, double, const Cut &c) {
    return r2 > c.rc2d;
}

// MODE 0: energy (unordered pairs), MODE 1: potential (A, U per point).
template <typename R, int MODE, int NT>
__global__ void __launch_bounds__(NT, 1) k_pair(const __grid_constant__ PairLaunch pl) {
    constexpr bool POT = (MODE == 1);
    using P = typename PT<R>::P;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    P *sp = reinterpret_cast<P *>(smem_raw);
    R *sn = reinterpret_cast<R *>(smem_raw + sizeof(P) * kJT);
    double *red = reinterpret_cast<double *>(smem_raw + (sizeof(P) + sizeof(R)) * kJT);
    unsigned long long *redu = reinterpret_cast<unsigned long long *>(red + 32);
    __shared__ unsigned int s_item;
    __shared__ unsigned int s_prefix[kMaxInst + 1];
    __shared__ int s_C[kMaxInst];

    const PairShared &sh = pl.sh;
    Table<R> tb;
    tb.S = sh.S;
    Consts<R> K;
    make_consts<R>(sh, K);
    if constexpr (sizeof(R) == 4) {
        tb.g = reinterpret_cast<const R *>(sh.tab32);
        float *band = reinterpret_cast<float *>(smem_raw + (sizeof(P) + sizeof(R)) * kJT + 64 * sizeof(double));
        tb.s = static_cast<uint32_t>(__cvta_generic_to_shared(band));
        tb.k0 = sh.ks0;
        tb.kn = sh.ksn;
        const int nb = sh.ksn * sh.S;
        const float *src = sh.tab32 + static_cast<size_t>(sh.ks0) * sh.S;
        for (int e = threadIdx.x; e < nb; e += NT) band[e] = __ldg(src + e);
    } else {
        tb.g = reinterpret_cast<const R *>(sh.tab64);
        tb.s = 0;
        tb.k0 = 0;
        tb.kn = 0;
    }
    // work items per instance: (i tiles) x (chunks of jtiles_per_item j tiles)
    if (threadIdx.x == 0) {
        unsigned int acc = 0;
        for (int k = 0; k < pl.ninst; ++k) {
            const int na = pl.inst[k].stats->n_active;
            const int nI = (na + NT - 1) / NT;
            const int nJ = (na + kJT - 1) / kJT;
            const int C = max(1, (nJ + sh.jtiles_per_item - 1) / sh.jtiles_per_item);
            s_prefix[k] = acc;
            s_C[k] = C;
            acc += static_cast<unsigned int>(nI) * static_cast<unsigned int>(C);
        }
        s_prefix[pl.ninst] = acc;
    }
    __syncthreads();
    const unsigned int n_items = min(s_prefix[pl.ninst], sh.item_limit);

    for (unsigned int iter = 0;; ++iter) {
        if (iter >= sh.max_iters) {
            if (threadIdx.x == 0) atomicAdd(&pl.inst[0].stats->guard_trips, 1u);
            break;
        }
        if (threadIdx.x == 0) s_item = atomicAdd(sh.queue, 1u);
        __syncthreads();
        const unsigned int item = s_item;
        __syncthreads();
        if (item >= n_items) break;
        int k = 0;
        while (k + 1 < pl.ninst && item >= s_prefix[k + 1]) ++k;
        const PairParams &pp = pl.inst[k];
        const unsigned int local = item - s_prefix[k];
        const int C = s_C[k];
        const int I = static_cast<int>(local / C), c = static_cast<int>(local % C);
        const int n_act = pp.stats->n_active;
        const int nJ = (n_act + kJT - 1) / kJT;

        R h2[3];
        float h2f[3], rcm[3];
        int dims[3], M[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            h2[a] = static_cast<R>(pp.h2[a]);
            h2f[a] = static_cast<float>(pp.h2[a]);
            dims[a] = pp.dims[a];
            M[a] = pp.M[a];
            // cutoff in index units along a, widened so that rounding never drops an image
            rcm[a] = pp.use_cut ? static_cast<float>(sqrt(pp.rc2 / pp.h2[a])) * 1.0001f + 1e-3f : 0.0f;
        }
        Cut cut;
        cut.rc2d = pp.rc2;
        cut.h2d[0] = pp.h2[0];
        cut.h2d[1] = pp.h2[1];
        cut.h2d[2] = pp.h2[2];
        cut.lo = static_cast<float>(pp.rc2) * (1.0f - 1e-5f);
        cut.hi = static_cast<float>(pp.rc2) * (1.0f + 1e-5f);
        const float rc2_box = static_cast<float>(pp.rc2) * 1.0002f + 1e-6f;
        const bool use_cut = pp.use_cut != 0;
        const P *pts = PT<R>::pts(pp);
        const R *nsrc = PT<R>::ns(pp);

        const int ig = I * NT + static_cast<int>(threadIdx.x);
        const bool act = ig < n_act;
        const int ni_act = min(NT, n_act - I * NT);
        R xi = 0, yi = 0, zi = 0, qi = 1, ni = 0;
        if (act) {
            const P pi = PT<R>::load(pts, ig);
            xi = pi.x;
            yi = pi.y;
            zi = pi.z;
            qi = pi.w;
            ni = __ldg(nsrc + ig);
        }
        const R inv_qi = R(1) / qi, qi2 = qi * qi;
        float ilo[3] = {3e38f, 3e38f, 3e38f}, ihi[3] = {-3e38f, -3e38f, -3e38f};
        for (int s = 0; s < NT / kJT; ++s) {
            const int t = I * (NT / kJT) + s;
            if (t * kJT < n_act) {
                const float4 lo = __ldg(pp.blo + t), hi = __ldg(pp.bhi + t);
                ilo[0] = fminf(ilo[0], lo.x);
                ilo[1] = fminf(ilo[1], lo.y);
                ilo[2] = fminf(ilo[2], lo.z);
                ihi[0] = fmaxf(ihi[0], hi.x);
                ihi[1] = fmaxf(ihi[1], hi.y);
                ihi[2] = fmaxf(ihi[2], hi.z);
            }
        }
        const int Js = POT ? 0 : (I * NT) / kJT;
        const int J0 = Js + c * sh.jtiles_per_item;
        const int J1 = min(nJ, J0 + sh.jtiles_per_item);
        double A64 = 0.0, U64 = 0.0;
        unsigned long long cnt = 0, nclamp = 0, evals = 0;
        for (int J = J0; J < J1; ++J) {
            const int jb = J * kJT;
            const int jn = min(kJT, n_act - jb);
            const float4 jlo = __ldg(pp.blo + J), jhi = __ldg(pp.bhi + J);
            const float jl[3] = {jlo.x, jlo.y, jlo.z}, jh[3] = {jhi.x, jhi.y, jhi.z};
            int mlo[3], mhi[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (M[a] == 0) {
                    mlo[a] = 0;
                    mhi[a] = 0;
                } else {
                    const float N = static_cast<float>(dims[a]);
                    mlo[a] = max(-M[a], static_cast<int>(ceilf((-rcm[a] - (ihi[a] - jl[a])) / N)));
                    mhi[a] = min(M[a], static_cast<int>(floorf((rcm[a] - (ilo[a] - jh[a])) / N)));
                }
            }
            bool any = false;
            for (int m0 = mlo[0]; m0 <= mhi[0] && !any; ++m0)
                for (int m1 = mlo[1]; m1 <= mhi[1] && !any; ++m1)
                    for (int m2 = mlo[2]; m2 <= mhi[2] && !any; ++m2) {
                        const int mm[3] = {m0, m1, m2};
                        any = !use_cut || box_gap2(ilo, ihi, jl, jh, mm, dims, h2f) <= rc2_box;
                    }
            if (!any) continue;
            if (static_cast<int>(threadIdx.x) < jn) {
                sp[threadIdx.x] = PT<R>::load(pts, jb + threadIdx.x);
                sn[threadIdx.x] = __ldg(nsrc + jb + threadIdx.x);
            }
            __syncthreads();
            const bool overlap = !POT && (jb < (I + 1) * NT);
            for (int m0 = mlo[0]; m0 <= mhi[0]; ++m0)
                for (int m1 = mlo[1]; m1 <= mhi[1]; ++m1)
                    for (int m2 = mlo[2]; m2 <= mhi[2]; ++m2) {
                        const int mm[3] = {m0, m1, m2};
                        if (use_cut && box_gap2(ilo, ihi, jl, jh, mm, dims, h2f) > rc2_box) continue;
                        const R xs = xi + static_cast<R>(m0 * dims[0]);
                        const R ys = yi + static_cast<R>(m1 * dims[1]);
                        const R zs = zi + static_cast<R>(m2 * dims[2]);
                        R a_acc = 0, u_acc = 0;
                        unsigned int c32 = 0, cl32 = 0;
                        evals += static_cast<unsigned long long>(jn) * static_cast<unsigned long long>(ni_act);
                        if (overlap) {
                            // per-pair weights: 2 (j > i), 1 (j == i), 0 (j < i)
                            for (int jj = 0; jj < jn; ++jj) {
                                const P pj = sp[jj];
                                const R nj = sn[jj];
                                const R dx = xs - pj.x, dy = ys - pj.y, dz = zs - pj.z;
                                const R r2 = h2[0] * (dx * dx) + h2[1] * (dy * dy) + h2[2] * (dz * dz);
                                const int jg = jb + jj;
                                const R wgt = (jg > ig) ? R(2) : ((jg == ig) ? R(1) : R(0));
                                if (wgt == R(0) || (use_cut && beyond(r2, dx, dy, dz, cut))) continue;
                                R phi, rd;
                                unsigned ncl = 0;
                                pair_phi<false, R>(r2, qi, pj.w, inv_qi, qi2, K, tb, phi, rd, ncl);
                                a_acc += wgt * nj * phi;
                                c32 += (r2 > R(0)) ? static_cast<unsigned>(wgt) : 0u;
                                cl32 += ncl * static_cast<unsigned>(wgt);
                            }
                            if (act) {
                                fold(a_acc, A64);
                                cnt += c32;
                                nclamp += cl32;
                            }
                        } else {
#pragma unroll 2
                            for (int jj = 0; jj < jn; ++jj) {
                                const P pj = sp[jj];
                                const R nj = sn[jj];
                                const R dx = xs - pj.x, dy = ys - pj.y, dz = zs - pj.z;
                                const R r2 = h2[0] * (dx * dx) + h2[1] * (dy * dy) + h2[2] * (dz * dz);
                                if (use_cut && beyond(r2, dx, dy, dz, cut)) continue;
                                R phi, rd = 0;
                                unsigned ncl = 0;
                                pair_phi<POT, R>(r2, qi, pj.w, inv_qi, qi2, K, tb, phi, rd, ncl);
                                a_acc += nj * phi;
                                if (POT) u_acc += nj * rd;
                                c32 += (r2 > R(0)) ? 1u : 0u;
                                cl32 += ncl;
                            }
                            if (act) {
                                if (POT) {
                                    fold(a_acc, A64);
                                    fold(u_acc, U64);
                                    cnt += c32;
                                    nclamp += cl32;
                                } else {
                                    double t = 0.0;
                                    fold(a_acc, t);
                                    A64 += 2.0 * t;
                                    cnt += 2ull * c32;
                                    nclamp += 2ull * cl32;
                                }
                            }
                        }
                    }
            __syncthreads();
        }
        if (POT) {
            if (act) {
                atomicAdd(pp.A + ig, A64);
                atomicAdd(pp.U + ig, static_cast<double>(ni) * U64);
            }
        } else {
            const double e = act ? static_cast<double>(ni) * A64 : 0.0;
            const double es = block_sum<double>(e, red);
            if (threadIdx.x == 0) atomicAdd(&pp.stats->E_pair, es);
        }
        const unsigned long long cs = block_sum<unsigned long long>(act ? cnt : 0ull, redu);
        if (threadIdx.x == 0) atomicAdd(&pp.stats->pairs, cs);
        const unsigned long long cl = block_sum<unsigned long long>(act ? nclamp : 0ull, redu);
        if (threadIdx.x == 0) {
            atomicAdd(&pp.stats->clamped, cl);
            atomicAdd(&pp.stats->evals, evals);
        }
    }
}

// The kernel at given (r, q_i, q_j), for isolated checks of the interpolation.
template <typename R>
__global__ void k_kernel_eval(const PairShared sh, int64_t npts, const double *r,
                              const double *qi, const double *qj, double *phi, double *rd) {
    Table<R> tb;
    tb.S = sh.S;
    tb.g = sizeof(R) == 4 ? reinterpret_cast<const R *>(sh.tab32) : reinterpret_cast<const R *>(sh.tab64);
    tb.s = 0;
    tb.k0 = 0;
    tb.kn = 0;
    Consts<R> K;
    make_consts<R>(sh, K);
    for (int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; p < npts;
         p += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const R rr = static_cast<R>(r[p]);
        const R a = static_cast<R>(qi[p]), b = static_cast<R>(qj[p]);
        R ph, rdv = 0;
        unsigned ncl = 0;
        pair_phi<true, R>(rr * rr, a, b, R(1) / a, a * a, K, tb, ph, rdv, ncl);
        phi[p] = static_cast<double>(ph);
        rd[p] = static_cast<double>(rdv);
    }
}

template <typename R, int MODE, int NT>
int launch_one(const PairLaunch &pl, int nctas, size_t smem, cudaStream_t st) {
    auto kern = k_pair<R, MODE, NT>;
    VDWDF_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        static_cast<int>(smem)));
    kern<<<nctas, NT, smem, st>>>(pl);
    count_launches(1);
    VDWDF_CUDA_TRY(cudaGetLastError());
    return VDWDF_OK;
}

template <typename R, int MODE>
int launch_nt(int threads, const PairLaunch &pl, int nctas, size_t smem, cudaStream_t st) {
    switch (threads) {
        case 256: return launch_one<R, MODE, 256>(pl, nctas, smem, st);
        case 1024: return launch_one<R, MODE, 1024>(pl, nctas, smem, st);
        default: return launch_one<R, MODE, 512>(pl, nctas, smem, st);
    }
}

}  // namespace

int pair_smem_bytes(int precision, int ksn, int S) {
    const size_t pt = precision == VDWDF_FP64 ? sizeof(dvec4) + sizeof(double) : sizeof(float4) + sizeof(float);
    size_t b = pt * kJT + 64 * sizeof(double);
    if (precision != VDWDF_FP64) b += static_cast<size_t>(ksn) * S * sizeof(float);
    return static_cast<int>(b);
}

int launch_pair(int precision, bool potential, int threads, const PairLaunch &pl, int nctas,
                cudaStream_t st) {
    const size_t smem = static_cast<size_t>(pair_smem_bytes(precision, pl.sh.ksn, pl.sh.S));
    if (precision == VDWDF_FP64)
        return potential ? launch_nt<double, 1>(threads, pl, nctas, smem, st)
                         : launch_nt<double, 0>(threads, pl, nctas, smem, st);
    return potential ? launch_nt<float, 1>(threads, pl, nctas, smem, st)
                     : launch_nt<float, 0>(threads, pl, nctas, smem, st);
}

int launch_kernel_eval(int precision, const PairShared &sh, int64_t npts, const double *r,
                       const double *qi, const double *qj, double *phi, double *rdphi,
                       cudaStream_t st) {
    const int bs = 256;
    int64_t nb = (npts + bs - 1) / bs;
    if (nb > 65535) nb = 65535;
    if (nb < 1) nb = 1;
    if (precision == VDWDF_FP64)
        k_kernel_eval<double><<<static_cast<int>(nb), bs, 0, st>>>(sh, npts, r, qi, qj, phi, rdphi);
    else
        k_kernel_eval<float><<<static_cast<int>(nb), bs, 0, st>>>(sh, npts, r, qi, qj, phi, rdphi);
    count_launches(1);
    VDWDF_CUDA_TRY(cudaGetLastError());
    return VDWDF_OK;
}

}  // namespace vdwdf
