// Pair kernels of the vdW-DF double sum (paper section 2, eq. (2)) and of its
// adjoint, with periodic images under a spherical cutoff (section 3).
//
// For active points i, j and image vectors L (periodic axes),
//   r = |r_i - r_j + L|,  D = r (q_i + q_j)/2,  delta = |q_i - q_j|/(q_i + q_j),
//   phi = bicubic B-spline of the node table at (D, delta)         if D <= Dmax,
//   phi = rho(delta) phi17,  phi17 = -C / (d1^2 d2^2 (d1^2 + d2^2))   otherwise,
// d1 = q_i r, d2 = q_j r (section 2: the kernel "can be redefined to depend on two
// quantities D and delta"; Dion eq. 17 for large D, scaled by the cubic spline
// rho of phi(Dmax, delta) / phi17(Dmax, delta) so that phi is continuous at Dmax).
// Energy mode sums each unordered pair once with weight 2 (phi is symmetric in
// i, j); potential mode gives, per point,
//   A_i = sum_{j,L} n_j phi,   U_i = n_i sum_{j,L} n_j r dphi/dd1,
//   r dphi/dd1 = r/2 phi_D + (1 - ds)/(q_i + q_j) phi_ds,  ds = (q_i - q_j)/(q_i + q_j),
// and beyond the table rho r dphi17/dd1 + phi17 (1 - ds)/(q_i + q_j) rho_ds with
// r dphi17/dd1 = -2 phi17 (1/q_i + q_i/(q_i^2 + q_j^2)).
//
// Work decomposition: persistent CTAs keep a band of B-spline rows resident in
// shared memory (FP32 path, staged once).  Each warp then works on its own:
// it pulls work items (instance, tile of kTile i points, range of j tiles) from
// one queue in global memory, culls every (j tile, image) against its i tile
// by bounding boxes, stages surviving j tiles in a private shared-memory
// buffer (warp-synchronous, no block barrier), and runs the pair loop with
// each lane owning one i and the j points read as broadcasts.  FP32 partial
// sums over one j tile are folded into FP64 accumulators.  The work loop is
// bounded (max_iters); nothing waits on another warp or CTA.
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

// Cubic B-spline weights times 6 and their t-derivatives times 6.
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
    const R *g;      // bicubic coefficients / 36 in global memory, row stride S
    const R *rho;    // rho(delta) coefficients / 6 (after the bicubic block)
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

// One pair: phi and (POT) r dphi/dd1, r dphi/dd2; counts a clamped delta.
// With ds = (q_i - q_j)/(q_i + q_j): dds/dd1 = (1 - ds)/(2D), dds/dd2 = -(1 + ds)/(2D).
template <bool POT, typename R>
__device__ __forceinline__ void pair_phi(R r2, R qi, R qj, R inv_qi, R qi2, const Consts<R> &K,
                                         const Table<R> &tb, R &phi, R &rd, R &rd2, unsigned &ncl) {
    const R r = rlen(r2);
    const R sq = qi + qj;
    const R dq = qi - qj;
    const R isq = recip(sq);
    // delta cell; beyond the last node the spline continues linearly with its end
    // slope (it has zero curvature there): the weights become w(u) + e w'(u), e the
    // distance past the node in cells.  No index leaves the table.
    const R dl = fabs(dq) * isq;
    const R td0 = dl * K.cd;
    const bool cl = td0 > K.tdmax;
    ncl += cl ? 1u : 0u;
    R td = fmin(fmax(td0, R(0)), K.tdclamp);
    R u;
    int l = floor_split(td, u);
    if (sizeof(R) == 8 && l > K.lmax) {  // FP64 keeps the exact end node: last cell at u = 1
        l = K.lmax;
        u = td - R(l);
    }
    R wd[4], dwd[4];
    bw<R>(u, wd);
    if (POT || cl) bdw<R>(u, dwd);
    if (cl) {
        const R e = td0 - td;
#pragma unroll
        for (int n = 0; n < 4; ++n) wd[n] += e * dwd[n];
    }
    const R sgn1 = dq > R(0) ? (R(1) - dl) : -(R(1) + dl);   // sign(ds) (1 - ds)
    const R sgn2 = dq > R(0) ? (R(1) + dl) : -(R(1) - dl);   // sign(ds) (1 + ds)
    R tD = r * sq * K.cD;
    // the table is read only for 0 <= tD <= nD - 1 (false for NaN as well)
    if (tD >= R(0) && tD <= K.tDmax) {
        tD = fmin(tD, K.tDclamp);
        R t;
        int k = floor_split(tD, t);
        if (sizeof(R) == 8 && k > K.kmax) {
            k = K.kmax;
            t = tD - R(k);
        }
        R wD[4], dwD[4];
        bw<R>(t, wD);
        if (POT) bdw<R>(t, dwD);
        R pt = 0, pu = 0;
        interp<POT, R>(tb, k, l, wD, dwD, wd, dwd, phi, pt, pu);
        if (POT) {
            const R a = r * K.cD * pt, b = isq * K.cd * pu;
            rd = a + b * sgn1;
            rd2 = a - b * sgn2;
        }
    } else {
        const R r4 = r2 * r2;
        const R qj2 = qj * qj;
        const R s2 = qi2 + qj2;
        const R p17 = -K.C * recip(r4 * r2 * qi2 * qj2 * s2);
        const R *rc = tb.rho + l;
        const R c0 = __ldg(rc), c1 = __ldg(rc + 1), c2 = __ldg(rc + 2), c3 = __ldg(rc + 3);
        const R rho = wd[0] * c0 + wd[1] * c1 + wd[2] * c2 + wd[3] * c3;
        phi = rho * p17;
        if (POT) {
            const R drho = dwd[0] * c0 + dwd[1] * c1 + dwd[2] * c2 + dwd[3] * c3;
            const R is2 = recip(s2);
            const R b = p17 * isq * K.cd * drho;
            rd = rho * (R(-2) * p17 * (inv_qi + qi * is2)) + b * sgn1;
            rd2 = rho * (R(-2) * p17 * (recip(qj) + qj * is2)) - b * sgn2;
        }
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

template <typename R>
__device__ void make_table(const PairShared &sh, Table<R> &tb) {
    tb.S = sh.S;
    tb.g = sizeof(R) == 4 ? reinterpret_cast<const R *>(sh.tab32) : reinterpret_cast<const R *>(sh.tab64);
    tb.rho = tb.g + static_cast<size_t>(sh.nD + 2) * sh.S;
    tb.s = 0;
    tb.k0 = 0;
    tb.kn = 0;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
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

// Per-warp running totals, flushed to the instance's counters when the warp
// moves to another instance and at exit (lane 0 holds the warp's total).
struct WarpTotals {
    double E;
    unsigned long long pairs, evals, clamped;
    int inst;
};

__device__ __forceinline__ void flush(WarpTotals &t, const PairLaunch &pl, bool energy) {
    const double E = warp_sum(t.E);
    const unsigned long long pairs = warp_sum(t.pairs), clamped = warp_sum(t.clamped);
    if (t.inst >= 0 && (threadIdx.x & 31) == 0) {
        Stats *s = pl.inst[t.inst].stats;
        if (energy && E != 0.0) atomicAdd(&s->E_pair, E);
        if (pairs) atomicAdd(&s->pairs, pairs);
        if (t.evals) atomicAdd(&s->evals, t.evals);
        if (clamped) atomicAdd(&s->clamped, clamped);
    }
    t.E = 0.0;
    t.pairs = t.evals = t.clamped = 0;
}

// MODE 0: energy (unordered pairs), MODE 1: potential (A, U per point).
template <typename R, int MODE, int NT>
__global__ void __launch_bounds__(NT, 1) k_pair(const __grid_constant__ PairLaunch pl) {
    constexpr bool POT = (MODE == 1);
    constexpr int NW = NT / 32;
    using P = typename PT<R>::P;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ unsigned int s_prefix[kMaxInst + 1];
    __shared__ int s_C[kMaxInst];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    P *sp = reinterpret_cast<P *>(smem_raw) + warp * kTile;
    R *sn = reinterpret_cast<R *>(smem_raw + sizeof(P) * kTile * NW) + warp * kTile;

    const PairShared &sh = pl.sh;
    Table<R> tb;
    make_table<R>(sh, tb);
    Consts<R> K;
    make_consts<R>(sh, K);
    if constexpr (sizeof(R) == 4) {
        float *band = reinterpret_cast<float *>(smem_raw + (sizeof(P) + sizeof(R)) * kTile * NW);
        tb.s = static_cast<uint32_t>(__cvta_generic_to_shared(band));
        tb.k0 = sh.ks0;
        tb.kn = sh.ksn;
        const int nb = sh.ksn * sh.S;
        const float *src = sh.tab32 + static_cast<size_t>(sh.ks0) * sh.S;
        for (int e = threadIdx.x; e < nb; e += NT) band[e] = __ldg(src + e);
    }
    // work items per instance: (i tiles) x (chunks of jtiles_per_item j tiles)
    if (threadIdx.x == 0) {
        unsigned int acc = 0;
        for (int k = 0; k < pl.ninst; ++k) {
            const int na = pl.inst[k].stats->n_active;
            const int nT = (na + kTile - 1) / kTile;
            const int C = max(1, (nT + sh.jtiles_per_item - 1) / sh.jtiles_per_item);
            s_prefix[k] = acc;
            s_C[k] = C;
            acc += static_cast<unsigned int>(pair_items(na, sh.jtiles_per_item));
        }
        s_prefix[pl.ninst] = acc;
    }
    __syncthreads();  // the only block barrier: table band and item counts ready
    const unsigned int n_items = min(s_prefix[pl.ninst], sh.item_limit);

    WarpTotals tot;
    tot.E = 0.0;
    tot.pairs = tot.evals = tot.clamped = 0;
    tot.inst = -1;

    for (unsigned int iter = 0;; ++iter) {
        if (iter >= sh.max_iters) {
            if (lane == 0) atomicAdd(&pl.inst[0].stats->guard_trips, 1u);
            break;
        }
        unsigned int item = 0;
        if (lane == 0) item = atomicAdd(sh.queue, 1u);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= n_items) break;
        int k = 0;
        while (k + 1 < pl.ninst && item >= s_prefix[k + 1]) ++k;
        if (k != tot.inst) {
            flush(tot, pl, !POT);
            tot.inst = k;
        }
        const PairParams &pp = pl.inst[k];
        const unsigned int local = item - s_prefix[k];
        const int C = s_C[k];
        const int I = static_cast<int>(local / C), c = static_cast<int>(local % C);
        const int n_act = pp.stats->n_active;
        const int nT = (n_act + kTile - 1) / kTile;
        const int Js = I;  // i <-> j folded: j tiles from the i tile on
        const int J0 = Js + c * sh.jtiles_per_item;
        const int J1 = min(nT, J0 + sh.jtiles_per_item);
        if (J0 >= J1) {
            if (!POT && lane == 0 && sh.item_E && item < sh.item_cap) sh.item_E[item] = 0.0;
            continue;
        }

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

        const int ig = I * kTile + lane;
        const bool act = ig < n_act;
        const int ni_act = min(kTile, n_act - I * kTile);
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
        const float4 ib0 = __ldg(pp.blo + I), ib1 = __ldg(pp.bhi + I);
        const float ilo[3] = {ib0.x, ib0.y, ib0.z}, ihi[3] = {ib1.x, ib1.y, ib1.z};
        double A64 = 0.0, U64 = 0.0;
        unsigned int cnt = 0, nclamp = 0;
        for (int J = J0; J < J1; ++J) {
            const int jb = J * kTile;
            const int jn = min(kTile, n_act - jb);
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
            __syncwarp();
            if (lane < jn) {
                sp[lane] = PT<R>::load(pts, jb + lane);
                sn[lane] = __ldg(nsrc + jb + lane);
            }
            __syncwarp();
            R a_acc = 0, u_acc = 0;  // i side (this lane's i)
            R ja = 0, ju = 0;        // j side: lane L collects j = jb + L
            // weights: off-diagonal tiles count every pair for i and for j; in the
            // diagonal tile j > i counts for both, j == i (self and self-images) for i only
            const bool diag = (J == I);
            for (int m0 = mlo[0]; m0 <= mhi[0]; ++m0)
                for (int m1 = mlo[1]; m1 <= mhi[1]; ++m1)
                    for (int m2 = mlo[2]; m2 <= mhi[2]; ++m2) {
                        const int mm[3] = {m0, m1, m2};
                        if (use_cut && box_gap2(ilo, ihi, jl, jh, mm, dims, h2f) > rc2_box) continue;
                        const R xs = xi + static_cast<R>(m0 * dims[0]);
                        const R ys = yi + static_cast<R>(m1 * dims[1]);
                        const R zs = zi + static_cast<R>(m2 * dims[2]);
                        tot.evals += static_cast<unsigned long long>(jn) * static_cast<unsigned long long>(ni_act);
#pragma unroll 2
                        for (int jj = 0; jj < jn; ++jj) {
                            const P pj = sp[jj];
                            const R nj = sn[jj];
                            const R dx = xs - pj.x, dy = ys - pj.y, dz = zs - pj.z;
                            const R r2 = h2[0] * (dx * dx) + h2[1] * (dy * dy) + h2[2] * (dz * dz);
                            const bool both = !diag || jj > lane;
                            const bool inside = act && (both || jj == lane) && !(use_cut && beyond(r2, dx, dy, dz, cut));
                            R cA = 0, cU = 0;
                            if (inside) {
                                R phi, rd = 0, rd2 = 0;
                                unsigned ncl = 0;
                                pair_phi<POT, R>(r2, qi, pj.w, inv_qi, qi2, K, tb, phi, rd, rd2, ncl);
                                const unsigned wt = both ? 2u : 1u;  // ordered pairs represented
                                if (POT) {
                                    a_acc += nj * phi;
                                    u_acc += nj * rd;
                                    if (both) {
                                        cA = ni * phi;
                                        cU = ni * rd2;
                                    }
                                } else {
                                    a_acc += static_cast<R>(wt) * nj * phi;
                                }
                                cnt += (r2 > R(0)) ? wt : 0u;
                                nclamp += ncl * wt;
                            }
                            if (POT && __any_sync(0xffffffffu, cA != R(0) || cU != R(0))) {
                                cA = warp_sum(cA);
                                cU = warp_sum(cU);
                                if (lane == jj) {
                                    ja += cA;
                                    ju += cU;
                                }
                            }
                        }
                    }
            A64 += static_cast<double>(a_acc);
            U64 += static_cast<double>(u_acc);
            if (POT && lane < jn) {
                if (ja != R(0)) atomicAdd(pp.A + jb + lane, static_cast<double>(ja));
                if (ju != R(0)) atomicAdd(pp.U + jb + lane, static_cast<double>(sn[lane]) * static_cast<double>(ju));
            }
        }
        if (act) {
            if (POT) {
                if (A64 != 0.0) atomicAdd(pp.A + ig, A64);
                if (U64 != 0.0) atomicAdd(pp.U + ig, static_cast<double>(ni) * U64);
            }
            tot.pairs += cnt;
            tot.clamped += nclamp;
        }
        if (!POT) {
            // the item's energy partial, summed over lanes in a fixed order
            const double e = warp_sum(act ? static_cast<double>(ni) * A64 : 0.0);
            if (lane == 0) {
                if (sh.item_E && item < sh.item_cap)
                    sh.item_E[item] = e;
                else
                    tot.E += e;
            }
        }
    }
    flush(tot, pl, !POT);
}

// Fixed-order sum of an instance's energy-mode item partials (block k: instance k).
__global__ void k_reduce_items(const __grid_constant__ PairLaunch pl) {
    const int k = blockIdx.x;
    if (k >= pl.ninst) return;
    unsigned int lo = 0;
    for (int t = 0; t < k; ++t)
        lo += static_cast<unsigned int>(pair_items(pl.inst[t].stats->n_active, pl.sh.jtiles_per_item));
    const unsigned int n = static_cast<unsigned int>(pair_items(pl.inst[k].stats->n_active, pl.sh.jtiles_per_item));
    const unsigned int hi = min(lo + n, pl.sh.item_cap);
    double s = 0.0;
    for (unsigned int i = lo + threadIdx.x; i < hi; i += blockDim.x) s += pl.sh.item_E[i];
    __shared__ double part[256];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (static_cast<int>(threadIdx.x) < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(&pl.inst[k].stats->E_pair, part[0]);
}

// The kernel at given (r, q_i, q_j), for isolated checks of the interpolation.
template <typename R>
__global__ void k_kernel_eval(const PairShared sh, int64_t npts, const double *r,
                              const double *qi, const double *qj, double *phi, double *rd) {
    Table<R> tb;
    make_table<R>(sh, tb);
    Consts<R> K;
    make_consts<R>(sh, K);
    for (int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; p < npts;
         p += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const R rr = static_cast<R>(r[p]);
        const R a = static_cast<R>(qi[p]), b = static_cast<R>(qj[p]);
        R ph, rdv = 0, rd2 = 0;
        unsigned ncl = 0;
        pair_phi<true, R>(rr * rr, a, b, R(1) / a, a * a, K, tb, ph, rdv, rd2, ncl);
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

int pair_smem_bytes(int precision, int threads, int ksn, int S) {
    const size_t pt = precision == VDWDF_FP64 ? sizeof(dvec4) + sizeof(double) : sizeof(float4) + sizeof(float);
    size_t b = pt * kTile * static_cast<size_t>(threads / 32);
    if (precision != VDWDF_FP64) b += static_cast<size_t>(ksn) * S * sizeof(float);
    return static_cast<int>(b);
}

int launch_pair(int precision, bool potential, int threads, const PairLaunch &pl, int nctas,
                cudaStream_t st) {
    const size_t smem = static_cast<size_t>(pair_smem_bytes(precision, threads, pl.sh.ksn, pl.sh.S));
    if (precision == VDWDF_FP64)
        return potential ? launch_nt<double, 1>(threads, pl, nctas, smem, st)
                         : launch_nt<double, 0>(threads, pl, nctas, smem, st);
    return potential ? launch_nt<float, 1>(threads, pl, nctas, smem, st)
                     : launch_nt<float, 0>(threads, pl, nctas, smem, st);
}

int launch_reduce_items(const PairLaunch &pl, cudaStream_t st) {
    if (!pl.sh.item_E) return VDWDF_OK;
    k_reduce_items<<<pl.ninst, 256, 0, st>>>(pl);
    count_launches(1);
    VDWDF_CUDA_TRY(cudaGetLastError());
    return VDWDF_OK;
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
