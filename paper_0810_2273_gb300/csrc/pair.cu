// Pair kernels of the vdW-DF double sum (paper section 2, eq. (2)) and of its
// adjoint, with periodic images under a spherical cutoff (section 3).
//
// For active points i, j and image vectors L (periodic axes),
//   r = |r_i - r_j + L|,  D = r (q_i + q_j)/2,  delta = |q_i - q_j|/(q_i + q_j),
//   phi = bicubic B-spline of the node table at (D, delta)         if D <= Dmax,
//   phi = g phi17,  phi17 = -C / (d1^2 d2^2 (d1^2 + d2^2))            otherwise,
// d1 = q_i r, d2 = q_j r (section 2: the kernel "can be redefined to depend on two
// quantities D and delta"; Dion eq. 17 for large D).  The factor
//   g = rho(delta*) + (1 - rho(0)) (1 - (Dmax/D)^2),  delta* = max(0, 1 - min(d1, d2)/Dmax),
// with rho the cubic spline of phi(Dmax, delta) / phi17(Dmax, delta), carries the
// table's departure from eq. 17 at Dmax to larger D along the smaller argument
// (on which that departure depends once the larger one is big), so phi is
// continuous at Dmax and tends to eq. 17 as both arguments grow.
// Energy mode sums each unordered pair once with weight 2 (phi is symmetric in
// i, j); potential mode gives, per point,
//   A_i = sum_{j,L} n_j phi,   U_i = n_i sum_{j,L} n_j r dphi/dd1,
//   r dphi/dd1 = r/2 phi_D + (1 - ds)/(q_i + q_j) phi_ds,  ds = (q_i - q_j)/(q_i + q_j),
// and beyond the table g r dphi17/dd1 + phi17 r dg/dd1 with
// r dphi17/dd1 = -2 phi17 (1/q_i + q_i/(q_i^2 + q_j^2)) and
// r dg/dd1 = (1 - rho(0)) (Dmax/D)^2 r/D - [d1 < d2] rho'(delta*) r/Dmax.
//
// Work decomposition: persistent CTAs keep a band of B-spline rows resident in
// shared memory (FP32 path, staged once; which rows is chosen on the device from
// a sampled histogram of the call's D cells).  Each warp then works on its own:
// it pulls work items (instance, tile of kTile i points, range of j tiles) from
// one queue in global memory, culls every (j tile, image) against its i tile
// by bounding boxes and then every (j point, image) against the i box, stages
// surviving j tiles in a private shared-memory buffer (warp-synchronous, no
// block barrier), and runs the pair loop with each lane owning one i, the j
// points read as broadcasts and the images of a pair innermost.  In FP32 two j
// points go through the loop together, one in each half of packed FP32x2
// arithmetic.  FP32 partial sums over one j tile are folded into FP64
// accumulators.  The work loop is
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

// Two FP32 values per instruction (sm_100-family packed FP32 arithmetic).
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 add2_rm(float2 a, float2 b) {
    unsigned long long d;
    asm("add.rm.f32x2 %0, %1, %2;"
        : "=l"(d)
        : "l"(*reinterpret_cast<const unsigned long long *>(&a)),
          "l"(*reinterpret_cast<const unsigned long long *>(&b)));
    return *reinterpret_cast<const float2 *>(&d);
}

// floor_split of two values at once (both non-negative and below 2^22)
__device__ __forceinline__ float2 floor_split2(float2 x, int &k0, int &k1) {
    const float2 b = add2_rm(x, f2(12582912.0f));
    k0 = __float_as_int(b.x) - 0x4B400000;
    k1 = __float_as_int(b.y) - 0x4B400000;
    const float2 f = fma2(f2(-1.0f), f2(12582912.0f), b);  // floor(x), exact
    return fma2(f, f2(-1.0f), x);                            // x - floor(x), exact
}

__device__ __forceinline__ void bw2(float2 t, float2 w[4]) {
    const float2 t2 = mul2(t, t), t3 = mul2(t2, t), s = fma2(t, f2(-1.0f), f2(1.0f));
    w[0] = mul2(mul2(s, s), s);
    w[1] = fma2(f2(3.0f), t3, fma2(f2(-6.0f), t2, f2(4.0f)));
    w[2] = fma2(f2(-3.0f), t3, fma2(f2(3.0f), t2, fma2(f2(3.0f), t, f2(1.0f))));
    w[3] = t3;
}
__device__ __forceinline__ void bdw2(float2 t, float2 d[4]) {
    const float2 t2 = mul2(t, t), s = fma2(t, f2(-1.0f), f2(1.0f));
    d[0] = mul2(f2(-3.0f), mul2(s, s));
    d[1] = fma2(f2(9.0f), t2, mul2(f2(-12.0f), t));
    d[2] = fma2(f2(-9.0f), t2, fma2(f2(6.0f), t, f2(3.0f)));
    d[3] = mul2(f2(3.0f), t2);
}

// The delta-derivative weights sum to zero, so sum_n dwd[n] c[n] is taken as
// sum_{n>=1} dwd[n] (c[n] - c[0]): neighbouring coefficients differ little and
// their differences are exact, which keeps the small derivative of an O(phi)
// row free of the cancellation that would otherwise scale its error by the
// number of delta cells.
template <bool POT, typename R>
__device__ __forceinline__ void combine(const R c[4][4], const R wD[4], const R dwD[4],
                                        const R wd[4], const R dwd[4], R &phi, R &pt, R &pu) {
    R p = 0, a = 0, b = 0;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const R row = wd[0] * c[m][0] + wd[1] * c[m][1] + wd[2] * c[m][2] + wd[3] * c[m][3];
        p += wD[m] * row;
        if (POT) {
            const R drow = dwd[1] * (c[m][1] - c[m][0]) + dwd[2] * (c[m][2] - c[m][0]) +
                           dwd[3] * (c[m][3] - c[m][0]);
            a += dwD[m] * row;
            b += wD[m] * drow;
        }
    }
    phi = p;
    pt = a;
    pu = b;
}

template <typename R>
using Consts = LoopConsts<R>;

template <typename R>
struct Table {
    const R *g;      // bicubic coefficients / 36 in global memory, row stride S
    const R *rho;    // rho(delta) coefficients / 6 (after the bicubic block)
    uint32_t s;      // shared-memory address of the resident band (FP32), row stride SB
    int k0, kn;      // band rows [k0, k0 + kn)
    int S, SB;
};

template <bool POT, typename R>
__device__ __forceinline__ void interp(const Table<R> &tb, int k, int l, const R wD[4],
                                       const R dwD[4], const R wd[4], const R dwd[4], R &p, R &pt,
                                       R &pu) {
    R c[4][4];
    if (sizeof(R) == 4 && k >= tb.k0 && k + 4 <= tb.k0 + tb.kn) {
        const uint32_t a0 = tb.s + 4u * static_cast<uint32_t>((k - tb.k0) * tb.SB + l);
        const uint32_t rs = 4u * static_cast<uint32_t>(tb.SB);
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

// The delta-dependent part of a pair, shared by all its periodic images: the
// delta cell and weights, the scale from r to the table's D coordinate, and the
// factors that turn the delta-derivative into r dphi/dd1 and r dphi/dd2.
// With ds = (q_i - q_j)/(q_i + q_j): dds/dd1 = (1 - ds)/(2D), dds/dd2 = -(1 + ds)/(2D),
// so b1 = cd sign(ds) (1 - ds)/(q_i + q_j) and b2 = -cd sign(ds) (1 + ds)/(q_i + q_j).
template <typename R>
struct Delta {
    R sqcD, b1, b2;  // (q_i + q_j) cD; the delta-derivative factors
    R wd[4], dwd[4];
    int l;
    bool cl;  // delta beyond the last node (weights continued linearly)
};

template <bool POT, typename R>
__device__ __forceinline__ void delta_part(R qi, R qj, const Consts<R> &K, Delta<R> &d) {
    const R sq = qi + qj;
    const R dq = qi - qj;
    const R isq = recip(sq);
    // beyond the last node the spline continues linearly with its end slope (it has
    // zero curvature there): the weights become w(u) + e w'(u), e the distance past
    // the node in cells.  No index leaves the table.
    const R dl = fabs(dq) * isq;
    const R td0 = dl * K.cd;
    d.cl = td0 > K.tdmax;
    const R td = fmin(fmax(td0, R(0)), K.tdclamp);
    R u;
    int l = floor_split(td, u);
    if (sizeof(R) == 8 && l > K.lmax) {  // FP64 keeps the exact end node: last cell at u = 1
        l = K.lmax;
        u = td - R(l);
    }
    d.l = l;
    bw<R>(u, d.wd);
    if (POT || d.cl) bdw<R>(u, d.dwd);
    if (d.cl) {
        const R e = td0 - td;
#pragma unroll
        for (int n = 0; n < 4; ++n) d.wd[n] += e * d.dwd[n];
    }
    const R bq = isq * K.cd;
    d.sqcD = sq * K.cD;
    d.b1 = bq * (dq > R(0) ? (R(1) - dl) : -(R(1) + dl));   // sign(ds) (1 - ds)
    d.b2 = -bq * (dq > R(0) ? (R(1) + dl) : -(R(1) - dl));  // sign(ds) (1 + ds)
}

// The delta parts of two pairs (i, j0) and (i, j1) in the two halves of packed
// FP32 values: the arithmetic of delta_part, two lanes per instruction.
struct Delta2 {
    float2 sqcD, b1, b2;
    float2 wd[4], dwd[4];
    int l0, l1;
};

template <bool POT>
__device__ __forceinline__ void delta_part2(float qi, float2 qj, const Consts<float> &K, Delta2 &d,
                                            bool &cl0, bool &cl1) {
    const float2 sq = add2(f2(qi), qj);
    const float2 dq = fma2(qj, f2(-1.0f), f2(qi));  // q_i - q_j, one rounding
    const float2 isq = make_float2(recip(sq.x), recip(sq.y));
    const float2 dl = mul2(make_float2(fabsf(dq.x), fabsf(dq.y)), isq);
    const float2 td0 = mul2(dl, f2(K.cd));
    cl0 = td0.x > K.tdmax;
    cl1 = td0.y > K.tdmax;
    const float2 td = make_float2(fminf(fmaxf(td0.x, 0.0f), K.tdclamp), fminf(fmaxf(td0.y, 0.0f), K.tdclamp));
    const float2 u = floor_split2(td, d.l0, d.l1);
    bw2(u, d.wd);
    if (POT || cl0 || cl1) bdw2(u, d.dwd);
    if (cl0 || cl1) {
        const float2 e = fma2(td, f2(-1.0f), td0);  // 0 in a half that is not past the node
#pragma unroll
        for (int n = 0; n < 4; ++n) d.wd[n] = fma2(e, d.dwd[n], d.wd[n]);
    }
    const float2 bq = mul2(isq, f2(K.cd));
    const float2 one = f2(1.0f);
    const float2 om = fma2(dl, f2(-1.0f), one), op = add2(dl, one);  // 1 - |ds|, 1 + |ds|
    d.sqcD = mul2(sq, f2(K.cD));
    d.b1 = mul2(bq, make_float2(dq.x > 0.0f ? om.x : -op.x, dq.y > 0.0f ? om.y : -op.y));
    d.b2 = mul2(bq, make_float2(dq.x > 0.0f ? -op.x : om.x, dq.y > 0.0f ? -op.y : om.y));
}

// Half s of a packed delta part as a scalar one (register renaming only).
template <int S>
__device__ __forceinline__ Delta<float> delta_half(const Delta2 &d) {
    Delta<float> r;
    r.sqcD = S ? d.sqcD.y : d.sqcD.x;
    r.b1 = S ? d.b1.y : d.b1.x;
    r.b2 = S ? d.b2.y : d.b2.x;
#pragma unroll
    for (int n = 0; n < 4; ++n) {
        r.wd[n] = S ? d.wd[n].y : d.wd[n].x;
        r.dwd[n] = S ? d.dwd[n].y : d.dwd[n].x;
    }
    r.l = S ? d.l1 : d.l0;
    r.cl = false;
    return r;
}

// The distance-dependent part: phi and (POT) r dphi/dd1, r dphi/dd2 at r^2.
template <bool POT, typename R>
__device__ __forceinline__ void dist_part(R r2, R qi, R qj, R inv_qi, R qi2, const Delta<R> &d,
                                          const Consts<R> &K, const Table<R> &tb, R &phi, R &rd,
                                          R &rd2) {
    const R r = rlen(r2);
    R tD = r * d.sqcD;
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
        interp<POT, R>(tb, k, d.l, wD, dwD, d.wd, d.dwd, phi, pt, pu);
        if (POT) {
            const R a = r * K.cD * pt;
            rd = a + pu * d.b1;
            rd2 = a + pu * d.b2;
        }
    } else {
        const R r4 = r2 * r2;
        const R qj2 = qj * qj;
        const R s2 = qi2 + qj2;
        const R p17 = -K.C * recip(r4 * r2 * qi2 * qj2 * s2);
        // rho at delta* = 1 - min(d1, d2)/Dmax, in delta cells; at or below 0 the
        // spline's value at delta = 0 with zero slope (its end condition), past the
        // last node its linear continuation.  No index leaves the rho block.
        const bool i_small = qi < qj;
        const R ts0 = (R(1) - r * fmin(qi, qj) * K.iDmax) * K.cd;
        const bool up = ts0 > R(0);
        const bool past = ts0 > K.tdmax;
        const R ts = fmin(fmax(ts0, R(0)), K.tdclamp);
        R u;
        int l = floor_split(ts, u);
        if (sizeof(R) == 8 && l > K.lmax) {
            l = K.lmax;
            u = ts - R(l);
        }
        R w[4], dw[4];
        bw<R>(u, w);
        const R *rc = tb.rho + l;
        const R c0 = __ldg(rc), c1 = __ldg(rc + 1), c2 = __ldg(rc + 2), c3 = __ldg(rc + 3);
        R rho = w[0] * c0 + w[1] * c1 + w[2] * c2 + w[3] * c3;
        R drho = R(0);  // d rho / d delta*, in cells
        if (POT || past) {
            bdw<R>(u, dw);
            drho = up ? dw[1] * (c1 - c0) + dw[2] * (c2 - c0) + dw[3] * (c3 - c0) : R(0);
            if (past) rho += (ts0 - ts) * drho;
        }
        const R Dr = K.tDmax * recip(tD);  // Dmax / D
        const R Dr2 = Dr * Dr;
        const R g = rho + K.om_rho0 * (R(1) - Dr2);
        phi = g * p17;
        if (POT) {
            const R is2 = recip(s2);
            // (1 - rho(0)) (Dmax/D)^2 r/D with r/D = 2 cD r / tD, and rho'(delta*) r/Dmax
            const R ramp = K.om_rho0 * Dr2 * R(2) * K.cD * r * recip(tD);
            const R sl = drho * K.cd * r * K.iDmax;
            rd = g * (R(-2) * p17 * (inv_qi + qi * is2)) + p17 * (i_small ? ramp - sl : ramp);
            rd2 = g * (R(-2) * p17 * (recip(qj) + qj * is2)) + p17 * (i_small ? ramp : ramp - sl);
        }
    }
}

// One pair: phi and (POT) r dphi/dd1, r dphi/dd2; counts a delta past the last node.
template <bool POT, typename R>
__device__ __forceinline__ void pair_phi(R r2, R qi, R qj, R inv_qi, R qi2, const Consts<R> &K,
                                         const Table<R> &tb, R &phi, R &rd, R &rd2, unsigned &ncl) {
    Delta<R> d;
    delta_part<POT, R>(qi, qj, K, d);
    ncl += d.cl ? 1u : 0u;
    dist_part<POT, R>(r2, qi, qj, inv_qi, qi2, d, K, tb, phi, rd, rd2);
}

template <typename R>
__device__ __forceinline__ void make_consts(const PairShared &sh, Consts<R> &K) {
    if constexpr (sizeof(R) == 4)
        K = sh.k32;
    else
        K = sh.k64;
}

template <typename R>
__device__ void make_table(const PairShared &sh, Table<R> &tb) {
    tb.S = sh.S;
    tb.SB = band_stride(sh.S);
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
    const PairParams *pp;  // FP64 metric and cutoff (kernel parameters), read only
                           // by the recheck near the boundary
    float lo, hi;
};
template <bool SKEW>
__device__ __forceinline__ bool beyond(float r2, float dx, float dy, float dz, const Cut &c) {
    if (r2 > c.hi) return true;
    if (r2 <= c.lo) return false;
    const PairParams &p = *c.pp;
    const double X = dx, Y = dy, Z = dz;
    double e = p.h2[0] * (X * X) + p.h2[1] * (Y * Y) + p.h2[2] * (Z * Z);
    if (SKEW) e += p.g2x[0] * (X * Y) + p.g2x[1] * (X * Z) + p.g2x[2] * (Y * Z);
    return e > p.rc2;
}
template <bool SKEW>
__device__ __forceinline__ bool beyond(double r2, double, double, double, const Cut &c) {
    return r2 > c.pp->rc2;
}

// Squared distance between the i box shifted by image m and the j box.
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

// Skewed cells: squared distance between the Cartesian box of the i tile shifted
// by image m (L = sum_a m_a N_a v_a) and the Cartesian box of the j tile.
__device__ __forceinline__ float box_gap2_cart(const float4 &il, const float4 &ih, const float4 &jl,
                                               const float4 &jh, const int m[3], const int dims[3],
                                               const CellRows &vr) {
    const float s0 = static_cast<float>(m[0] * dims[0]), s1 = static_cast<float>(m[1] * dims[1]),
                s2 = static_cast<float>(m[2] * dims[2]);
    const float L0 = s0 * vr.v[0] + s1 * vr.v[3] + s2 * vr.v[6];
    const float L1 = s0 * vr.v[1] + s1 * vr.v[4] + s2 * vr.v[7];
    const float L2 = s0 * vr.v[2] + s1 * vr.v[5] + s2 * vr.v[8];
    const float g0 = fmaxf(0.0f, fmaxf(il.x + L0 - jh.x, jl.x - ih.x - L0));
    const float g1 = fmaxf(0.0f, fmaxf(il.y + L1 - jh.y, jl.y - ih.y - L1));
    const float g2 = fmaxf(0.0f, fmaxf(il.z + L2 - jh.z, jl.z - ih.z - L2));
    return g0 * g0 + g1 * g1 + g2 * g2;
}

// The counters of a finished work item, summed over the warp and added by lane 0
// to the instance's totals (integer atomics: the totals do not depend on order).
__device__ __forceinline__ void count_item(Stats *s, unsigned cnt, unsigned nclamp, unsigned evals) {
    const unsigned pairs = warp_sum(cnt), clamped = warp_sum(nclamp);
    if ((threadIdx.x & 31) == 0) {
        if (pairs) atomicAdd(&s->pairs, static_cast<unsigned long long>(pairs));
        if (evals) atomicAdd(&s->evals, static_cast<unsigned long long>(evals));
        if (clamped) atomicAdd(&s->clamped, static_cast<unsigned long long>(clamped));
    }
}

// Two evaluations in the resident band at once: half s at cell coordinate tD.s and
// delta row l_s (a half that is not wanted reads no coefficient and returns 0).
// wd, dwd: the delta weights of the two halves.  Returns phi and, with POT, the
// cell-coordinate derivatives pt (along D) and pu (along delta).
template <bool POT>
__device__ __forceinline__ void band_pair2(const Table<float> &tb, float2 tD, int l0, int l1, bool use0,
                                           bool use1, const float2 wdb[4], const float2 dwdb[4],
                                           float2 &p, float2 &pt, float2 &pu) {
    int k0, k1;
    const float2 t = floor_split2(tD, k0, k1);
    float2 wD[4], dwD[4];
    bw2(t, wD);
    if (POT) bdw2(t, dwD);
    const uint32_t a0 = tb.s + 4u * static_cast<uint32_t>((k0 - tb.k0) * tb.SB + l0);
    const uint32_t a1 = tb.s + 4u * static_cast<uint32_t>((k1 - tb.k0) * tb.SB + l1);
    const uint32_t rs = 4u * static_cast<uint32_t>(tb.SB);
    p = f2(0.0f);
    pt = f2(0.0f);
    pu = f2(0.0f);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        float2 c[4];
#pragma unroll
        for (int n = 0; n < 4; ++n)  // an unused half reads nothing
            c[n] = make_float2(use0 ? lds32(a0 + m * rs + 4u * n) : 0.0f, use1 ? lds32(a1 + m * rs + 4u * n) : 0.0f);
        const float2 row = fma2(wdb[3], c[3], fma2(wdb[2], c[2], fma2(wdb[1], c[1], mul2(wdb[0], c[0]))));
        p = fma2(wD[m], row, p);
        if (POT) {
            // delta derivative from exact coefficient differences (see combine);
            // fma(c0, -1, c_n) is c_n - c0 with one rounding
            const float2 m1 = f2(-1.0f);
            const float2 drow = fma2(dwdb[3], fma2(c[0], m1, c[3]),
                                     fma2(dwdb[2], fma2(c[0], m1, c[2]), mul2(dwdb[1], fma2(c[0], m1, c[1]))));
            pt = fma2(dwD[m], row, pt);
            pu = fma2(wD[m], drow, pu);
        }
    }
}

// The same two evaluations from the table's copy in global memory (read-only
// path, rows of stride S), for steps where a half lies off the resident band.
template <bool POT>
__device__ __forceinline__ void table_pair2(const Table<float> &tb, float2 tD, int l0, int l1, bool use0,
                                           bool use1, const float2 wdb[4], const float2 dwdb[4],
                                           float2 &p, float2 &pt, float2 &pu) {
    int k0, k1;
    const float2 t = floor_split2(tD, k0, k1);
    float2 wD[4], dwD[4];
    bw2(t, wD);
    if (POT) bdw2(t, dwD);
    const float *g0 = tb.g + static_cast<size_t>(k0) * tb.S + l0;
    const float *g1 = tb.g + static_cast<size_t>(k1) * tb.S + l1;
    const int rs = tb.S;
    p = f2(0.0f);
    pt = f2(0.0f);
    pu = f2(0.0f);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        float2 c[4];
#pragma unroll
        for (int n = 0; n < 4; ++n)  // an unused half reads nothing
            c[n] = make_float2(use0 ? __ldg(g0 + m * rs + n) : 0.0f, use1 ? __ldg(g1 + m * rs + n) : 0.0f);
        const float2 row = fma2(wdb[3], c[3], fma2(wdb[2], c[2], fma2(wdb[1], c[1], mul2(wdb[0], c[0]))));
        p = fma2(wD[m], row, p);
        if (POT) {
            // delta derivative from exact coefficient differences (see combine);
            // fma(c0, -1, c_n) is c_n - c0 with one rounding
            const float2 m1 = f2(-1.0f);
            const float2 drow = fma2(dwdb[3], fma2(c[0], m1, c[3]),
                                     fma2(dwdb[2], fma2(c[0], m1, c[2]), mul2(dwdb[1], fma2(c[0], m1, c[1]))));
            pt = fma2(dwD[m], row, pt);
            pu = fma2(wD[m], drow, pu);
        }
    }
}

// The images of two j points j0, j1 for one i point (FP32): half 0 runs over the
// images of mask m0 (those of j0), half 1 over m1 (those of j1), one image of each
// per step; a half whose mask is spent idles.  ex, ey, ez: x_i - x_j per half in
// index units (integers, so every shifted difference is exact).  ok0, ok1: the
// pair counts for this lane.  Adds sum_images phi, r dphi/dd1, r dphi/dd2 per half
// to A2, U2, V2 and counts per half the inside evaluations (ins; the self term,
// the one at r = 0, is taken off once per point by the caller).
template <bool POT, bool SKEW>
__device__ __forceinline__ void images2_f32(unsigned m0, unsigned m1, const float4 *simg, float2 ex, float2 ey,
                                            float2 ez, float qi, float inv_qi, float qi2, float2 qj,
                                            const float h2[3], const float g2x[3], bool ok0, bool ok1,
                                            bool use_cut, const Cut &cut, const Delta2 &dp,
                                            const Consts<float> &K, const Table<float> &tb, float band_lo,
                                            float band_hi, float2 &A2, float2 &U2, float2 &V2,
                                            unsigned &ins0, unsigned &ins1) {
    const float2 H0 = f2(h2[0]), H1 = f2(h2[1]), H2 = f2(h2[2]);
    const float2 cD2 = f2(K.cD);
    A2 = f2(0.0f);
    U2 = f2(0.0f);
    V2 = f2(0.0f);
    // band evaluations: r dphi/dd1 = cD r pt + b1 pu with b1, b2 fixed for the j point,
    // so the sums of r pt and of pu over the images are scaled once at the end
    float2 Srpt = f2(0.0f), Spu = f2(0.0f);
    do {
        const bool u0 = m0 != 0u, u1 = m1 != 0u;
        const int i0 = u0 ? __ffs(m0) - 1 : 0;  // a spent half reads a valid slot
        const int i1 = u1 ? __ffs(m1) - 1 : 0;
        m0 &= m0 - 1u;
        m1 &= m1 - 1u;
        const float4 s0 = simg[i0], s1 = simg[i1];
        const float2 dx = add2(ex, make_float2(s0.x, s1.x));
        const float2 dy = add2(ey, make_float2(s0.y, s1.y));
        const float2 dz = add2(ez, make_float2(s0.z, s1.z));
        float2 r2 = mul2(H2, mul2(dz, dz));
        r2 = fma2(H1, mul2(dy, dy), r2);
        r2 = fma2(H0, mul2(dx, dx), r2);
        if (SKEW) {
            r2 = fma2(f2(g2x[0]), mul2(dx, dy), r2);
            r2 = fma2(f2(g2x[1]), mul2(dx, dz), r2);
            r2 = fma2(f2(g2x[2]), mul2(dy, dz), r2);
        }
        const bool in0 = u0 && ok0 && !(use_cut && beyond<SKEW>(r2.x, dx.x, dy.x, dz.x, cut));
        const bool in1 = u1 && ok1 && !(use_cut && beyond<SKEW>(r2.y, dx.y, dy.y, dz.y, cut));
        if (!(in0 || in1)) continue;
        ins0 += in0 ? 1u : 0u;
        ins1 += in1 ? 1u : 0u;
        const float2 rr = mul2(r2, make_float2(rsqrtf(fmaxf(r2.x, 1e-30f)), rsqrtf(fmaxf(r2.y, 1e-30f))));
        const float2 tD = mul2(rr, dp.sqcD);
        const bool f0 = !in0 || (tD.x >= band_lo && tD.x < band_hi);
        const bool f1 = !in1 || (tD.y >= band_lo && tD.y < band_hi);
        // nearly every step has both halves in the band: lay that path out as the
        // fall-through one (measured 7 % faster for E + v than without the hint)
        if (__builtin_expect(f0 && f1, 1)) {
            // both halves in the resident band; an idle half reads nothing: p, pt,
            // pu are 0 there and add nothing
            const float2 tq = make_float2(in0 ? tD.x : band_lo, in1 ? tD.y : band_lo);
            float2 p, pt, pu;
            band_pair2<POT>(tb, tq, dp.l0, dp.l1, in0, in1, dp.wd, dp.dwd, p, pt, pu);
            A2 = add2(A2, p);
            if (POT) {
                Srpt = fma2(rr, pt, Srpt);
                Spu = add2(Spu, pu);
            }
        } else if (POT && (!in0 || tD.x <= K.tDmax) && (!in1 || tD.y <= K.tDmax)) {
            // E + v: a half off the resident band but both on the table: both halves
            // from the table's global copy, packed as in the band (measured 1-2 %
            // faster on the monolayer and the molecule, 1 % slower on the slab;
            // energy mode keeps the scalar path, where it cost registers)
            const float2 tq = make_float2(in0 ? fminf(tD.x, K.tDclamp) : 0.0f, in1 ? fminf(tD.y, K.tDclamp) : 0.0f);
            float2 p, pt, pu;
            table_pair2<POT>(tb, tq, dp.l0, dp.l1, in0, in1, dp.wd, dp.dwd, p, pt, pu);
            A2 = add2(A2, p);
            if (POT) {
                Srpt = fma2(rr, pt, Srpt);
                Spu = add2(Spu, pu);
            }
        } else {
            if (in0) {
                float phi, rd = 0.0f, rd2 = 0.0f;
                dist_part<POT, float>(r2.x, qi, qj.x, inv_qi, qi2, delta_half<0>(dp), K, tb, phi, rd, rd2);
                A2.x += phi;
                U2.x += rd;
                V2.x += rd2;
            }
            if (in1) {
                float phi, rd = 0.0f, rd2 = 0.0f;
                dist_part<POT, float>(r2.y, qi, qj.y, inv_qi, qi2, delta_half<1>(dp), K, tb, phi, rd, rd2);
                A2.y += phi;
                U2.y += rd;
                V2.y += rd2;
            }
        }
    } while ((m0 | m1) != 0u);
    if (POT) {
        const float2 a = mul2(Srpt, cD2);
        U2 = add2(U2, fma2(Spu, dp.b1, a));
        V2 = add2(V2, fma2(Spu, dp.b2, a));
    }
}

// Warp sums of four values: the total of v_k ends in lanes 8k .. 8k+7.  Two
// halving exchanges (each lane keeps half of its values and sends the other
// half) and three butterflies: 8 shuffles instead of 20 for four plain sums.
__device__ __forceinline__ float warp_sum4(float v0, float v1, float v2, float v3) {
    const unsigned lane = threadIdx.x & 31u;
    const bool h16 = (lane & 16u) != 0u, h8 = (lane & 8u) != 0u;
    const float w0 = (h16 ? v2 : v0) + __shfl_xor_sync(0xffffffffu, h16 ? v0 : v2, 16);
    const float w1 = (h16 ? v3 : v1) + __shfl_xor_sync(0xffffffffu, h16 ? v1 : v3, 16);
    float x = (h8 ? w1 : w0) + __shfl_xor_sync(0xffffffffu, h8 ? w0 : w1, 8);
    x += __shfl_xor_sync(0xffffffffu, x, 4);
    x += __shfl_xor_sync(0xffffffffu, x, 2);
    x += __shfl_xor_sync(0xffffffffu, x, 1);
    return x;
}

// MODE 0: energy (unordered pairs), MODE 1: potential (A, U per point).
//
// Per work item the warp holds an i tile (lane = i point).  For each j tile it
// lists the images whose shifted i box comes within the cutoff of the j box, then
// each lane marks, for its own j point, which of those images bring the i box
// within the cutoff of that point.  The pair loop runs over j points (broadcast)
// and, inside, over the marked images: the delta part of a pair is computed once
// for all its images.  FP32 takes the j points with images two at a time, half x
// of every packed step on the images of the first and half y on those of the
// second, and reduces the four j-side sums of the potential over the warp once
// per such pair (warp_sum4); FP64 takes them one at a time.
template <typename R, int MODE, int NT, bool SKEW>
__global__ void __launch_bounds__(NT, 1) k_pair(const __grid_constant__ PairLaunch pl) {
    constexpr bool POT = (MODE == 1);
    constexpr int NW = NT / 32;
    using P = typename PT<R>::P;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ unsigned int s_prefix[kMaxInst + 1];
    __shared__ int s_C[kMaxInst];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    P *sp = reinterpret_cast<P *>(smem_raw) + warp * kTile;             // j tile
    P *simg = reinterpret_cast<P *>(smem_raw) + (NW + warp) * kTile;    // image shifts
    R *sn = reinterpret_cast<R *>(smem_raw + 2 * sizeof(P) * kTile * NW) + warp * kTile;

    const PairShared &sh = pl.sh;
    Table<R> tb;
    make_table<R>(sh, tb);
    Consts<R> K;
    make_consts<R>(sh, K);
    if constexpr (sizeof(R) == 4) {
        float *band = reinterpret_cast<float *>(smem_raw + (2 * sizeof(P) + sizeof(R)) * kTile * NW);
        tb.s = static_cast<uint32_t>(__cvta_generic_to_shared(band));
        tb.k0 = sh.ks0 >= 0 ? sh.ks0 : pl.inst[0].stats->band_row0;
        tb.kn = sh.ksn;
        const int S = sh.S, SB = tb.SB;
        const float *src = sh.tab32 + static_cast<size_t>(tb.k0) * S;
        for (int row = warp; row < sh.ksn; row += NW)
            for (int col = lane; col < S; col += 32) band[row * SB + col] = __ldg(src + row * S + col);
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
    // cell coordinates tD with all four rows of the cell in the resident band
    const float band_lo = static_cast<float>(tb.k0);
    const float band_hi = static_cast<float>(min(tb.k0 + tb.kn - 3, sh.nD - 1));
    __syncthreads();  // the only block barrier: table band and item counts ready
    // autotuning samples every item_stride-th item (item * stride < the total)
    const unsigned int stride = max(1u, sh.item_stride);
    const unsigned int n_items = min((s_prefix[pl.ninst] + stride - 1u) / stride, sh.item_limit);


    for (unsigned int iter = 0;; ++iter) {
        if (iter >= sh.max_iters) {
            if (lane == 0) atomicAdd(&pl.inst[0].stats->guard_trips, 1u);
            break;
        }
        unsigned int item = 0;
        if (lane == 0) item = atomicAdd(sh.queue, 1u);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= n_items) break;
        item *= stride;
        int k = 0;
        while (k + 1 < pl.ninst && item >= s_prefix[k + 1]) ++k;
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

        R h2[3], g2x[3];
        float h2f[3], g2f[3], rcm[3];
        int dims[3], M[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            h2[a] = static_cast<R>(pp.h2[a]);
            g2x[a] = static_cast<R>(pp.g2x[a]);
            h2f[a] = static_cast<float>(pp.h2[a]);
            g2f[a] = static_cast<float>(pp.g2x[a]);
            dims[a] = pp.dims[a];
            M[a] = pp.M[a];
            // cutoff in index units along a, widened so that rounding never drops an image
            rcm[a] = pp.rcm[a];
        }
        // culling metric: h2 on orthogonal cells, a lower bound of r^2/|d|^2 on skewed ones
        const float cull[3] = {pp.cull_h2[0], pp.cull_h2[1], pp.cull_h2[2]};
        (void)h2f;
        Cut cut;
        cut.pp = &pp;
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
        float4 cil = make_float4(0.f, 0.f, 0.f, 0.f), cih = cil;  // skewed: Cartesian i box
        if (SKEW) {
            cil = __ldg(pp.clo + I);
            cih = __ldg(pp.chi + I);
        }
        double A64 = 0.0, U64 = 0.0;
        unsigned int cnt = 0, nclamp = 0;
        unsigned int item_evals = 0;  // (j point, image) steps of this item (times ni_act at the end)
        for (int J = J0; J < J1; ++J) {
            const int jb = J * kTile;
            const int jn = min(kTile, n_act - jb);
            const float4 jlo = __ldg(pp.blo + J), jhi = __ldg(pp.bhi + J);
            const float jl[3] = {jlo.x, jlo.y, jlo.z}, jh[3] = {jhi.x, jhi.y, jhi.z};
            int mlo[3], nm[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (M[a] == 0) {
                    mlo[a] = 0;
                    nm[a] = 1;
                } else {
                    const float N = static_cast<float>(dims[a]);
                    mlo[a] = max(-M[a], static_cast<int>(ceilf((-rcm[a] - (ihi[a] - jl[a])) / N)));
                    const int mhi = min(M[a], static_cast<int>(floorf((rcm[a] - (ilo[a] - jh[a])) / N)));
                    nm[a] = max(0, mhi - mlo[a] + 1);
                }
            }
            const int n_cand = nm[0] * nm[1] * nm[2];
            float4 cjl = make_float4(0.f, 0.f, 0.f, 0.f), cjh = cjl;  // skewed: Cartesian j box
            if (SKEW) {
                cjl = __ldg(pp.clo + J);
                cjh = __ldg(pp.chi + J);
            }
            const bool diag = (J == I);
            bool staged = false;
            // candidate images in chunks of 32, one per lane
            for (int c0 = 0; c0 < n_cand; c0 += 32) {
                const int t = c0 + lane;
                bool ok = false;
                int mm[3] = {0, 0, 0};
                if (t < n_cand) {
                    mm[2] = mlo[2] + t % nm[2];
                    const int t1 = t / nm[2];
                    mm[1] = mlo[1] + t1 % nm[1];
                    mm[0] = mlo[0] + t1 / nm[1];
                    if (SKEW)
                        ok = !use_cut || box_gap2_cart(cil, cih, cjl, cjh, mm, dims, pp.vrow) <= rc2_box;
                    else
                        ok = !use_cut || box_gap2(ilo, ihi, jl, jh, mm, dims, cull) <= rc2_box;
                }
                const unsigned bal = __ballot_sync(0xffffffffu, ok);
                if (bal == 0u) continue;
                __syncwarp();  // earlier reads of simg, sp, sn are done
                if (ok) {
                    P sft;
                    sft.x = static_cast<R>(mm[0] * dims[0]);
                    sft.y = static_cast<R>(mm[1] * dims[1]);
                    sft.z = static_cast<R>(mm[2] * dims[2]);
                    sft.w = R(0);
                    simg[__popc(bal & ((1u << lane) - 1u))] = sft;
                }
                if (!staged) {
                    if (lane < jn) {
                        sp[lane] = PT<R>::load(pts, jb + lane);
                        sn[lane] = __ldg(nsrc + jb + lane);
                    }
                    staged = true;
                }
                __syncwarp();
                const int nimg = __popc(bal);
                // this lane's j point: images that bring the i box within the cutoff
                unsigned jm = 0u;
                if (lane < jn) {
                    const P pjl = sp[lane];
                    const float px = static_cast<float>(pjl.x), py = static_cast<float>(pjl.y),
                                pz = static_cast<float>(pjl.z);
                    for (int b = 0; b < nimg; ++b) {
                        const P sft = simg[b];
                        const float sx = static_cast<float>(sft.x), sy = static_cast<float>(sft.y),
                                    sz = static_cast<float>(sft.z);
                        float d2;
                        if (SKEW) {
                            // the point less the shift, in Cartesian coordinates, against the i box
                            const float ux = px - sx, uy = py - sy, uz = pz - sz;
                            const CellRows &vr = pp.vrow;
                            const float q0c = ux * vr.v[0] + uy * vr.v[3] + uz * vr.v[6];
                            const float q1c = ux * vr.v[1] + uy * vr.v[4] + uz * vr.v[7];
                            const float q2c = ux * vr.v[2] + uy * vr.v[5] + uz * vr.v[8];
                            const float gx = fmaxf(0.0f, fmaxf(cil.x - q0c, q0c - cih.x));
                            const float gy = fmaxf(0.0f, fmaxf(cil.y - q1c, q1c - cih.y));
                            const float gz = fmaxf(0.0f, fmaxf(cil.z - q2c, q2c - cih.z));
                            d2 = gx * gx + gy * gy + gz * gz;
                        } else {
                            const float gx = fmaxf(0.0f, fmaxf(ilo[0] + sx - px, px - ihi[0] - sx));
                            const float gy = fmaxf(0.0f, fmaxf(ilo[1] + sy - py, py - ihi[1] - sy));
                            const float gz = fmaxf(0.0f, fmaxf(ilo[2] + sz - pz, pz - ihi[2] - sz));
                            d2 = cull[0] * gx * gx + cull[1] * gy * gy + cull[2] * gz * gz;
                        }
                        if (!use_cut || d2 <= rc2_box) jm |= 1u << b;
                    }
                }
                R a_acc = 0, u_acc = 0;  // i side (this lane's i)
                R ja = 0, ju = 0;        // j side: lane L collects j = jb + L
                if constexpr (sizeof(R) == 4) {
                    // two j points per pass (packed halves), in order of their lanes
                    unsigned jset = __ballot_sync(0xffffffffu, jm != 0u);
                    while (jset != 0u) {
                        const int j0 = __ffs(jset) - 1;
                        jset &= jset - 1u;
                        const bool has1 = jset != 0u;
                        const int j1 = has1 ? __ffs(jset) - 1 : j0;
                        jset &= jset - 1u;
                        const unsigned m0 = __shfl_sync(0xffffffffu, jm, j0);
                        const unsigned m1s = __shfl_sync(0xffffffffu, jm, j1);
                        const unsigned m1 = has1 ? m1s : 0u;
                        item_evals += static_cast<unsigned>(__popc(m0) + __popc(m1));
                        const float4 p0 = sp[j0], p1 = sp[j1];
                        // weights: off-diagonal tiles count every pair for i and for j; in
                        // the diagonal tile j > i counts for both, j == i (self and
                        // self-images) for i only
                        const bool both0 = !diag || j0 > lane, both1 = !diag || j1 > lane;
                        const bool ok0 = act && (both0 || j0 == lane);
                        const bool ok1 = has1 && act && (both1 || j1 == lane);
                        Delta2 dp;
                        bool cl0, cl1;
                        const float2 qj = make_float2(p0.w, p1.w);
                        delta_part2<POT>(qi, qj, K, dp, cl0, cl1);
                        float2 A2, U2, V2;
                        unsigned ins0 = 0, ins1 = 0;
                        images2_f32<POT, SKEW>(m0, m1, simg, make_float2(xi - p0.x, xi - p1.x),
                                               make_float2(yi - p0.y, yi - p1.y), make_float2(zi - p0.z, zi - p1.z),
                                               qi, inv_qi, qi2, qj, h2, g2f, ok0, ok1, use_cut, cut, dp, K, tb,
                                               band_lo, band_hi, A2, U2, V2, ins0, ins1);
                        const unsigned wt0 = both0 ? 2u : 1u, wt1 = both1 ? 2u : 1u;  // ordered pairs
                        cnt += ins0 * wt0 + ins1 * wt1;
                        nclamp += (cl0 ? ins0 * wt0 : 0u) + (cl1 ? ins1 * wt1 : 0u);
                        const float n0 = sn[j0], n1 = sn[j1];
                        if (POT) {
                            a_acc += n0 * A2.x + n1 * A2.y;
                            u_acc += n0 * U2.x + n1 * U2.y;
                            const float cA0 = both0 ? ni * A2.x : 0.0f, cU0 = both0 ? ni * V2.x : 0.0f;
                            const float cA1 = both1 ? ni * A2.y : 0.0f, cU1 = both1 ? ni * V2.y : 0.0f;
                            if (__any_sync(0xffffffffu, cA0 != 0.0f || cU0 != 0.0f || cA1 != 0.0f || cU1 != 0.0f)) {
                                const float tot = warp_sum4(cA0, cU0, cA1, cU1);
                                const bool second = has1 && lane == j1;
                                const float gA = __shfl_sync(0xffffffffu, tot, second ? 16 : 0);
                                const float gU = __shfl_sync(0xffffffffu, tot, second ? 24 : 8);
                                if (lane == j0 || second) {
                                    ja += gA;
                                    ju += gU;
                                }
                            }
                        } else {
                            a_acc += static_cast<float>(wt0) * n0 * A2.x + static_cast<float>(wt1) * n1 * A2.y;
                        }
                    }
                } else {
                    for (int jj = 0; jj < jn; ++jj) {
                        unsigned m = __shfl_sync(0xffffffffu, jm, jj);
                        if (m == 0u) continue;
                        item_evals += static_cast<unsigned>(__popc(m));
                        const P pj = sp[jj];
                        const R nj = sn[jj];
                        const bool both = !diag || jj > lane;
                        const bool lane_ok = act && (both || jj == lane);
                        Delta<R> dp;
                        delta_part<POT, R>(qi, pj.w, K, dp);
                        R sA = 0, sU = 0, cA = 0, cU = 0;
                        unsigned ins = 0, hits = 0;
                        do {
                            const int b = __ffs(m) - 1;
                            m &= m - 1u;
                            const P sft = simg[b];
                            const R dx = (xi + sft.x) - pj.x, dy = (yi + sft.y) - pj.y, dz = (zi + sft.z) - pj.z;
                            R r2 = h2[0] * (dx * dx) + h2[1] * (dy * dy) + h2[2] * (dz * dz);
                            if (SKEW) r2 += g2x[0] * (dx * dy) + g2x[1] * (dx * dz) + g2x[2] * (dy * dz);
                            if (lane_ok && !(use_cut && beyond<SKEW>(r2, dx, dy, dz, cut))) {
                                R phi, rd = 0, rd2 = 0;
                                dist_part<POT, R>(r2, qi, pj.w, inv_qi, qi2, dp, K, tb, phi, rd, rd2);
                                sA += phi;
                                if (POT) {
                                    sU += rd;
                                    cA += phi;
                                    cU += rd2;
                                }
                                ins += 1u;
                                hits += (r2 > R(0)) ? 1u : 0u;
                            }
                        } while (m != 0u);
                        const unsigned wt = both ? 2u : 1u;  // ordered pairs represented
                        cnt += hits * wt;
                        nclamp += dp.cl ? ins * wt : 0u;
                        if (POT) {
                            a_acc += nj * sA;
                            u_acc += nj * sU;
                        } else {
                            a_acc += static_cast<R>(wt) * nj * sA;
                        }
                        if (POT) {
                            cA = both ? ni * cA : R(0);
                            cU = both ? ni * cU : R(0);
                            if (__any_sync(0xffffffffu, cA != R(0) || cU != R(0))) {
                                cA = warp_sum(cA);
                                cU = warp_sum(cU);
                                if (lane == jj) {
                                    ja += cA;
                                    ju += cU;
                                }
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
        }
        // FP32 counts every inside evaluation; the self term (j = i, L = 0, the one
        // evaluation at r = 0) sits in the diagonal tile, which chunk 0 holds
        if (sizeof(R) == 4 && c == 0 && act) cnt -= 1u;
        if (act && POT) {
            if (A64 != 0.0) atomicAdd(pp.A + ig, A64);
            if (U64 != 0.0) atomicAdd(pp.U + ig, static_cast<double>(ni) * U64);
        }
        count_item(pp.stats, act ? cnt : 0u, act ? nclamp : 0u, item_evals * static_cast<unsigned>(ni_act));
        if (!POT) {
            // the item's energy partial, summed over lanes in a fixed order (items
            // beyond the partials' capacity are added atomically)
            const double e = warp_sum(act ? static_cast<double>(ni) * A64 : 0.0);
            if (lane == 0) {
                if (sh.item_E && item < sh.item_cap)
                    sh.item_E[item] = e;
                else if (e != 0.0)
                    atomicAdd(&pp.stats->E_pair, e);
            }
        }
    }
}

// The splitmix64 output function (Steele, Lea and Flood, "Fast splittable
// pseudorandom number generators", 2014): a counter-based stream for sampling.
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

constexpr int kBandSamples = 8;  // samples per thread of k_band_hist

// Sampled histogram of the table's D cell over the evaluations of one problem:
// uniform (i, j, image) triples (image index uniform in [-M_a, M_a] per periodic
// axis), kept where r <= r_cut, binned by the stencil's first row floor(tD);
// evaluations past the table (tD > nD - 1) read no row and are not counted.
// The counts depend only on the sample indices: the result is reproducible.
__global__ void k_band_hist(const __grid_constant__ PairShared sh, const __grid_constant__ PairParams pp,
                            unsigned int *__restrict__ hist, unsigned int salt) {
    __shared__ unsigned int h[kBandBins];
    for (int b = threadIdx.x; b < kBandBins; b += blockDim.x) h[b] = 0u;
    __syncthreads();
    const int na = pp.stats->n_active;
    const int kmax = sh.nD - 2;
    if (na > 0 && kmax < kBandBins) {
        const float h0 = static_cast<float>(pp.h2[0]), h1 = static_cast<float>(pp.h2[1]),
                    h2 = static_cast<float>(pp.h2[2]);
        const float g0 = static_cast<float>(pp.g2x[0]), g1 = static_cast<float>(pp.g2x[1]),
                    g2 = static_cast<float>(pp.g2x[2]);
        const float rc2 = static_cast<float>(pp.rc2), cD = static_cast<float>(sh.cD),
                    tmax = static_cast<float>(sh.nD - 1);
        const unsigned long long t0 =
            (static_cast<unsigned long long>(blockIdx.x) * blockDim.x + threadIdx.x) * kBandSamples;
        for (int s = 0; s < kBandSamples; ++s) {
            const unsigned long long x = mix64((static_cast<unsigned long long>(salt) << 40) + t0 + s);
            const unsigned long long y = mix64(x ^ 0x9e3779b97f4a7c15ull);
            const int i = static_cast<int>((x & 0xffffffffull) % static_cast<unsigned>(na));
            const int j = static_cast<int>((x >> 32) % static_cast<unsigned>(na));
            int m[3];
#pragma unroll
            for (int a = 0; a < 3; ++a)
                m[a] = pp.M[a] > 0 ? static_cast<int>((y >> (21 * a)) % (2u * pp.M[a] + 1u)) - pp.M[a] : 0;
            const float4 pi = __ldg(pp.p32 + i), pj = __ldg(pp.p32 + j);
            const float dx = (pi.x - pj.x) + static_cast<float>(m[0] * pp.dims[0]);
            const float dy = (pi.y - pj.y) + static_cast<float>(m[1] * pp.dims[1]);
            const float dz = (pi.z - pj.z) + static_cast<float>(m[2] * pp.dims[2]);
            const float r2 = h0 * dx * dx + h1 * dy * dy + h2 * dz * dz + g0 * dx * dy + g1 * dx * dz + g2 * dy * dz;
            if (pp.use_cut && r2 > rc2) continue;
            const float t = sqrtf(fmaxf(r2, 0.0f)) * (pi.w + pj.w) * cD;
            if (!(t <= tmax)) continue;
            atomicAdd(&h[min(static_cast<int>(t), kmax)], 1u);
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < kBandBins; b += blockDim.x)
        if (h[b]) atomicAdd(hist + b, h[b]);
}

// The band start r0 in [0, nD + 2 - ksn] whose stencils [r0, r0 + ksn - 4] hold the
// most sampled evaluations; among starts within 0.2 % of the total of the best,
// the last (evaluations that miss the band then have small D, where a warp's lanes
// tend to miss together).  The block stages the histogram in shared memory; one
// thread then slides the window over at most kBandBins rows.
__global__ void k_band_choose(const __grid_constant__ PairShared sh, const unsigned int *__restrict__ hist,
                              Stats *out) {
    __shared__ unsigned int h[kBandBins];
    for (int b = threadIdx.x; b < kBandBins; b += blockDim.x) h[b] = hist[b];
    __syncthreads();
    if (threadIdx.x != 0) return;
    const int nk = sh.nD - 1;              // stencil starts 0 .. nD - 2
    const int span = sh.ksn - 3;           // stencil starts a band of ksn rows holds
    const int r0max = sh.nD + 2 - sh.ksn;  // last start that keeps the band in the table
    int choice = 0;
    if (nk <= kBandBins && span > 0 && r0max > 0) {
        unsigned long long total = 0, cov = 0;
        for (int k = 0; k < nk; ++k) total += h[k];
        for (int k = 0; k < min(span, nk); ++k) cov += h[k];
        unsigned long long best = cov, c = cov;
        for (int r0 = 1; r0 <= r0max; ++r0) {
            c -= h[r0 - 1];
            if (r0 + span - 1 < nk) c += h[r0 + span - 1];
            best = c > best ? c : best;
        }
        const unsigned long long tol = total / 500;
        c = cov;
        for (int r0 = 0; r0 <= r0max; ++r0) {
            if (r0 > 0) {
                c -= h[r0 - 1];
                if (r0 + span - 1 < nk) c += h[r0 + span - 1];
            }
            if (c + tol >= best) choice = r0;
        }
    }
    out->band_row0 = choice;
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

// Voxel-averaged kernel at delta = 0 (the diagonal "phi0" step):
//   phi0(q) = int_{[-1,1]^3} prod_a (1 - |t_a|) phi_0(q |sum_a t_a v_a|) d^3t,
// phi_0(D) the kernel at delta = 0 for D >= D_1 and -(2/pi) ln D + psi0 + c2 D^2
// below (the divergence of eq. 14 at D -> 0 that the table's row 0 softens).
// Block (q, octant): one of the eight sign octants of t times a tensor rule of
// nn nodes (x, w on [0, 1]) per axis.  The integrand is evaluated in FP32 (the
// FP32 table path, errors ~1e-7 relative per term, far below the rule's
// ~1e-5) and summed in FP64; the octant sums are added in a fixed order.
__global__ void k_phi0(const PairShared sh, Phi0Rule rule, const double *__restrict__ q,
                       const double *__restrict__ xw, double *__restrict__ part) {
    Table<float> tb;
    make_table<float>(sh, tb);
    Consts<float> K;
    make_consts<float>(sh, K);
    const int nn = rule.nn;
    const float qq = static_cast<float>(q[blockIdx.x]);
    const int sg = blockIdx.y;
    const float s0 = (sg & 1) ? -1.0f : 1.0f, s1 = (sg & 2) ? -1.0f : 1.0f, s2 = (sg & 4) ? -1.0f : 1.0f;
    float v[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) v[k] = static_cast<float>(rule.v[k]);
    const float D1 = static_cast<float>(rule.D1), psi0 = static_cast<float>(rule.psi0),
                c2 = static_cast<float>(rule.c2);
    const int total = nn * nn * nn;
    double acc = 0.0;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int i = e / (nn * nn), j = (e / nn) % nn, k = e % nn;
        const float t0 = s0 * static_cast<float>(xw[i]), t1 = s1 * static_cast<float>(xw[j]),
                    t2 = s2 * static_cast<float>(xw[k]);
        const float r0 = t0 * v[0] + t1 * v[3] + t2 * v[6];
        const float r1 = t0 * v[1] + t1 * v[4] + t2 * v[7];
        const float r2 = t0 * v[2] + t1 * v[5] + t2 * v[8];
        const float D = qq * sqrtf(r0 * r0 + r1 * r1 + r2 * r2);
        float phi;
        if (D < D1) {
            phi = -0.63661977236758134f * logf(D) + psi0 + c2 * D * D;
        } else {
            float rd = 0.0f, rd2 = 0.0f;
            unsigned ncl = 0;
            pair_phi<false, float>(D * D, 1.0f, 1.0f, 1.0f, 1.0f, K, tb, phi, rd, rd2, ncl);
        }
        const double wt = xw[nn + i] * xw[nn + j] * xw[nn + k] * (1.0 - xw[i]) * (1.0 - xw[j]) * (1.0 - xw[k]);
        acc += wt * static_cast<double>(phi);
    }
    __shared__ double red[256];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (static_cast<int>(threadIdx.x) < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x * 8 + blockIdx.y] = red[0];
}

__global__ void k_phi0_sum(const double *__restrict__ part, int nq, double *__restrict__ out) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nq; t += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int o = 0; o < 8; ++o) s += part[t * 8 + o];
        out[t] = s;
    }
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

template <typename R, int MODE, int NT, bool SKEW>
int launch_one(const PairLaunch &pl, int nctas, size_t smem, cudaStream_t st) {
    auto kern = k_pair<R, MODE, NT, SKEW>;
    VDWDF_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        static_cast<int>(smem)));
    kern<<<nctas, NT, smem, st>>>(pl);
    count_launches(1);
    VDWDF_CUDA_TRY(cudaGetLastError());
    return VDWDF_OK;
}

// Skewed cells run the 512-thread kernel only (the launch configuration is
// chosen for 512 threads when any instance is skewed).
template <typename R, int MODE>
int launch_nt(int threads, bool skew, const PairLaunch &pl, int nctas, size_t smem, cudaStream_t st) {
    if (skew) {
        if (threads == 448) return launch_one<R, MODE, 448, true>(pl, nctas, smem, st);
        return threads == 384 ? launch_one<R, MODE, 384, true>(pl, nctas, smem, st)
                              : launch_one<R, MODE, 512, true>(pl, nctas, smem, st);
    }
    switch (threads) {
        case 256: return launch_one<R, MODE, 256, false>(pl, nctas, smem, st);
        case 384: return launch_one<R, MODE, 384, false>(pl, nctas, smem, st);
        case 448: return launch_one<R, MODE, 448, false>(pl, nctas, smem, st);
        case 1024: return launch_one<R, MODE, 1024, false>(pl, nctas, smem, st);
        default: return launch_one<R, MODE, 512, false>(pl, nctas, smem, st);
    }
}

}  // namespace

int pair_smem_bytes(int precision, int threads, int ksn, int S) {
    // per warp: j tile (points, densities) and image shifts; FP32: the table band
    const size_t pt = precision == VDWDF_FP64 ? 2 * sizeof(dvec4) + sizeof(double)
                                              : 2 * sizeof(float4) + sizeof(float);
    size_t b = pt * kTile * static_cast<size_t>(threads / 32);
    if (precision != VDWDF_FP64) b += static_cast<size_t>(ksn) * band_stride(S) * sizeof(float);
    return static_cast<int>(b);
}

int launch_pair(int precision, bool potential, bool skew, int threads, const PairLaunch &pl, int nctas,
                cudaStream_t st) {
    if (skew && threads != 512 && threads != 448 && threads != 384) return VDWDF_EINVAL;  // skewed: 384, 448, 512
    const size_t smem = static_cast<size_t>(pair_smem_bytes(precision, threads, pl.sh.ksn, pl.sh.S));
    if (precision == VDWDF_FP64)
        return potential ? launch_nt<double, 1>(threads, skew, pl, nctas, smem, st)
                         : launch_nt<double, 0>(threads, skew, pl, nctas, smem, st);
    return potential ? launch_nt<float, 1>(threads, skew, pl, nctas, smem, st)
                     : launch_nt<float, 0>(threads, skew, pl, nctas, smem, st);
}

int launch_band_choose(const PairLaunch &pl, unsigned int *hist, cudaStream_t st) {
    VDWDF_CUDA_TRY(cudaMemsetAsync(hist, 0, sizeof(unsigned int) * kBandBins, st));
    int dev = 0, sms = 0;
    VDWDF_CUDA_TRY(cudaGetDevice(&dev));
    VDWDF_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    for (int k = 0; k < pl.ninst; ++k)
        k_band_hist<<<2 * (sms > 0 ? sms : 1), 256, 0, st>>>(pl.sh, pl.inst[k], hist, static_cast<unsigned>(k));
    k_band_choose<<<1, 256, 0, st>>>(pl.sh, hist, pl.inst[0].stats);
    count_launches(pl.ninst + 1);
    VDWDF_CUDA_TRY(cudaGetLastError());
    return VDWDF_OK;
}

int launch_reduce_items(const PairLaunch &pl, cudaStream_t st) {
    if (!pl.sh.item_E) return VDWDF_OK;
    k_reduce_items<<<pl.ninst, 256, 0, st>>>(pl);
    count_launches(1);
    VDWDF_CUDA_TRY(cudaGetLastError());
    return VDWDF_OK;
}

int launch_phi0(const PairShared &sh, const Phi0Rule &rule, int nq, const double *q, const double *xw,
                double *part, double *out, cudaStream_t st) {
    if (nq <= 0) return VDWDF_OK;
    k_phi0<<<dim3(nq, 8), 256, 0, st>>>(sh, rule, q, xw, part);
    k_phi0_sum<<<(nq + 255) / 256, 256, 0, st>>>(part, nq, out);
    count_launches(2);
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
