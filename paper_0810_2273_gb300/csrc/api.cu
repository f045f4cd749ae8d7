// extern "C" entry points of libvdwdf (declared in include/vdwdf.h).
//
// A call validates its arguments on the host, takes scratch with
// cudaMallocAsync on the caller's stream, runs
//   gradient + q0  ->  trimming into brick order  ->  tile boxes  ->  pair kernel
//   (-> potential assembly)  ->  reductions,
// reads the counters back and frees the scratch on the same stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "table.h"

struct vdwdf_table {
    int nD, nd;
    double Dmax;
    unsigned long long gen = 0;  // unique per table of this process (graph-cache keys)
    std::vector<double> nodes;   // nD * nd, D outer
    std::vector<double> coef64;  // (nD + 2) * (nd + 2), / 36
    std::vector<float> coef32;
    std::mutex mu;
    std::map<int, std::pair<double *, float *>> dev;  // device id -> copies
};

namespace vdwdf {

namespace {

std::atomic<long long> g_launches{0};
std::atomic<unsigned long long> g_table_gen{0};  // generation ids of tables

// Fault injection for tests, on the host only (no device fault is ever caused):
//   VDWDF_FAIL_ALLOC=1  every scratch allocation of a call fails (VDWDF_EALLOC);
//   VDWDF_MAX_ITERS=k   the persistent pair kernels stop after k work items per
//                       CTA, as their iteration guard would, so the call returns
//                       VDWDF_ETIMEOUT.
bool fail_alloc_requested() {
    const char *e = std::getenv("VDWDF_FAIL_ALLOC");
    return e && e[0] == '1';
}
unsigned int max_iters_override(unsigned int v) {
    const char *e = std::getenv("VDWDF_MAX_ITERS");
    if (!e || !e[0]) return v;
    const long long k = std::atoll(e);
    return (k > 0 && static_cast<unsigned long long>(k) < v) ? static_cast<unsigned int>(k) : v;
}
// cudaMallocAsync / cudaMalloc of a call's scratch, with the fault-injection hook
cudaError_t scratch_malloc_async(void **p, size_t bytes, cudaStream_t st) {
    if (fail_alloc_requested()) return cudaErrorMemoryAllocation;
    return cudaMallocAsync(p, bytes, st);
}
cudaError_t scratch_malloc(void **p, size_t bytes) {
    if (fail_alloc_requested()) return cudaErrorMemoryAllocation;
    return cudaMalloc(p, bytes);
}
constexpr double kPi = 3.14159265358979323846;
constexpr int kMaxImages = 64;

// Device layout of the coefficients: (nD + 2) x (nd + 2) bicubic coefficients / 36,
// then nd + 2 coefficients / 6 of the beyond-table normalisation rho(delta).
int finish_table(vdwdf_table *t) {
    t->gen = ++g_table_gen;
    const int S = t->nd + 2;
    const size_t main = static_cast<size_t>(t->nD + 2) * S;
    try {
        t->coef64.assign(main + S, 0.0);
        t->coef32.assign(main + S, 0.0f);
    } catch (const std::bad_alloc &) {
        return VDWDF_EALLOC;
    }
    spline_coefficients(t->nD, t->nd, t->nodes.data(), t->coef64.data());
    rho_coefficients(t->nD, t->Dmax, t->nd, t->nodes.data(), t->coef64.data() + main);
    for (size_t i = 0; i < t->coef64.size(); ++i) {
        t->coef64[i] /= (i < main) ? 36.0 : 6.0;
        t->coef32[i] = static_cast<float>(t->coef64[i]);
    }
    return VDWDF_OK;
}

int table_on_device(const vdwdf_table *tc, double **d64, float **d32) {
    vdwdf_table *t = const_cast<vdwdf_table *>(tc);
    int dev = 0;
    VDWDF_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(t->mu);
    auto it = t->dev.find(dev);
    if (it == t->dev.end()) {
        double *a = nullptr;
        float *b = nullptr;
        const size_t n = t->coef64.size();
        if (cudaMalloc(&a, n * sizeof(double)) != cudaSuccess) return VDWDF_EALLOC;
        if (cudaMalloc(&b, n * sizeof(float)) != cudaSuccess) {
            cudaFree(a);
            return VDWDF_EALLOC;
        }
        VDWDF_CUDA_TRY(cudaMemcpy(a, t->coef64.data(), n * sizeof(double), cudaMemcpyHostToDevice));
        VDWDF_CUDA_TRY(cudaMemcpy(b, t->coef32.data(), n * sizeof(float), cudaMemcpyHostToDevice));
        it = t->dev.emplace(dev, std::make_pair(a, b)).first;
    }
    *d64 = it->second.first;
    *d32 = it->second.second;
    return VDWDF_OK;
}

// Morton order of the 4x4x4 bricks of a grid, cached per (device, dims).
std::mutex g_brick_mu;
std::map<std::tuple<int, int, int, int>, std::pair<int *, int>> g_bricks;

uint64_t spread3(uint32_t v) {
    uint64_t x = v & 0x1fffff;
    x = (x | x << 32) & 0x1f00000000ffffULL;
    x = (x | x << 16) & 0x1f0000ff0000ffULL;
    x = (x | x << 8) & 0x100f00f00f00f00fULL;
    x = (x | x << 4) & 0x10c30c30c30c30c3ULL;
    x = (x | x << 2) & 0x1249249249249249ULL;
    return x;
}

int brick_order(const int dims[3], int **order, int *nb) {
    int dev = 0;
    VDWDF_CUDA_TRY(cudaGetDevice(&dev));
    const auto key = std::make_tuple(dev, dims[0], dims[1], dims[2]);
    std::lock_guard<std::mutex> lk(g_brick_mu);
    auto it = g_bricks.find(key);
    if (it == g_bricks.end()) {
        const int bx = (dims[0] + kBrick - 1) / kBrick, by = (dims[1] + kBrick - 1) / kBrick,
                  bz = (dims[2] + kBrick - 1) / kBrick;
        const int n = bx * by * bz;
        std::vector<std::pair<uint64_t, int>> keys(n);
        for (int x = 0; x < bx; ++x)
            for (int y = 0; y < by; ++y)
                for (int z = 0; z < bz; ++z) {
                    const int id = (x * by + y) * bz + z;
                    keys[id] = {spread3(x) << 2 | spread3(y) << 1 | spread3(z), id};
                }
        std::sort(keys.begin(), keys.end());
        std::vector<int> ord(n);
        for (int i = 0; i < n; ++i) ord[i] = keys[i].second;
        int *d = nullptr;
        if (cudaMalloc(&d, sizeof(int) * n) != cudaSuccess) return VDWDF_EALLOC;
        VDWDF_CUDA_TRY(cudaMemcpy(d, ord.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
        it = g_bricks.emplace(key, std::make_pair(d, n)).first;
    }
    *order = it->second.first;
    *nb = it->second.second;
    return VDWDF_OK;
}

int sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}

// ---------------------------------------------------------------------------
// argument checks and geometry
// ---------------------------------------------------------------------------
struct Geom {
    int dims[3];
    int per[3];
    double L[3], h[3];  // |M_a| and |M_a| / N_a
    double dV;
    long long N;
    int M[3];
    double rc;
    bool use_cut;
    double B[9];        // reciprocal rows: B_a . M_b = delta_ab
    double met[6];      // metric in index units: 00, 11, 22, 01, 02, 12
    double lmin;        // its smallest eigenvalue
    bool skew;          // non-diagonal metric
    AxisMap am;         // grid-axis derivatives to Cartesian gradient
    CellRows vrow;      // M_a / N_a (float), for Cartesian tile boxes
    bool spectral;      // gradient by the band-limited (FFT) derivative
};

// Smallest eigenvalue of the symmetric 3x3 matrix (a00, a11, a22, a01, a02, a12)
// (trigonometric solution of the characteristic cubic).
double sym3_min_eig(const double m[6]) {
    const double p1 = m[3] * m[3] + m[4] * m[4] + m[5] * m[5];
    if (p1 == 0.0) return std::min(m[0], std::min(m[1], m[2]));
    const double q = (m[0] + m[1] + m[2]) / 3.0;
    const double p2 = (m[0] - q) * (m[0] - q) + (m[1] - q) * (m[1] - q) + (m[2] - q) * (m[2] - q) + 2.0 * p1;
    const double p = std::sqrt(p2 / 6.0);
    const double b00 = (m[0] - q) / p, b11 = (m[1] - q) / p, b22 = (m[2] - q) / p;
    const double b01 = m[3] / p, b02 = m[4] / p, b12 = m[5] / p;
    const double detB = b00 * (b11 * b22 - b12 * b12) - b01 * (b01 * b22 - b12 * b02) + b02 * (b01 * b12 - b11 * b02);
    const double r = std::max(-1.0, std::min(1.0, detB / 2.0));
    const double phi = std::acos(r) / 3.0;
    return q + 2.0 * p * std::cos(phi + 2.0 * kPi / 3.0);
}

int check_grid(const vdwdf_grid *g, Geom &G) {
    if (!g) return VDWDF_EINVAL;
    long long N = 1;
    const double(*M)[3] = g->cell;
    for (int a = 0; a < 3; ++a) {
        if (g->n[a] < 1 || g->n[a] > (1 << 20)) return VDWDF_EINVAL;
        if (g->periodic[a] != 0 && g->periodic[a] != 1) return VDWDF_EINVAL;
        if (g->n[a] > 12800 && g->gradient == VDWDF_GRAD_SPECTRAL) return VDWDF_EUNSUPPORTED;
        N *= g->n[a];
        for (int b = 0; b < 3; ++b)
            if (!std::isfinite(M[a][b])) return VDWDF_EINVAL;
    }
    if (N > (1LL << 31) - 1) return VDWDF_EINVAL;
    if (g->gradient != VDWDF_GRAD_FD && g->gradient != VDWDF_GRAD_SPECTRAL) return VDWDF_EINVAL;
    G.spectral = g->gradient == VDWDF_GRAD_SPECTRAL;
    const double det = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
                       M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                       M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
    if (!(std::fabs(det) > 0.0) || !std::isfinite(det)) return VDWDF_EINVAL;
    bool diagonal = true;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            if (a != b && M[a][b] != 0.0) diagonal = false;
    if (diagonal)
        for (int a = 0; a < 3; ++a)
            if (!(M[a][a] > 0.0)) return VDWDF_EINVAL;
    for (int a = 0; a < 3; ++a) {
        G.dims[a] = g->n[a];
        G.per[a] = g->periodic[a];
        G.L[a] = diagonal ? M[a][a] : std::sqrt(M[a][0] * M[a][0] + M[a][1] * M[a][1] + M[a][2] * M[a][2]);
        G.h[a] = G.L[a] / g->n[a];
        // B_a = (M_b x M_c) / det, (a, b, c) cyclic
        const double *u = M[(a + 1) % 3], *v = M[(a + 2) % 3];
        G.B[3 * a + 0] = (u[1] * v[2] - u[2] * v[1]) / det;
        G.B[3 * a + 1] = (u[2] * v[0] - u[0] * v[2]) / det;
        G.B[3 * a + 2] = (u[0] * v[1] - u[1] * v[0]) / det;
    }
    G.N = N;
    G.dV = diagonal ? G.L[0] * G.L[1] * G.L[2] / static_cast<double>(N) : std::fabs(det) / static_cast<double>(N);
    auto dot = [&](int a, int b) { return M[a][0] * M[b][0] + M[a][1] * M[b][1] + M[a][2] * M[b][2]; };
    for (int a = 0; a < 3; ++a) G.met[a] = diagonal ? G.h[a] * G.h[a] : dot(a, a) / (double(G.dims[a]) * G.dims[a]);
    G.met[3] = diagonal ? 0.0 : dot(0, 1) / (double(G.dims[0]) * G.dims[1]);
    G.met[4] = diagonal ? 0.0 : dot(0, 2) / (double(G.dims[0]) * G.dims[2]);
    G.met[5] = diagonal ? 0.0 : dot(1, 2) / (double(G.dims[1]) * G.dims[2]);
    G.skew = G.met[3] != 0.0 || G.met[4] != 0.0 || G.met[5] != 0.0;
    G.lmin = sym3_min_eig(G.met);
    if (!(G.lmin > 0.0)) return VDWDF_EINVAL;
    for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) G.vrow.v[3 * a + c] = static_cast<float>(M[a][c] / G.dims[a]);
    G.am.general = diagonal ? 0 : 1;
    for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c)
            G.am.S[3 * a + c] = diagonal ? (a == c ? (1.0 / G.h[a]) / 12.0 : 0.0) : G.dims[a] * G.B[3 * a + c] / 12.0;
    return VDWDF_OK;
}

int check_cut(double n_cut, double r_cut, Geom &G) {
    if (!(n_cut > 0.0) || !std::isfinite(n_cut)) return VDWDF_EINVAL;
    if (std::isnan(r_cut) || std::isinf(r_cut)) return VDWDF_EINVAL;
    const bool any_per = G.per[0] || G.per[1] || G.per[2];
    if (any_per && !(r_cut > 0.0)) return VDWDF_EINVAL;
    G.use_cut = r_cut > 0.0;
    G.rc = G.use_cut ? r_cut : 0.0;
    for (int a = 0; a < 3; ++a) {
        // every image L with |r_i - r_j + L| <= r_cut has |m_a| <= r_cut |B_a| + 1
        const double bl = std::sqrt(G.B[3 * a] * G.B[3 * a] + G.B[3 * a + 1] * G.B[3 * a + 1] +
                                    G.B[3 * a + 2] * G.B[3 * a + 2]);
        const double ext = G.skew ? r_cut * bl : r_cut / G.L[a];
        G.M[a] = G.per[a] ? static_cast<int>(std::ceil(ext)) + 1 : 0;
        if (G.M[a] > kMaxImages) return VDWDF_EINVAL;
    }
    return VDWDF_OK;
}

// ---------------------------------------------------------------------------
// scratch
// ---------------------------------------------------------------------------
struct Carve {
    size_t off = 0;
    template <typename T>
    size_t take(size_t count) {
        const size_t o = off;
        off += (count * sizeof(T) + 255) & ~static_cast<size_t>(255);
        return o;
    }
};

struct Work {
    unsigned char *base = nullptr;
    double *q0 = nullptr, *qn = nullptr, *qg = nullptr;
    int *cnt = nullptr, *off = nullptr, *slot = nullptr;
    float4 *p32 = nullptr;
    float *n32 = nullptr;
    dvec4 *p64 = nullptr;
    double *n64 = nullptr;
    float4 *blo = nullptr, *bhi = nullptr;
    float4 *clo = nullptr, *chi = nullptr;  // skewed cells only
    double *A = nullptr, *U = nullptr;
    Stats *stats = nullptr;
    unsigned int *queue = nullptr;
    unsigned int *hist = nullptr;  // kBandBins counters: the band-start histogram
    double *gsp = nullptr, *coef = nullptr, *div = nullptr;  // spectral gradient only
};

size_t layout(const Geom &G, int nb, bool pot, bool fp64, Work *w, unsigned char *base) {
    Carve c;
    const size_t N = static_cast<size_t>(G.N);
    const size_t tiles = (N + kTile - 1) / kTile;
    const size_t o_q0 = c.take<double>(N);
    const size_t o_qn = pot ? c.take<double>(N) : 0;
    const size_t o_qg = pot ? c.take<double>(3 * N) : 0;
    const size_t o_cnt = c.take<int>(nb);
    const size_t o_off = c.take<int>(nb + 1);
    const size_t o_slot = c.take<int>(N);
    const size_t o_p32 = c.take<float4>(N);
    const size_t o_n32 = c.take<float>(N);
    const size_t o_p64 = fp64 ? c.take<dvec4>(N) : 0;
    const size_t o_n64 = c.take<double>(N);
    const size_t o_blo = c.take<float4>(tiles);
    const size_t o_bhi = c.take<float4>(tiles);
    const size_t o_clo = G.skew ? c.take<float4>(tiles) : 0;
    const size_t o_chi = G.skew ? c.take<float4>(tiles) : 0;
    const size_t o_A = pot ? c.take<double>(N) : 0;
    const size_t o_U = pot ? c.take<double>(N) : 0;
    const size_t o_st = c.take<Stats>(1);
    const size_t o_q = c.take<unsigned int>(1);
    const size_t o_h = c.take<unsigned int>(kBandBins);
    const size_t o_gsp = G.spectral ? c.take<double>(3 * N) : 0;
    const size_t o_coef = G.spectral ? c.take<double>(G.dims[0] + G.dims[1] + G.dims[2]) : 0;
    const size_t o_div = (G.spectral && pot) ? c.take<double>(N) : 0;
    if (w && base) {
        w->base = base;
        w->q0 = reinterpret_cast<double *>(base + o_q0);
        w->qn = pot ? reinterpret_cast<double *>(base + o_qn) : nullptr;
        w->qg = pot ? reinterpret_cast<double *>(base + o_qg) : nullptr;
        w->cnt = reinterpret_cast<int *>(base + o_cnt);
        w->off = reinterpret_cast<int *>(base + o_off);
        w->slot = reinterpret_cast<int *>(base + o_slot);
        w->p32 = reinterpret_cast<float4 *>(base + o_p32);
        w->n32 = reinterpret_cast<float *>(base + o_n32);
        w->p64 = fp64 ? reinterpret_cast<dvec4 *>(base + o_p64) : nullptr;
        w->n64 = reinterpret_cast<double *>(base + o_n64);
        w->blo = reinterpret_cast<float4 *>(base + o_blo);
        w->bhi = reinterpret_cast<float4 *>(base + o_bhi);
        w->clo = G.skew ? reinterpret_cast<float4 *>(base + o_clo) : nullptr;
        w->chi = G.skew ? reinterpret_cast<float4 *>(base + o_chi) : nullptr;
        w->A = pot ? reinterpret_cast<double *>(base + o_A) : nullptr;
        w->U = pot ? reinterpret_cast<double *>(base + o_U) : nullptr;
        w->stats = reinterpret_cast<Stats *>(base + o_st);
        w->queue = reinterpret_cast<unsigned int *>(base + o_q);
        w->hist = reinterpret_cast<unsigned int *>(base + o_h);
        w->gsp = G.spectral ? reinterpret_cast<double *>(base + o_gsp) : nullptr;
        w->coef = G.spectral ? reinterpret_cast<double *>(base + o_coef) : nullptr;
        w->div = (G.spectral && pot) ? reinterpret_cast<double *>(base + o_div) : nullptr;
    }
    return c.off;
}

// Zero the counters; q0 minimum starts above every float.
int reset_stats(Stats *s, cudaStream_t st) {
    VDWDF_CUDA_TRY(cudaMemsetAsync(s, 0, sizeof(Stats), st));
    VDWDF_CUDA_TRY(cudaMemsetAsync(&s->qmin_bits, 0xFF, sizeof(unsigned int), st));
    return VDWDF_OK;
}

Recip recip_of(const Geom &G) {
    Recip R;
    for (int k = 0; k < 9; ++k) R.B[k] = G.B[k];
    return R;
}

// The gradient the q0 step reads: the caller's; else, on a grid with the spectral
// option, the FFT gradient written to gsp (3 N) with coef (N0 + N1 + N2) as
// scratch; else none (the q0 kernel's own finite differences).
int q0_gradient(const Geom &G, const double *n_dev, const double *grad_dev, double *gsp, double *coef,
                const double **use, cudaStream_t st) {
    *use = grad_dev;
    if (grad_dev || !G.spectral) return VDWDF_OK;
    *use = gsp;
    return launch_gradient_spectral(G.dims, recip_of(G), n_dev, gsp, coef, st);
}

// v (and the A, U grids) from A, U at the active points, with the transpose of
// the grid's own gradient: the spectral one through W (3 N) and div (N), else
// the stencil inside the assembly kernel.
int assemble_v(const Geom &G, const int *slot, const double *A, const double *U, const double *qn,
               const double *qg, double *W, double *div, double *coef, double *v, double *A_grid, double *U_grid,
               cudaStream_t st) {
    const double *dp = nullptr;
    if (G.spectral) {
        const int rc = launch_div_spectral(G.dims, recip_of(G), slot, U, qg, W, div, coef, st);
        if (rc) return rc;
        dp = div;
    }
    return launch_assemble(G.dims, G.am, G.dV, slot, A, U, qn, qg, dp, v, A_grid, U_grid, st);
}

// gradient, q0, trimming and tiles of one problem into w
int prepare(const Geom &G, const double *n_dev, const double *grad_dev, double n_cut, bool pot,
            Work &w, cudaStream_t st) {
    int *order = nullptr, nb = 0;
    int rc = brick_order(G.dims, &order, &nb);
    if (rc) return rc;
    rc = reset_stats(w.stats, st);
    if (rc) return rc;
    const double *g_use = nullptr;
    rc = q0_gradient(G, n_dev, grad_dev, w.gsp, w.coef, &g_use, st);
    if (rc) return rc;
    rc = launch_grad_q0(G.dims, G.am, n_dev, g_use, w.q0, w.qn, w.qg, st);
    if (rc) return rc;
    rc = launch_compact(G.dims, n_dev, n_cut, w.q0, order, nb, w.cnt, w.off, pot ? w.slot : nullptr,
                        w.p32, w.n32, w.p64, w.n64, w.blo, w.bhi, w.stats, st);
    if (rc || !G.skew) return rc;
    return launch_tiles_cart(w.p32, w.stats, G.vrow, w.clo, w.chi, G.N, st);
}

void fill_params(const Geom &G, const Work &w, PairParams &pp) {
    pp.rc2 = G.rc * G.rc * (1.0 + 1e-12);  // inclusive cutoff, rounding ties inside
    for (int a = 0; a < 3; ++a) {
        pp.h2[a] = G.met[a];
        pp.g2x[a] = 2.0 * G.met[3 + a];
        pp.dims[a] = G.dims[a];
        pp.M[a] = G.M[a];
        // culling: exact per-axis metric on orthogonal cells, its smallest eigenvalue
        // (a lower bound of r^2 / |d|^2) on skewed ones; the cutoff's extent in index
        // units along a is r_cut sqrt(1/h2) or r_cut |B_a| N_a
        pp.cull_h2[a] = static_cast<float>(G.skew ? G.lmin : G.met[a]);
        const double bl = std::sqrt(G.B[3 * a] * G.B[3 * a] + G.B[3 * a + 1] * G.B[3 * a + 1] +
                                    G.B[3 * a + 2] * G.B[3 * a + 2]);
        const double ext = G.skew ? std::sqrt(pp.rc2) * bl * G.dims[a] : std::sqrt(pp.rc2 / G.met[a]);
        pp.rcm[a] = G.use_cut ? static_cast<float>(ext) * 1.0001f + 1e-3f : 0.0f;
    }
    pp.use_cut = G.use_cut ? 1 : 0;
    pp.p32 = w.p32;
    pp.n32 = w.n32;
    pp.p64 = w.p64;
    pp.n64 = w.n64;
    pp.blo = w.blo;
    pp.bhi = w.bhi;
    pp.clo = w.clo;
    pp.chi = w.chi;
    pp.vrow = G.vrow;
    pp.A = w.A;
    pp.U = w.U;
    pp.stats = w.stats;
}

struct Launch {
    int threads = 512;
    int nctas = 1;
    int jt = 64;
    int ks0 = 0, ksn = 0;
};

// Opt-in shared memory per block on this device, less 1 KiB for static arrays.
int smem_budget() {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess || v <= 0)
        v = kMaxSmemBytes;
    return std::min(v, kMaxSmemBytes) - 1024;
}

int smem_rows_available(int threads, int S) {
    const int base = pair_smem_bytes(VDWDF_FP32, threads, 0, S);
    return std::max(0, (smem_budget() - base) / (band_stride(S) * static_cast<int>(sizeof(float))));
}

int ctas_per_sm(int precision, bool pot, int threads, int ksn, int S) {
    (void)pot;
    if (precision == VDWDF_FP32) return 1;  // the resident table band takes the shared memory
    (void)ksn;
    (void)S;
    return std::max(1, 1024 / threads);
}

// The pair loop's constants in precision R from the FP64 ones of sh.
template <typename R>
void fill_loop_consts(const PairShared &sh, LoopConsts<R> &k) {
    k.cD = static_cast<R>(sh.cD);
    k.cd = static_cast<R>(sh.cd);
    k.C = static_cast<R>(sh.C_asym);
    k.tDmax = static_cast<R>(sh.nD - 1);
    k.tdmax = static_cast<R>(sh.nd - 1);
    // FP32: the largest float below nD - 1 (nd - 1), so that the last cell is reached
    // with t < 1; FP64 clamps to the node and moves the last cell's index down instead
    k.tDclamp = sizeof(R) == 4 ? static_cast<R>(std::nextafter(static_cast<float>(sh.nD - 1), 0.0f)) : k.tDmax;
    k.tdclamp = sizeof(R) == 4 ? static_cast<R>(std::nextafter(static_cast<float>(sh.nd - 1), 0.0f)) : k.tdmax;
    k.iDmax = static_cast<R>(2.0 * sh.cD / (sh.nD - 1));  // cD = 1/(2 hD), Dmax = (nD - 1) hD
    k.om_rho0 = static_cast<R>(sh.om_rho0);
    k.kmax = sh.nD - 2;
    k.lmax = sh.nd - 2;
}

void fill_shared(const vdwdf_table *t, const double *d64, const float *d32, const Launch &ln,
                 unsigned int *queue, unsigned int max_iters, PairShared &sh) {
    sh.tab64 = d64;
    sh.tab32 = d32;
    sh.S = t->nd + 2;
    sh.nD = t->nD;
    sh.nd = t->nd;
    const double hD = t->Dmax / (t->nD - 1);
    sh.cD = 0.5 / hD;
    sh.cd = static_cast<double>(t->nd);
    sh.C_asym = 12.0 * std::pow(4.0 * kPi / 9.0, 3);
    // rho(0): the last node row at delta = 0 over eq. (17) at d1 = d2 = Dmax
    const double Dm = t->Dmax, Dm2 = Dm * Dm;
    const double p17 = -sh.C_asym / (2.0 * Dm2 * Dm2 * Dm2);
    sh.om_rho0 = 1.0 - t->nodes[static_cast<size_t>(t->nD - 1) * t->nd] / p17;
    fill_loop_consts(sh, sh.k32);
    fill_loop_consts(sh, sh.k64);
    sh.ks0 = ln.ks0;
    sh.ksn = ln.ksn;
    sh.jtiles_per_item = ln.jt;
    sh.item_limit = 0xFFFFFFFFu;
    sh.item_stride = 1u;
    sh.max_iters = max_iters_override(max_iters);
    sh.queue = queue;
    sh.item_E = nullptr;
    sh.item_cap = 0;
}

// A caller's launch shape: VDWDF_EINVAL outside the documented values,
// VDWDF_EUNSUPPORTED for a thread count the skewed kernel is not built for.
// The autotuner's candidate launch shapes (threads, items per warp slot, shared
// band rows, band start); the fourth is the energy-mode default.
constexpr int kTuneCount = 8;
constexpr vdwdf_tuning kTuneCandidates[kTuneCount] = {
    {256, 256, 0, -1}, {384, 256, 0, -1}, {448, 256, 0, -1}, {512, 256, 0, -1},
    {1024, 256, 0, -1}, {512, 64, 0, -1}, {512, 1024, 0, -1}, {512, 256, -1, 0}};

int check_tuning(const vdwdf_tuning *tu, bool skew, bool allow_auto = false) {
    if (!tu) return VDWDF_OK;
    const int t = tu->threads;
    if (allow_auto && t == VDWDF_TUNE_AUTO) return VDWDF_OK;  // the other fields are ignored
    if (t != 0 && t != 256 && t != 384 && t != 448 && t != 512 && t != 1024) return VDWDF_EINVAL;
    if (tu->items_per_sm < 0 || tu->smem_rows < -1 || tu->smem_row0 < -1) return VDWDF_EINVAL;
    if (skew && (t == 256 || t == 1024)) return VDWDF_EUNSUPPORTED;
    return VDWDF_OK;
}

// n_active: active points of one instance (the mean over a batch of ninst
// instances, whose items share the queue: the item target is split among them).
Launch choose_launch(int precision, bool pot, const vdwdf_tuning *tu, const vdwdf_table *t,
                     long long n_active, bool skew, int ninst = 1) {
    Launch ln;
    const int S = t->nd + 2;
    // Default shape: 512 threads, and for FP32 E + v 448 (384 on skewed cells).  The
    // potential pass ran 1-3 % faster with 14 warps (448 threads) than with 16 (512)
    // or 12 (384); 448 and 512 threads both cap a thread at 128 registers (up to
    // four warps share one scheduler's 16384), 384 at 168.  The skewed instance,
    // with its cross terms, was fastest at 384 and 8 % slower at 448.  Energy mode
    // gains from the extra warps of 512 threads.
    if (pot && precision == VDWDF_FP32) ln.threads = skew ? 384 : 448;
    if (tu && (tu->threads == 384 || tu->threads == 448 || tu->threads == 512 ||
               (!skew && (tu->threads == 256 || tu->threads == 1024))))
        ln.threads = tu->threads;  // skewed cells: the 384-, 448- and 512-thread kernels only
    const int sms = sm_count();
    ln.nctas = sms * ctas_per_sm(precision, pot, ln.threads, 0, S);
    // work items are (tile of kTile i points) x (jt j tiles); aim at ipsm items per
    // warp slot so that the dynamic queue balances uneven (culled) items
    int ipsm = (tu && tu->items_per_sm > 0) ? tu->items_per_sm : 256;
    const long long nT = std::max<long long>(1, (n_active + kTile - 1) / kTile);
    const long long want = std::max<long long>(1, static_cast<long long>(ipsm) * sms * (ln.threads / 32) / std::max(1, ninst));
    long long C = std::max<long long>(1, (want + nT - 1) / nT);
    C = std::min<long long>(C, nT);
    ln.jt = static_cast<int>(std::max<long long>(1, (nT + C - 1) / C));
    if (precision == VDWDF_FP32) {
        const int avail = smem_rows_available(ln.threads, S);
        int rows = std::min(avail, t->nD + 2);
        if (tu && tu->smem_rows < 0) rows = 0;
        if (tu && tu->smem_rows > 0) rows = std::min(rows, tu->smem_rows);
        ln.ksn = rows;
        // the band start is chosen on the device from the call's pairs (launch_band_choose);
        // below kBandAutoMin active points the choice would cost more than it can save
        constexpr long long kBandAutoMin = 16384;
        if ((!tu || tu->smem_row0 < 0) && rows >= 4 && rows < t->nD + 2 && t->nD - 1 <= kBandBins &&
            n_active >= kBandAutoMin) {
            ln.ks0 = -1;
        } else {
            const int r0 = (tu && tu->smem_row0 > 0) ? tu->smem_row0 : 0;
            ln.ks0 = std::max(0, std::min(r0, t->nD + 2 - rows));
        }
    }
    return ln;
}

struct Timer {
    cudaEvent_t e[4] = {nullptr, nullptr, nullptr, nullptr};
    bool ok = false;
    Timer() {
        ok = true;
        for (auto &x : e)
            if (cudaEventCreate(&x) != cudaSuccess) ok = false;
    }
    ~Timer() {
        for (auto &x : e)
            if (x) cudaEventDestroy(x);
    }
    void mark(int i, cudaStream_t st) {
        if (ok) cudaEventRecord(e[i], st);
    }
    float ms(int a, int b) {
        float v = 0.0f;
        if (ok && cudaEventElapsedTime(&v, e[a], e[b]) == cudaSuccess) return v;
        return 0.0f;
    }
};

void fill_result(const Stats &s, const Geom &G, const vdwdf_table *t, vdwdf_result *out) {
    out->E = 0.5 * G.dV * G.dV * s.E_pair;
    out->E_diag = 0.5 * G.dV * G.dV * s.n2sum * t->nodes[0];
    out->n_active = s.n_active;
    out->pairs = static_cast<int64_t>(s.pairs);
    out->pairs_evaluated = static_cast<int64_t>(s.evals);
    out->n_clamped = static_cast<int64_t>(s.clamped);
    float fmin, fmax;
    std::memcpy(&fmin, &s.qmin_bits, 4);
    std::memcpy(&fmax, &s.qmax_bits, 4);
    out->q0_min = s.n_active > 0 ? fmin : 0.0;
    out->q0_max = s.n_active > 0 ? fmax : 0.0;
}

// Single problem, energy or potential.
int run_single(const vdwdf_grid *grid, const double *n_dev, const double *grad_dev, double n_cut,
               double r_cut, const vdwdf_table *table, int precision, const vdwdf_tuning *tu,
               bool pot, double *v_dev, double *A_grid, double *U_grid, vdwdf_result *out,
               void *stream) {
    Geom G;
    int rc = check_grid(grid, G);
    if (rc) return rc;
    rc = check_cut(n_cut, r_cut, G);
    if (rc) return rc;
    if (!n_dev) return VDWDF_EINVAL;
    if (pot && !v_dev && !A_grid && !U_grid) return VDWDF_EINVAL;
    if (!table) return VDWDF_ENOTABLE;
    if (precision != VDWDF_FP32 && precision != VDWDF_FP64) return VDWDF_EINVAL;
    rc = check_tuning(tu, G.skew);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const long long launches0 = g_launches.load();
    double *d64 = nullptr;
    float *d32 = nullptr;
    rc = table_on_device(table, &d64, &d32);
    if (rc) return rc;
    int *order = nullptr, nb = 0;
    rc = brick_order(G.dims, &order, &nb);
    if (rc) return rc;
    const bool fp64 = precision == VDWDF_FP64;
    const size_t bytes = layout(G, nb, pot, fp64, nullptr, nullptr);
    unsigned char *base = nullptr;
    if (scratch_malloc_async(reinterpret_cast<void **>(&base), bytes, st) != cudaSuccess) return VDWDF_EALLOC;
    Work w;
    layout(G, nb, pot, fp64, &w, base);
    Timer tm;
    Stats hs;
    std::memset(&hs, 0, sizeof(hs));
    double *item_buf = nullptr;
    int row0 = 0;  // the band start given to the pair kernel (-1: chosen on the device)
    int threads = 0;  // the pair kernel's threads per CTA
    auto body = [&]() -> int {
        tm.mark(0, st);
        int r = prepare(G, n_dev, grad_dev, n_cut, pot, w, st);
        if (r) return r;
        VDWDF_CUDA_TRY(cudaMemcpyAsync(&hs, w.stats, sizeof(Stats), cudaMemcpyDeviceToHost, st));
        VDWDF_CUDA_TRY(cudaStreamSynchronize(st));
        tm.mark(1, st);
        if (pot) {
            VDWDF_CUDA_TRY(cudaMemsetAsync(w.A, 0, sizeof(double) * G.N, st));
            VDWDF_CUDA_TRY(cudaMemsetAsync(w.U, 0, sizeof(double) * G.N, st));
        }
        if (hs.n_active > 0) {
            Launch ln = choose_launch(precision, pot, tu, table, hs.n_active, G.skew);
            VDWDF_CUDA_TRY(cudaMemsetAsync(w.queue, 0, sizeof(unsigned int), st));
            PairLaunch pl;
            std::memset(&pl, 0, sizeof(pl));
            const long long items = pair_items(hs.n_active, ln.jt);
            if (items > 0xFFFFFFF0LL) return VDWDF_EINVAL;
            fill_shared(table, d64, d32, ln, w.queue, static_cast<unsigned int>(items + 2), pl.sh);
            if (!pot) {
                // one energy partial per work item, summed afterwards in a fixed order
                if (scratch_malloc_async(reinterpret_cast<void **>(&item_buf), sizeof(double) * items, st) != cudaSuccess)
                    return VDWDF_EALLOC;
                pl.sh.item_E = item_buf;
                pl.sh.item_cap = static_cast<unsigned int>(items);
            }
            pl.ninst = 1;
            fill_params(G, w, pl.inst[0]);
            if (ln.ks0 < 0) {
                r = launch_band_choose(pl, w.hist, st);
                if (r) return r;
            }
            row0 = ln.ks0;
            threads = ln.threads;
            r = launch_pair(precision, pot, G.skew, ln.threads, pl, ln.nctas, st);
            if (r) return r;
            r = launch_reduce_items(pl, st);
            if (r) return r;
        }
        tm.mark(2, st);
        if (pot) {
            r = assemble_v(G, w.slot, w.A, w.U, w.qn, w.qg, w.gsp, w.div, w.coef, v_dev, A_grid, U_grid, st);
            if (r) return r;
            r = launch_energy_from_A(static_cast<int>(G.N), w.A, w.n64, w.stats, st);
            if (r) return r;
        }
        tm.mark(3, st);
        VDWDF_CUDA_TRY(cudaMemcpyAsync(&hs, w.stats, sizeof(Stats), cudaMemcpyDeviceToHost, st));
        VDWDF_CUDA_TRY(cudaStreamSynchronize(st));
        return VDWDF_OK;
    };
    rc = body();
    if (item_buf) cudaFreeAsync(item_buf, st);
    cudaFreeAsync(base, st);
    if (rc == VDWDF_OK && hs.guard_trips) rc = VDWDF_ETIMEOUT;
    // non-finite input values (an Inf, or a NaN next to an active point) show up as
    // a non-finite sum; report them instead of returning NaN
    if (rc == VDWDF_OK && !std::isfinite(hs.E_pair)) rc = VDWDF_EINVAL;
    if (rc == VDWDF_OK && out) {
        std::memset(out, 0, sizeof(*out));
        fill_result(hs, G, table, out);
        out->ms_prep = tm.ms(0, 1);
        out->ms_pairs = tm.ms(1, 2);
        out->ms_post = tm.ms(2, 3);
        out->launches = static_cast<int32_t>(g_launches.load() - launches0);
        out->smem_row0 = precision == VDWDF_FP32 ? (row0 >= 0 ? row0 : hs.band_row0) : -1;
        out->pair_threads = threads;
    }
    if (rc == VDWDF_OK) {
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            note_cuda_error(e, "cudaStreamSynchronize", __FILE__, __LINE__);
            rc = VDWDF_ECUDA;
        }
    }
    return rc;
}

// ---------------------------------------------------------------------------
// batched energies: one persistent pair launch per kMaxInst instances,
// recorded into a CUDA graph and replayed for the same inputs
// ---------------------------------------------------------------------------
struct BatchPlan {
    unsigned long long table_gen = 0;  // the table the graph reads (its device copies)
    unsigned long long last_use = 0;   // for least-recently-used eviction
    std::vector<Geom> geo;
    std::vector<Work> work;
    std::vector<unsigned char *> bufs;
    unsigned int *queues = nullptr;  // one per pair launch
    std::vector<double *> item_bufs; // energy partials per work item, one buffer per launch
    std::vector<long long> item_caps;
    cudaGraphExec_t exec = nullptr;
    int device = 0;
    int launches_per_replay = 0;
    int row0 = 0;                    // band start of the first launch (-1: chosen on the device)
    int threads = 0;                 // the pair kernel's threads per CTA
    vdwdf_tuning tuned = {0, 0, 0, 0};  // VDWDF_TUNE_AUTO: the shape the autotuner chose
    ~BatchPlan() {
        if (exec) cudaGraphExecDestroy(exec);
        for (auto *b : bufs) cudaFree(b);
        for (auto *b : item_bufs) cudaFree(b);
        if (queues) cudaFree(queues);
    }
};

// Recorded batch graphs, keyed by everything the recording baked in.  At most
// kMaxPlans are kept (least recently used goes first); the plans of a table are
// dropped when it is freed.  A plan is only ever destroyed under g_batch_mu, which
// a batched call holds until its replay has finished on its stream.
std::mutex g_batch_mu;
std::map<std::vector<uintptr_t>, BatchPlan *> g_batches;
constexpr size_t kMaxPlans = 8;
unsigned long long g_batch_clock = 0;

void destroy_plan(BatchPlan *bp) {
    int cur = 0;
    const bool have = cudaGetDevice(&cur) == cudaSuccess;
    if (!have || cur != bp->device) cudaSetDevice(bp->device);
    const int dev = bp->device;
    delete bp;
    if (have && cur != dev) cudaSetDevice(cur);
}

int record_batch(BatchPlan &bp, int ninst, const double *const *n_dev, double n_cut,
                 const vdwdf_table *table, int precision, const vdwdf_tuning *tu, double *d64,
                 float *d32, cudaStream_t st) {
    long long nmax = 0, nsum = 0;
    for (int k = 0; k < ninst; ++k) {
        nmax = std::max(nmax, bp.geo[k].N);
        nsum += bp.geo[k].N;
    }
    const int ngroups = (ninst + kMaxInst - 1) / kMaxInst;
    for (int k = 0; k < ninst; ++k) {
        int rc = prepare(bp.geo[k], n_dev[k], nullptr, n_cut, false, bp.work[k], st);
        if (rc) return rc;
    }
    for (int g = 0; g < ngroups; ++g) {
        const int k0 = g * kMaxInst, k1 = std::min(ninst, k0 + kMaxInst);
        long long gsum = 0;
        for (int k = k0; k < k1; ++k) gsum += bp.geo[k].N;
        bool gskew = false;
        for (int k = k0; k < k1; ++k) gskew = gskew || bp.geo[k].skew;
        Launch ln = choose_launch(precision, false, tu, table, std::max<long long>(1, gsum / (k1 - k0)), gskew, k1 - k0);
        VDWDF_CUDA_TRY(cudaMemsetAsync(bp.queues + g, 0, sizeof(unsigned int), st));
        PairLaunch pl;
        std::memset(&pl, 0, sizeof(pl));
        long long items = 0;
        for (int k = k0; k < k1; ++k) items += pair_items(bp.geo[k].N, ln.jt);
        if (items > 0xFFFFFFF0LL) return VDWDF_EINVAL;
        fill_shared(table, d64, d32, ln, bp.queues + g, static_cast<unsigned int>(items + 2), pl.sh);
        pl.sh.item_E = bp.item_bufs[g];
        pl.sh.item_cap = static_cast<unsigned int>(bp.item_caps[g]);
        pl.ninst = k1 - k0;
        bool skew = false;
        for (int k = k0; k < k1; ++k) {
            fill_params(bp.geo[k], bp.work[k], pl.inst[k - k0]);
            skew = skew || bp.geo[k].skew;
        }
        if (g == 0) {
            bp.row0 = ln.ks0;
            bp.threads = ln.threads;
        }
        if (ln.ks0 < 0) {
            int rc = launch_band_choose(pl, bp.work[k0].hist, st);
            if (rc) return rc;
        }
        int rc = launch_pair(precision, false, skew, ln.threads, pl, ln.nctas, st);
        if (rc) return rc;
        rc = launch_reduce_items(pl, st);
        if (rc) return rc;
    }
    (void)nmax;
    (void)nsum;
    return VDWDF_OK;
}

// ---------------------------------------------------------------------------
// voxel-averaged diagonal: the quadrature rule and the small-D model
// ---------------------------------------------------------------------------
constexpr int kPhi0Panels = 6, kPhi0Points = 8;

// Gauss-Legendre nodes and weights on [-1, 1] (Newton on the three-term recurrence).
void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = std::cos(kPi * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            const double pn = (n == 1) ? z : p1, pm = (n == 1) ? 1.0 : p0;
            dp = n * (z * pn - pm) / (z * z - 1.0);
            const double dz = pn / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = -z;
        x[n - 1 - i] = z;
        w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// Nodes then weights on [0, 1]: np-point Gauss rules on the geometric panels
// [0, 2^-(P-1)], ..., [1/4, 1/2], [1/2, 1], graded towards the singular corner.
void phi0_rule(std::vector<double> &xw) {
    std::vector<double> gx, gw;
    gauss_legendre(kPhi0Points, gx, gw);
    const int nn = kPhi0Panels * kPhi0Points;
    xw.assign(2 * nn, 0.0);
    for (int p = 0; p < kPhi0Panels; ++p) {
        const double a = (p == 0) ? 0.0 : std::ldexp(1.0, p - kPhi0Panels);
        const double b = std::ldexp(1.0, p + 1 - kPhi0Panels);
        for (int k = 0; k < kPhi0Points; ++k) {
            xw[p * kPhi0Points + k] = 0.5 * (a + b) + 0.5 * (b - a) * gx[k];
            xw[nn + p * kPhi0Points + k] = 0.5 * (b - a) * gw[k];
        }
    }
}

// The kernel at delta = 0 below D_1 = Dmax/(nD - 1): -(2/pi) ln D + psi0 + c2 D^2,
// psi = phi + (2/pi) ln D fitted at the nodes D_1 and D_2.
void phi0_model(const vdwdf_table *t, const double vox[9], Phi0Rule &rule) {
    for (int k = 0; k < 9; ++k) rule.v[k] = vox[k];
    const double D1 = t->Dmax / (t->nD - 1);
    const double psi1 = t->nodes[static_cast<size_t>(1) * t->nd] + (2.0 / kPi) * std::log(D1);
    const double psi2 = t->nodes[static_cast<size_t>(2) * t->nd] + (2.0 / kPi) * std::log(2.0 * D1);
    rule.D1 = D1;
    rule.psi0 = (4.0 * psi1 - psi2) / 3.0;
    rule.c2 = (psi1 - rule.psi0) / (D1 * D1);
    rule.nn = kPhi0Panels * kPhi0Points;
}

}  // namespace

void note_cuda_error(cudaError_t e, const char *what, const char *file, int line) {
    if (std::getenv("VDWDF_VERBOSE"))
        std::fprintf(stderr, "vdwdf: %s failed: %s (%s:%d)\n", what, cudaGetErrorString(e), file, line);
}

void count_launches(int n) { g_launches.fetch_add(n); }

}  // namespace vdwdf

using namespace vdwdf;

extern "C" {

const char *vdwdf_strerror(int s) {
    switch (s) {
        case VDWDF_OK: return "ok";
        case VDWDF_EINVAL: return "invalid argument";
        case VDWDF_EUNSUPPORTED: return "valid input beyond what this entry point supports";
        case VDWDF_ECUDA: return "CUDA runtime error";
        case VDWDF_EALLOC: return "allocation failed";
        case VDWDF_ETIMEOUT: return "device work loop hit its iteration cap";
        case VDWDF_ENOTABLE: return "missing or mismatched kernel table";
        default: return "unknown status";
    }
}

int vdwdf_version(void) { return VDWDF_VERSION; }

int vdwdf_total_energy_nl(double E_tot_dft, const vdwdf_semilocal_result *semi, double E_c_nl, int exchange,
                          double *E_out) {
    if (!semi || !E_out || (exchange != VDWDF_X_PBE && exchange != VDWDF_X_REVPBE)) return VDWDF_EINVAL;
    const double ex = exchange == VDWDF_X_PBE ? semi->Ex_pbe : semi->Ex_revpbe;
    // eq. (3): the PBE exchange-correlation is taken out and replaced by the
    // chosen exchange, LDA correlation and the nonlocal correlation
    const double E = E_tot_dft - semi->Ex_pbe - semi->Ec_pbe + (ex + semi->Ec_lda + E_c_nl);
    if (!std::isfinite(E)) return VDWDF_EINVAL;
    *E_out = E;
    return VDWDF_OK;
}

int64_t vdwdf_launch_count(void) { return g_launches.load(); }

int vdwdf_table_build(int nD, double Dmax, int ndelta, int quad_level, double *phi_nodes_out,
                      vdwdf_table **out) {
    if (!out || nD < 4 || ndelta < 4 || !(Dmax > 0.0) || !std::isfinite(Dmax) || quad_level < 0 ||
        quad_level > 2 || static_cast<long long>(nD) * ndelta > (1LL << 26))
        return VDWDF_EINVAL;
    vdwdf_table *t = new (std::nothrow) vdwdf_table;
    if (!t) return VDWDF_EALLOC;
    t->nD = nD;
    t->nd = ndelta;
    t->Dmax = Dmax;
    try {
        t->nodes.assign(static_cast<size_t>(nD) * ndelta, 0.0);
    } catch (const std::bad_alloc &) {
        delete t;
        return VDWDF_EALLOC;
    }
    if (build_phi_nodes(nD, Dmax, ndelta, quad_level, t->nodes.data()) != 0) {
        delete t;
        return VDWDF_EALLOC;
    }
    int rc = finish_table(t);
    if (rc) {
        delete t;
        return rc;
    }
    if (phi_nodes_out) std::memcpy(phi_nodes_out, t->nodes.data(), sizeof(double) * t->nodes.size());
    *out = t;
    return VDWDF_OK;
}

int vdwdf_table_from_nodes(int nD, double Dmax, int ndelta, const double *phi_nodes, vdwdf_table **out) {
    if (!out || !phi_nodes || nD < 4 || ndelta < 4 || !(Dmax > 0.0) || !std::isfinite(Dmax) ||
        static_cast<long long>(nD) * ndelta > (1LL << 26))
        return VDWDF_EINVAL;
    for (long long i = 0; i < static_cast<long long>(nD) * ndelta; ++i)
        if (!std::isfinite(phi_nodes[i])) return VDWDF_EINVAL;
    vdwdf_table *t = new (std::nothrow) vdwdf_table;
    if (!t) return VDWDF_EALLOC;
    t->nD = nD;
    t->nd = ndelta;
    t->Dmax = Dmax;
    try {
        t->nodes.assign(phi_nodes, phi_nodes + static_cast<size_t>(nD) * ndelta);
    } catch (const std::bad_alloc &) {
        delete t;
        return VDWDF_EALLOC;
    }
    int rc = finish_table(t);
    if (rc) {
        delete t;
        return rc;
    }
    *out = t;
    return VDWDF_OK;
}

int vdwdf_table_nodes(const vdwdf_table *t, double *phi_nodes_out) {
    if (!t || !phi_nodes_out) return VDWDF_EINVAL;
    std::memcpy(phi_nodes_out, t->nodes.data(), sizeof(double) * t->nodes.size());
    return VDWDF_OK;
}

int vdwdf_table_info(const vdwdf_table *t, int *nD, double *Dmax, int *ndelta) {
    if (!t) return VDWDF_EINVAL;
    if (nD) *nD = t->nD;
    if (Dmax) *Dmax = t->Dmax;
    if (ndelta) *ndelta = t->nd;
    return VDWDF_OK;
}

void vdwdf_table_free(vdwdf_table *t) {
    if (!t) return;
    {
        // recorded batch graphs read this table's device copies: drop them first
        std::lock_guard<std::mutex> lk(g_batch_mu);
        for (auto it = g_batches.begin(); it != g_batches.end();) {
            if (it->second->table_gen == t->gen) {
                destroy_plan(it->second);
                it = g_batches.erase(it);
            } else {
                ++it;
            }
        }
    }
    int cur = 0;
    const bool have = cudaGetDevice(&cur) == cudaSuccess;
    for (auto &kv : t->dev) {
        if (cudaSetDevice(kv.first) == cudaSuccess) {
            cudaFree(kv.second.first);
            cudaFree(kv.second.second);
        }
    }
    if (have) cudaSetDevice(cur);
    delete t;
}

int vdwdf_kernel_eval(const vdwdf_table *t, int precision, int64_t npts, const double *r_dev,
                      const double *qi_dev, const double *qj_dev, double *phi_dev, double *rdphi_dev,
                      void *cuda_stream) {
    if (!t) return VDWDF_ENOTABLE;
    if (npts < 0 || (npts > 0 && (!r_dev || !qi_dev || !qj_dev || !phi_dev || !rdphi_dev)))
        return VDWDF_EINVAL;
    if (precision != VDWDF_FP32 && precision != VDWDF_FP64) return VDWDF_EINVAL;
    if (npts == 0) return VDWDF_OK;
    double *d64 = nullptr;
    float *d32 = nullptr;
    int rc = table_on_device(t, &d64, &d32);
    if (rc) return rc;
    Launch ln;
    PairShared sh;
    std::memset(&sh, 0, sizeof(sh));
    fill_shared(t, d64, d32, ln, nullptr, 0, sh);
    return launch_kernel_eval(precision, sh, npts, r_dev, qi_dev, qj_dev, phi_dev, rdphi_dev,
                              static_cast<cudaStream_t>(cuda_stream));
}

int vdwdf_q0(const vdwdf_grid *grid, const double *n_dev, const double *grad_dev, double n_cut,
             double *q0_dev, double *dq0dn_dev, double *dq0dg_dev, void *cuda_stream) {
    (void)n_cut;
    Geom G;
    int rc = check_grid(grid, G);
    if (rc) return rc;
    if (!n_dev || !q0_dev) return VDWDF_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (grad_dev || !G.spectral) return launch_grad_q0(G.dims, G.am, n_dev, grad_dev, q0_dev, dq0dn_dev, dq0dg_dev, st);
    double *buf = nullptr;
    const size_t nd = 3 * static_cast<size_t>(G.N) + G.dims[0] + G.dims[1] + G.dims[2];
    if (scratch_malloc_async(reinterpret_cast<void **>(&buf), nd * sizeof(double), st) != cudaSuccess)
        return VDWDF_EALLOC;
    const double *g_use = nullptr;
    rc = q0_gradient(G, n_dev, nullptr, buf, buf + 3 * G.N, &g_use, st);
    if (rc == VDWDF_OK) rc = launch_grad_q0(G.dims, G.am, n_dev, g_use, q0_dev, dq0dn_dev, dq0dg_dev, st);
    cudaFreeAsync(buf, st);
    return rc;
}

int vdwdf_gradient(const vdwdf_grid *grid, const double *n_dev, double *grad_dev, void *cuda_stream) {
    Geom G;
    int rc = check_grid(grid, G);
    if (rc) return rc;
    if (!n_dev || !grad_dev) return VDWDF_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (!G.spectral) return launch_gradient_fd(G.dims, G.am, n_dev, grad_dev, st);
    double *coef = nullptr;
    const size_t nc = static_cast<size_t>(G.dims[0] + G.dims[1] + G.dims[2]);
    if (scratch_malloc_async(reinterpret_cast<void **>(&coef), nc * sizeof(double), st) != cudaSuccess)
        return VDWDF_EALLOC;
    rc = launch_gradient_spectral(G.dims, recip_of(G), n_dev, grad_dev, coef, st);
    cudaFreeAsync(coef, st);
    return rc;
}

int vdwdf_semilocal(const vdwdf_grid *grid, const double *n_dev, const double *grad_dev,
                    vdwdf_semilocal_result *out, void *cuda_stream) {
    Geom G;
    int rc = check_grid(grid, G);
    if (rc) return rc;
    if (!n_dev || !out) return VDWDF_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const long long launches0 = g_launches.load();
    const size_t nd = static_cast<size_t>(semilocal_scratch_doubles());
    // the spectral gradient (when the grid asks for it and none is given) after the sums
    const size_t nsp = (G.spectral && !grad_dev) ? 3 * static_cast<size_t>(G.N) + G.dims[0] + G.dims[1] + G.dims[2] : 0;
    double *scratch = nullptr;
    if (scratch_malloc_async(reinterpret_cast<void **>(&scratch), (nd + nsp) * sizeof(double), st) != cudaSuccess)
        return VDWDF_EALLOC;
    Timer tm;
    double sums[6] = {0, 0, 0, 0, 0, 0};
    tm.mark(0, st);
    const double *g_use = nullptr;
    rc = q0_gradient(G, n_dev, grad_dev, scratch + nd, scratch + nd + 3 * G.N, &g_use, st);
    if (rc == VDWDF_OK) rc = launch_semilocal(G.dims, G.am, n_dev, g_use, scratch, st);
    tm.mark(1, st);
    if (rc == VDWDF_OK &&
        cudaMemcpyAsync(sums, scratch + nd - 6, sizeof(sums), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        rc = VDWDF_ECUDA;
    cudaFreeAsync(scratch, st);
    if (rc == VDWDF_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = VDWDF_ECUDA;
    if (rc) return rc;
    std::memset(out, 0, sizeof(*out));
    out->Ex_lda = G.dV * sums[0];
    out->Ec_lda = G.dV * sums[1];
    out->Ex_pbe = G.dV * sums[2];
    out->Ec_pbe = G.dV * sums[3];
    out->Ex_revpbe = G.dV * sums[4];
    out->n_points = static_cast<int64_t>(sums[5]);
    out->ms = tm.ms(0, 1);
    out->launches = static_cast<int32_t>(g_launches.load() - launches0);
    return VDWDF_OK;
}

int vdwdf_phi0_eval(const vdwdf_table *table, const double *voxel, int64_t nq, const double *q_dev,
                    double *phi0_dev, void *cuda_stream) {
    if (!table) return VDWDF_ENOTABLE;
    if (!voxel || nq < 0 || nq > (1LL << 30) || (nq > 0 && (!q_dev || !phi0_dev))) return VDWDF_EINVAL;
    for (int k = 0; k < 9; ++k)
        if (!std::isfinite(voxel[k])) return VDWDF_EINVAL;
    if (table->nD < 3) return VDWDF_EINVAL;
    if (nq == 0) return VDWDF_OK;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    double *d64 = nullptr;
    float *d32 = nullptr;
    int rc = table_on_device(table, &d64, &d32);
    if (rc) return rc;
    Phi0Rule rule;
    phi0_model(table, voxel, rule);
    std::vector<double> xw;
    phi0_rule(xw);
    double *xw_dev = nullptr;
    if (scratch_malloc_async(reinterpret_cast<void **>(&xw_dev), sizeof(double) * (xw.size() + 8 * nq), st) !=
        cudaSuccess)
        return VDWDF_EALLOC;
    Launch ln;
    PairShared sh;
    std::memset(&sh, 0, sizeof(sh));
    fill_shared(table, d64, d32, ln, nullptr, 0, sh);
    if (cudaMemcpyAsync(xw_dev, xw.data(), sizeof(double) * xw.size(), cudaMemcpyHostToDevice, st) != cudaSuccess)
        rc = VDWDF_ECUDA;
    if (rc == VDWDF_OK)
        rc = launch_phi0(sh, rule, static_cast<int>(nq), q_dev, xw_dev, xw_dev + xw.size(), phi0_dev, st);
    cudaFreeAsync(xw_dev, st);
    if (rc == VDWDF_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = VDWDF_ECUDA;
    return rc;
}

}  // extern "C"

namespace vdwdf {
namespace {

// The voxel diagonal; with dv_dev, also the change of v from replacing the table
// self term by it (library stencil only).
int diag_voxel(const vdwdf_grid *grid, const double *n_dev, const double *grad_dev, double n_cut,
               const vdwdf_table *table, int nphi0, double *dv_dev, vdwdf_diag_result *out, void *cuda_stream) {
    Geom G;
    int rc = check_grid(grid, G);
    if (rc) return rc;
    if (!n_dev || !out) return VDWDF_EINVAL;
    if (!(n_cut > 0.0) || !std::isfinite(n_cut)) return VDWDF_EINVAL;
    if (!table) return VDWDF_ENOTABLE;
    const int nq = nphi0 == 0 ? 100 : nphi0;
    if (nq < 4 || nq > 100000) return VDWDF_EINVAL;
    if (table->nD < 3) return VDWDF_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const long long launches0 = g_launches.load();
    double *d64 = nullptr;
    float *d32 = nullptr;
    rc = table_on_device(table, &d64, &d32);
    if (rc) return rc;
    Phi0Rule rule;
    double vox[9];
    for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) vox[3 * a + c] = grid->cell[a][c] / G.dims[a];
    phi0_model(table, vox, rule);
    std::vector<double> xw;
    phi0_rule(xw);
    // scratch: q0 [N], range (3), block sums (2 x 608), sums (2), q grid and table [nq], rule nodes
    const bool pot = dv_dev != nullptr;
    Carve c;
    const size_t o_q0 = c.take<double>(G.N), o_mm = c.take<unsigned long long>(3), o_part = c.take<double>(2 * 608),
                 o_sums = c.take<double>(2), o_qg = c.take<double>(nq), o_tab = c.take<double>(nq),
                 o_xw = c.take<double>(xw.size()), o_op = c.take<double>(8 * static_cast<size_t>(nq));
    const size_t o_qn = pot ? c.take<double>(G.N) : 0, o_qgr = pot ? c.take<double>(3 * G.N) : 0,
                 o_slot = pot ? c.take<int>(G.N) : 0, o_A = pot ? c.take<double>(G.N) : 0,
                 o_U = pot ? c.take<double>(G.N) : 0;
    // spectral gradient: the gradient (then the potential's weights), coefficients, divergence
    const size_t o_gsp = G.spectral ? c.take<double>(3 * G.N) : 0,
                 o_coef = G.spectral ? c.take<double>(G.dims[0] + G.dims[1] + G.dims[2]) : 0,
                 o_div = (G.spectral && pot) ? c.take<double>(G.N) : 0;
    unsigned char *base = nullptr;
    if (scratch_malloc_async(reinterpret_cast<void **>(&base), c.off, st) != cudaSuccess) return VDWDF_EALLOC;
    double *q0 = reinterpret_cast<double *>(base + o_q0);
    unsigned long long *mm = reinterpret_cast<unsigned long long *>(base + o_mm);
    double *part = reinterpret_cast<double *>(base + o_part), *sums = reinterpret_cast<double *>(base + o_sums);
    double *qg = reinterpret_cast<double *>(base + o_qg), *tab = reinterpret_cast<double *>(base + o_tab);
    double *xw_dev = reinterpret_cast<double *>(base + o_xw), *opart = reinterpret_cast<double *>(base + o_op);
    double *qn = pot ? reinterpret_cast<double *>(base + o_qn) : nullptr;
    double *qgr = pot ? reinterpret_cast<double *>(base + o_qgr) : nullptr;
    int *slot = pot ? reinterpret_cast<int *>(base + o_slot) : nullptr;
    double *Ad = pot ? reinterpret_cast<double *>(base + o_A) : nullptr;
    double *Ud = pot ? reinterpret_cast<double *>(base + o_U) : nullptr;
    double *gsp = G.spectral ? reinterpret_cast<double *>(base + o_gsp) : nullptr;
    double *coef = G.spectral ? reinterpret_cast<double *>(base + o_coef) : nullptr;
    double *divb = (G.spectral && pot) ? reinterpret_cast<double *>(base + o_div) : nullptr;
    Timer tm;
    unsigned long long hmm[3] = {0, 0, 0};
    double hs[2] = {0.0, 0.0};
    std::vector<double> qh(nq);
    double lnq0 = 0.0, dlnq = 1.0;
    auto body = [&]() -> int {
        tm.mark(0, st);
        const double *g_use = nullptr;
        int r = q0_gradient(G, n_dev, grad_dev, gsp, coef, &g_use, st);
        if (r) return r;
        r = launch_grad_q0(G.dims, G.am, n_dev, g_use, q0, qn, qgr, st);
        if (r) return r;
        if (pot) VDWDF_CUDA_TRY(cudaMemsetAsync(dv_dev, 0, sizeof(double) * G.N, st));
        VDWDF_CUDA_TRY(cudaMemsetAsync(mm, 0xFF, sizeof(unsigned long long), st));
        VDWDF_CUDA_TRY(cudaMemsetAsync(mm + 1, 0, 2 * sizeof(unsigned long long), st));
        r = launch_diag_range(G.N, n_dev, q0, n_cut, mm, st);
        if (r) return r;
        VDWDF_CUDA_TRY(cudaMemcpyAsync(hmm, mm, sizeof(hmm), cudaMemcpyDeviceToHost, st));
        VDWDF_CUDA_TRY(cudaStreamSynchronize(st));
        if (hmm[2] == 0) return VDWDF_OK;
        double qmin, qmax;
        std::memcpy(&qmin, &hmm[0], 8);
        std::memcpy(&qmax, &hmm[1], 8);
        // log-spaced table, slightly wider than the range so that every q0 interpolates inside
        const double lo = std::log(qmin), hi = std::log(qmax);
        const double pad = 1e-6 + 1e-9 * std::fabs(hi);
        lnq0 = lo - pad;
        dlnq = (hi + pad - lnq0) / (nq - 1);
        for (int k = 0; k < nq; ++k) qh[k] = std::exp(lnq0 + k * dlnq);
        VDWDF_CUDA_TRY(cudaMemcpyAsync(qg, qh.data(), sizeof(double) * nq, cudaMemcpyHostToDevice, st));
        VDWDF_CUDA_TRY(cudaMemcpyAsync(xw_dev, xw.data(), sizeof(double) * xw.size(), cudaMemcpyHostToDevice, st));
        Launch ln;
        PairShared sh;
        std::memset(&sh, 0, sizeof(sh));
        fill_shared(table, d64, d32, ln, nullptr, 0, sh);
        r = launch_phi0(sh, rule, nq, qg, xw_dev, opart, tab, st);
        if (r) return r;
        r = launch_diag_sum(G.N, n_dev, q0, n_cut, tab, nq, lnq0, dlnq, part, sums, st);
        if (r) return r;
        if (pot) {
            r = launch_diag_AU(G.N, n_dev, q0, n_cut, tab, nq, lnq0, dlnq, table->nodes[0], slot, Ad, Ud, st);
            if (r) return r;
            r = assemble_v(G, slot, Ad, Ud, qn, qgr, gsp, divb, coef, dv_dev, nullptr, nullptr, st);
            if (r) return r;
        }
        tm.mark(1, st);
        VDWDF_CUDA_TRY(cudaMemcpyAsync(hs, sums, sizeof(hs), cudaMemcpyDeviceToHost, st));
        VDWDF_CUDA_TRY(cudaStreamSynchronize(st));
        return VDWDF_OK;
    };
    rc = body();
    cudaFreeAsync(base, st);
    if (rc == VDWDF_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = VDWDF_ECUDA;
    if (rc) return rc;
    std::memset(out, 0, sizeof(*out));
    out->n_active = static_cast<int64_t>(hmm[2]);
    out->nphi0 = nq;
    if (hmm[2]) {
        std::memcpy(&out->q0_min, &hmm[0], 8);
        std::memcpy(&out->q0_max, &hmm[1], 8);
        out->E_diag_voxel = 0.5 * G.dV * G.dV * hs[0];
        out->E_diag_table = 0.5 * G.dV * G.dV * hs[1] * table->nodes[0];
        out->ms = tm.ms(0, 1);
    }
    out->launches = static_cast<int32_t>(g_launches.load() - launches0);
    return VDWDF_OK;
}

// The autotuner: the energy pass of each candidate launch shape on a strided
// sample of the work items (every stride-th item, about 16 items per warp slot,
// spread over the whole i <-> j triangle), timed twice with CUDA events on the
// stream; the second timing counts.  The candidate with the most pair
// evaluations per millisecond wins.
int autotune_one(const Geom &G, const double *n_dev, double n_cut, const vdwdf_table *table, int precision,
                 vdwdf_tuning *best, cudaStream_t st) {
    double *d64 = nullptr;
    float *d32 = nullptr;
    int rc = table_on_device(table, &d64, &d32);
    if (rc) return rc;
    int *order = nullptr, nb = 0;
    rc = brick_order(G.dims, &order, &nb);
    if (rc) return rc;
    const bool fp64 = precision == VDWDF_FP64;
    const size_t bytes = layout(G, nb, false, fp64, nullptr, nullptr);
    unsigned char *base = nullptr;
    if (scratch_malloc_async(reinterpret_cast<void **>(&base), bytes, st) != cudaSuccess) return VDWDF_EALLOC;
    Work w;
    layout(G, nb, false, fp64, &w, base);
    rc = prepare(G, n_dev, nullptr, n_cut, false, w, st);
    Stats hs;
    std::memset(&hs, 0, sizeof(hs));
    if (rc == VDWDF_OK && cudaMemcpyAsync(&hs, w.stats, sizeof(Stats), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        rc = VDWDF_ECUDA;
    if (rc == VDWDF_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = VDWDF_ECUDA;
    double best_rate = -1.0;
    vdwdf_tuning choice = kTuneCandidates[3];
    Timer tm;
    for (int ci = 0; ci < kTuneCount && rc == VDWDF_OK && hs.n_active > 0; ++ci) {
        const vdwdf_tuning &cd = kTuneCandidates[ci];
        if (fp64 && cd.smem_rows != 0) continue;
        if (check_tuning(&cd, G.skew) != VDWDF_OK) continue;  // no such kernel for this cell
        Launch ln = choose_launch(precision, false, &cd, table, hs.n_active, G.skew);
        const long long total = pair_items(hs.n_active, ln.jt);
        const long long want = 16LL * ln.nctas * (ln.threads / 32);
        const long long stride = std::max<long long>(1, total / std::max<long long>(1, want));
        for (int rep = 0; rep < 2 && rc == VDWDF_OK; ++rep) {
            if (cudaMemsetAsync(w.queue, 0, sizeof(unsigned int), st) != cudaSuccess) rc = VDWDF_ECUDA;
            Stats zero;
            std::memset(&zero, 0, sizeof(zero));
            zero.n_active = hs.n_active;
            if (rc == VDWDF_OK &&
                cudaMemcpyAsync(w.stats, &zero, sizeof(Stats), cudaMemcpyHostToDevice, st) != cudaSuccess)
                rc = VDWDF_ECUDA;
            PairLaunch pl;
            std::memset(&pl, 0, sizeof(pl));
            fill_shared(table, d64, d32, ln, w.queue, 0xFFFFFFF0u, pl.sh);
            pl.sh.item_limit = static_cast<unsigned int>(std::min<long long>(want, 0xFFFFFFF0LL));
            pl.sh.item_stride = static_cast<unsigned int>(std::min<long long>(stride, 0xFFFFFFF0LL));
            pl.ninst = 1;
            fill_params(G, w, pl.inst[0]);
            if (rc == VDWDF_OK && ln.ks0 < 0) rc = launch_band_choose(pl, w.hist, st);
            tm.mark(0, st);
            if (rc == VDWDF_OK) rc = launch_pair(precision, false, G.skew, ln.threads, pl, ln.nctas, st);
            tm.mark(1, st);
            Stats out;
            if (rc == VDWDF_OK &&
                cudaMemcpyAsync(&out, w.stats, sizeof(Stats), cudaMemcpyDeviceToHost, st) != cudaSuccess)
                rc = VDWDF_ECUDA;
            if (rc == VDWDF_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = VDWDF_ECUDA;
            const double ms = tm.ms(0, 1);
            if (rc == VDWDF_OK && rep == 1 && ms > 0.0) {
                const double rate = static_cast<double>(out.evals) / ms;
                if (rate > best_rate) {
                    best_rate = rate;
                    choice = cd;
                }
            }
        }
    }
    cudaFreeAsync(base, st);
    if (rc == VDWDF_OK) *best = choice;
    return rc;
}

}  // namespace
}  // namespace vdwdf

extern "C" {

int vdwdf_far_tail(const vdwdf_grid *grid, const double *n_dev, const double *grad_dev, double n_cut,
                   double r_cut, double *v_dev, vdwdf_tail_result *out, void *cuda_stream) {
    using namespace vdwdf;
    Geom G;
    int rc = check_grid(grid, G);
    if (rc) return rc;
    if (!n_dev || !out) return VDWDF_EINVAL;
    const bool pot = v_dev != nullptr;
    if (pot && grad_dev) return VDWDF_EINVAL;  // the potential needs the library's own gradient
    if (!(n_cut > 0.0) || !std::isfinite(n_cut) || !(r_cut > 0.0) || !std::isfinite(r_cut)) return VDWDF_EINVAL;
    const int nper = (G.per[0] != 0) + (G.per[1] != 0) + (G.per[2] != 0);
    if (nper < 1) return VDWDF_EUNSUPPORTED;
    // geometry: the cell's volume; with two periodic axes the area of their plane, its
    // unit normal e and the spacing dz = |M_ax . e| / N_ax of the planes along the
    // third axis ax; with one periodic axis ax its length, and the metric of the
    // other two axes' grid steps with their components along M_ax removed
    double M[3][3];
    for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) M[a][c] = grid->cell[a][c];
    auto cross = [](const double *x, const double *y, double *z) {
        z[0] = x[1] * y[2] - x[2] * y[1];
        z[1] = x[2] * y[0] - x[0] * y[2];
        z[2] = x[0] * y[1] - x[1] * y[0];
    };
    auto dot = [](const double *x, const double *y) { return x[0] * y[0] + x[1] * y[1] + x[2] * y[2]; };
    double x01[3];
    cross(M[0], M[1], x01);
    const double V = std::fabs(dot(x01, M[2]));
    int ax = 0, np = 1;
    double dz = 0.0, c2 = 0.0, c3 = 0.0;
    double gbb = 0.0, gbc = 0.0, gcc = 0.0, pref = 0.0;
    int nlines = 0, Nc = 1;
    if (nper == 2) {
        ax = G.per[0] == 0 ? 0 : (G.per[1] == 0 ? 1 : 2);
        const int a = ax == 0 ? 1 : 0, b = ax == 2 ? 1 : 2;
        double e[3];
        cross(M[a], M[b], e);
        const double A = std::sqrt(dot(e, e));
        dz = std::fabs(dot(M[ax], e)) / A / G.dims[ax];
        np = G.dims[ax];
        c2 = (2.0 * kPi / A) / 4.0;
    } else if (nper == 3) {
        c3 = (4.0 * kPi / V) / (3.0 * r_cut * r_cut * r_cut);
    } else {
        ax = G.per[0] ? 0 : (G.per[1] ? 1 : 2);
        const int b = ax == 0 ? 1 : 0, c = ax == 2 ? 1 : 2;
        const double alen = std::sqrt(dot(M[ax], M[ax]));
        double wb[3], wc[3];
        for (int k = 0; k < 3; ++k) {
            wb[k] = M[b][k] / G.dims[b];
            wc[k] = M[c][k] / G.dims[c];
        }
        const double pb = dot(wb, M[ax]) / (alen * alen), pc = dot(wc, M[ax]) / (alen * alen);
        for (int k = 0; k < 3; ++k) {
            wb[k] -= pb * M[ax][k];
            wc[k] -= pc * M[ax][k];
        }
        gbb = dot(wb, wb);
        gbc = dot(wb, wc);
        gcc = dot(wc, wc);
        pref = 2.0 / alen;
        Nc = G.dims[c];
        nlines = G.dims[b] * G.dims[c];
    }
    constexpr int kMaxNodes = 4096;
    constexpr int kMaxLines = 65536;   // active lines of one periodic axis (K over their pairs)
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const long long launches0 = g_launches.load();
    // the planes' F and G; for one periodic axis the lines' buffers come later, once
    // the active lines are known
    const size_t ngroup = nper == 1 ? 1 : static_cast<size_t>(np);
    Carve cv;
    const size_t o_q0 = cv.take<double>(G.N), o_mm = cv.take<unsigned long long>(3),
                 o_F = cv.take<double>(static_cast<size_t>(kMaxNodes) * ngroup), o_Tk = cv.take<double>(kMaxNodes),
                 o_out = cv.take<double>(1);
    const size_t o_gsp = G.spectral ? cv.take<double>(3 * G.N) : 0,
                 o_coef = G.spectral ? cv.take<double>(G.dims[0] + G.dims[1] + G.dims[2]) : 0;
    const size_t o_flags = nper == 1 ? cv.take<int>(nlines) : 0;
    // the potential: G_k(p), dq0/dn, dq0/dgrad n, the slot map, A and U on the grid, and
    // the spectral divergence
    const size_t o_G = pot ? cv.take<double>(static_cast<size_t>(kMaxNodes) * ngroup) : 0,
                 o_qn = pot ? cv.take<double>(G.N) : 0, o_qg = pot ? cv.take<double>(3 * G.N) : 0,
                 o_slot = pot ? cv.take<int>(G.N) : 0, o_A = pot ? cv.take<double>(G.N) : 0,
                 o_U = pot ? cv.take<double>(G.N) : 0, o_div = (pot && G.spectral) ? cv.take<double>(G.N) : 0;
    unsigned char *base = nullptr;
    if (scratch_malloc_async(reinterpret_cast<void **>(&base), cv.off, st) != cudaSuccess) return VDWDF_EALLOC;
    double *Gk = pot ? reinterpret_cast<double *>(base + o_G) : nullptr;
    double *qn = pot ? reinterpret_cast<double *>(base + o_qn) : nullptr;
    double *qgr = pot ? reinterpret_cast<double *>(base + o_qg) : nullptr;
    int *slot = pot ? reinterpret_cast<int *>(base + o_slot) : nullptr;
    double *Ad = pot ? reinterpret_cast<double *>(base + o_A) : nullptr;
    double *Ud = pot ? reinterpret_cast<double *>(base + o_U) : nullptr;
    double *divb = (pot && G.spectral) ? reinterpret_cast<double *>(base + o_div) : nullptr;
    double *q0 = reinterpret_cast<double *>(base + o_q0);
    unsigned long long *mm = reinterpret_cast<unsigned long long *>(base + o_mm);
    double *F = reinterpret_cast<double *>(base + o_F), *Tk = reinterpret_cast<double *>(base + o_Tk);
    double *Tout = reinterpret_cast<double *>(base + o_out);
    double *gsp = G.spectral ? reinterpret_cast<double *>(base + o_gsp) : nullptr;
    double *coef = G.spectral ? reinterpret_cast<double *>(base + o_coef) : nullptr;
    int *flags = nper == 1 ? reinterpret_cast<int *>(base + o_flags) : nullptr;
    unsigned char *lbase = nullptr;  // one periodic axis: the lines' buffers
    Timer tm;
    unsigned long long hmm[3] = {0, 0, 0};
    double T = 0.0;
    int nodes = 0, groups = np;
    auto body = [&]() -> int {
        tm.mark(0, st);
        const double *g_use = nullptr;
        int r = q0_gradient(G, n_dev, grad_dev, gsp, coef, &g_use, st);
        if (r) return r;
        r = launch_grad_q0(G.dims, G.am, n_dev, g_use, q0, qn, qgr, st);
        if (r) return r;
        if (pot) VDWDF_CUDA_TRY(cudaMemsetAsync(v_dev, 0, sizeof(double) * G.N, st));
        VDWDF_CUDA_TRY(cudaMemsetAsync(mm, 0xFF, sizeof(unsigned long long), st));
        VDWDF_CUDA_TRY(cudaMemsetAsync(mm + 1, 0, 2 * sizeof(unsigned long long), st));
        r = launch_diag_range(G.N, n_dev, q0, n_cut, mm, st);
        if (r) return r;
        VDWDF_CUDA_TRY(cudaMemcpyAsync(hmm, mm, sizeof(hmm), cudaMemcpyDeviceToHost, st));
        VDWDF_CUDA_TRY(cudaStreamSynchronize(st));
        if (hmm[2] == 0) return VDWDF_OK;  // no active point: T = 0 and v = 0
        double qmin, qmax;
        std::memcpy(&qmin, &hmm[0], 8);
        std::memcpy(&qmax, &hmm[1], 8);
        if (!(qmin > 0.0) || !std::isfinite(qmax)) return VDWDF_EINVAL;
        // nodes x_k = x0 + k hx of int_0^inf e^{-c s} ds = int e^{-c e^x} e^x dx over
        // c = u_i + u_j in [2 umin, 2 umax]: the part below x0 is under 1e-17 of 1/c
        // for every c, e^{-c e^x} has fallen below e^-45 past the last node, and the
        // step's error (exp(-pi^2 / hx) up to a factor) measures 1.2e-13 relative for
        // 1/c and 2.5e-12 for 1/c^2 (the potential's second sum) over that range
        const double umin = qmin * qmin, umax = qmax * qmax, hx = 0.3;
        const double x0 = std::log(1e-17 / (2.0 * umax)), x1 = std::log(45.0 / (2.0 * umin));
        nodes = static_cast<int>(std::ceil((x1 - x0) / hx)) + 1;
        if (nodes > kMaxNodes) return VDWDF_EUNSUPPORTED;
        const double Cas = 12.0 * std::pow(4.0 * kPi / 9.0, 3);
        const double scale = -0.5 * G.dV * G.dV * Cas;
        const int *line_slot = nullptr;
        double *Gl = Gk;
        if (nper == 1) {
            // the lines along the periodic axis that hold an active point
            VDWDF_CUDA_TRY(cudaMemsetAsync(flags, 0, sizeof(int) * nlines, st));
            r = launch_far_tail_line_flags(G.dims, ax, n_dev, n_cut, flags, st);
            if (r) return r;
            std::vector<int> hf(nlines), list, lslot(nlines, -1);
            VDWDF_CUDA_TRY(cudaMemcpyAsync(hf.data(), flags, sizeof(int) * nlines, cudaMemcpyDeviceToHost, st));
            VDWDF_CUDA_TRY(cudaStreamSynchronize(st));
            for (int l = 0; l < nlines; ++l)
                if (hf[l]) {
                    lslot[l] = static_cast<int>(list.size());
                    list.push_back(l);
                }
            const int La = static_cast<int>(list.size());
            if (La < 1) return VDWDF_EINVAL;  // active points counted above, so not reached
            if (La > kMaxLines) return VDWDF_EUNSUPPORTED;
            groups = La;
            const int Nb = nlines / Nc;
            Carve lc;
            const size_t o_list = lc.take<int>(La), o_lslot = lc.take<int>(nlines),
                         o_lF = lc.take<double>(static_cast<size_t>(nodes) * La),
                         o_lG = lc.take<double>(static_cast<size_t>(nodes) * La),
                         o_Kt = lc.take<double>(static_cast<size_t>(Nb) * (2 * Nc - 1));
            if (scratch_malloc_async(reinterpret_cast<void **>(&lbase), lc.off, st) != cudaSuccess) return VDWDF_EALLOC;
            int *dlist = reinterpret_cast<int *>(lbase + o_list);
            int *dlslot = reinterpret_cast<int *>(lbase + o_lslot);
            double *lF = reinterpret_cast<double *>(lbase + o_lF), *lG = reinterpret_cast<double *>(lbase + o_lG);
            double *Kt = reinterpret_cast<double *>(lbase + o_Kt);
            VDWDF_CUDA_TRY(cudaMemcpyAsync(dlist, list.data(), sizeof(int) * La, cudaMemcpyHostToDevice, st));
            VDWDF_CUDA_TRY(cudaMemcpyAsync(dlslot, lslot.data(), sizeof(int) * nlines, cudaMemcpyHostToDevice, st));
            r = launch_far_tail_lines(G.dims, ax, La, dlist, n_dev, q0, n_cut, x0, hx, nodes, gbb, gbc, gcc, r_cut,
                                      pref, scale, lF, Kt, lG, Tk, Tout, st);
            if (r) return r;
            line_slot = dlslot;
            Gl = lG;
            // the host vectors are read by the copies above before they are freed: the
            // copies from pageable memory return once the data is staged
        } else {
            r = launch_far_tail(G.dims, ax, np, n_dev, q0, n_cut, x0, hx, nodes, dz, r_cut, c2, c3, scale, F, Tk,
                                Gk, Tout, st);
            if (r) return r;
        }
        if (pot) {
            r = launch_far_tail_AU(G.dims, ax, groups, line_slot, n_dev, q0, n_cut, x0, hx, nodes, Gl, Cas, slot, Ad,
                                   Ud, st);
            if (r) return r;
            r = assemble_v(G, slot, Ad, Ud, qn, qgr, gsp, divb, coef, v_dev, nullptr, nullptr, st);
            if (r) return r;
        }
        tm.mark(1, st);
        VDWDF_CUDA_TRY(cudaMemcpyAsync(&T, Tout, sizeof(double), cudaMemcpyDeviceToHost, st));
        VDWDF_CUDA_TRY(cudaStreamSynchronize(st));
        if (!std::isfinite(T)) return VDWDF_EINVAL;  // a non-finite density (as vdwdf_energy)
        return VDWDF_OK;
    };
    rc = body();
    if (lbase) cudaFreeAsync(lbase, st);
    cudaFreeAsync(base, st);
    if (rc == VDWDF_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = VDWDF_ECUDA;
    if (rc) return rc;
    std::memset(out, 0, sizeof(*out));
    out->T = T;
    out->n_active = static_cast<int64_t>(hmm[2]);
    out->nodes = nodes;
    out->planes = groups;
    if (hmm[2]) out->ms = tm.ms(0, 1);
    out->launches = static_cast<int32_t>(g_launches.load() - launches0);
    return VDWDF_OK;
}

int vdwdf_diag_voxel(const vdwdf_grid *grid, const double *n_dev, const double *grad_dev, double n_cut,
                     const vdwdf_table *table, int nphi0, vdwdf_diag_result *out, void *cuda_stream) {
    return vdwdf::diag_voxel(grid, n_dev, grad_dev, n_cut, table, nphi0, nullptr, out, cuda_stream);
}

int vdwdf_diag_voxel_potential(const vdwdf_grid *grid, const double *n_dev, double n_cut,
                               const vdwdf_table *table, int nphi0, double *dv_dev, vdwdf_diag_result *out,
                               void *cuda_stream) {
    if (!dv_dev) return VDWDF_EINVAL;
    return vdwdf::diag_voxel(grid, n_dev, nullptr, n_cut, table, nphi0, dv_dev, out, cuda_stream);
}

int vdwdf_energy(const vdwdf_grid *grid, const double *n_dev, const double *grad_dev, double n_cut,
                 double r_cut, const vdwdf_table *table, int precision, const vdwdf_tuning *tuning,
                 vdwdf_result *out, void *cuda_stream) {
    return run_single(grid, n_dev, grad_dev, n_cut, r_cut, table, precision, tuning, false, nullptr,
                      nullptr, nullptr, out, cuda_stream);
}

int vdwdf_potential(const vdwdf_grid *grid, const double *n_dev, double n_cut, double r_cut,
                    const vdwdf_table *table, int precision, const vdwdf_tuning *tuning, double *v_dev,
                    double *A_dev, double *U_dev, vdwdf_result *out, void *cuda_stream) {
    return run_single(grid, n_dev, nullptr, n_cut, r_cut, table, precision, tuning, true, v_dev, A_dev,
                      U_dev, out, cuda_stream);
}

int vdwdf_energy_batched(int ninst, const vdwdf_grid *grids, const double *const *n_dev, double n_cut,
                         double r_cut, const vdwdf_table *table, int precision,
                         const vdwdf_tuning *tuning, double *E_out, vdwdf_result *out,
                         void *cuda_stream) {
    if (ninst < 1 || ninst > 4096 || !grids || !n_dev || !E_out) return VDWDF_EINVAL;
    if (!table) return VDWDF_ENOTABLE;
    if (precision != VDWDF_FP32 && precision != VDWDF_FP64) return VDWDF_EINVAL;
    std::vector<Geom> geo(ninst);
    for (int k = 0; k < ninst; ++k) {
        int rc = check_grid(&grids[k], geo[k]);
        if (rc) return rc;
        rc = check_cut(n_cut, r_cut, geo[k]);
        if (rc) return rc;
        if (!n_dev[k]) return VDWDF_EINVAL;
        rc = check_tuning(tuning, geo[k].skew, true);
        if (rc) return rc;
    }
    const bool tune_auto = tuning && tuning->threads == VDWDF_TUNE_AUTO;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    double *d64 = nullptr;
    float *d32 = nullptr;
    int rc = table_on_device(table, &d64, &d32);
    if (rc) return rc;
    int dev = 0;
    VDWDF_CUDA_TRY(cudaGetDevice(&dev));
    // signature of the recorded graph: everything the recording bakes in -- inputs,
    // shapes, the whole cell, periodicity, gradient kind, cutoffs, the table (its
    // generation and device copies), precision and tuning
    std::vector<uintptr_t> key;
    key.push_back(static_cast<uintptr_t>(dev));
    key.push_back(static_cast<uintptr_t>(ninst));
    key.push_back(static_cast<uintptr_t>(table->gen));
    key.push_back(reinterpret_cast<uintptr_t>(d64));
    key.push_back(reinterpret_cast<uintptr_t>(d32));
    key.push_back(static_cast<uintptr_t>(precision));
    uint64_t bits;
    std::memcpy(&bits, &n_cut, 8);
    key.push_back(static_cast<uintptr_t>(bits));
    std::memcpy(&bits, &r_cut, 8);
    key.push_back(static_cast<uintptr_t>(bits));
    if (tuning) {
        key.push_back(static_cast<uintptr_t>(tuning->threads));
        key.push_back(static_cast<uintptr_t>(tuning->items_per_sm));
        key.push_back(static_cast<uintptr_t>(static_cast<uint32_t>(tuning->smem_rows)));
        key.push_back(static_cast<uintptr_t>(static_cast<uint32_t>(tuning->smem_row0)));
    }
    for (int k = 0; k < ninst; ++k) {
        key.push_back(reinterpret_cast<uintptr_t>(n_dev[k]));
        key.push_back(static_cast<uintptr_t>(static_cast<uint32_t>(grids[k].gradient)));
        for (int a = 0; a < 3; ++a) {
            key.push_back(static_cast<uintptr_t>(grids[k].n[a]));
            key.push_back(static_cast<uintptr_t>(grids[k].periodic[a]));
            for (int b = 0; b < 3; ++b) {
                std::memcpy(&bits, &grids[k].cell[a][b], 8);
                key.push_back(static_cast<uintptr_t>(bits));
            }
        }
    }
    const long long launches0 = g_launches.load();
    std::lock_guard<std::mutex> lk(g_batch_mu);
    BatchPlan *bp = nullptr;
    vdwdf_tuning tuned = {0, 0, 0, 0};
    const vdwdf_tuning *use = tune_auto ? nullptr : tuning;
    auto it = g_batches.find(key);
    if (it != g_batches.end()) {
        bp = it->second;
    } else {
        // make room: the least recently used plan goes (no replay of it is in
        // flight: every batched call synchronises its stream before releasing the lock)
        while (g_batches.size() >= kMaxPlans) {
            auto old = g_batches.begin();
            for (auto jt = g_batches.begin(); jt != g_batches.end(); ++jt)
                if (jt->second->last_use < old->second->last_use) old = jt;
            destroy_plan(old->second);
            g_batches.erase(old);
        }
        bp = new (std::nothrow) BatchPlan;
        if (!bp) return VDWDF_EALLOC;
        bp->device = dev;
        bp->table_gen = table->gen;
        bp->geo = geo;
        bp->work.resize(ninst);
        const int ngroups = (ninst + kMaxInst - 1) / kMaxInst;
        for (int k = 0; k < ninst; ++k) {
            int *order = nullptr, nb = 0;
            rc = brick_order(geo[k].dims, &order, &nb);
            if (rc) {
                delete bp;
                return rc;
            }
            const size_t bytes = layout(geo[k], nb, false, precision == VDWDF_FP64, nullptr, nullptr);
            unsigned char *b = nullptr;
            if (scratch_malloc(reinterpret_cast<void **>(&b), bytes) != cudaSuccess) {
                delete bp;
                return VDWDF_EALLOC;
            }
            bp->bufs.push_back(b);
            layout(geo[k], nb, false, precision == VDWDF_FP64, &bp->work[k], b);
        }
        if (scratch_malloc(reinterpret_cast<void **>(&bp->queues), sizeof(unsigned int) * ngroups) != cudaSuccess) {
            delete bp;
            return VDWDF_EALLOC;
        }
        for (int g = 0; g < ngroups; ++g) {
            const int k0 = g * kMaxInst, k1 = std::min(ninst, k0 + kMaxInst);
            long long gsum = 0;
            bool gskew = false;
            for (int k = k0; k < k1; ++k) {
                gsum += geo[k].N;
                gskew = gskew || geo[k].skew;
            }
            // room for one partial per work item of the shape used (of any candidate
            // shape when the autotuner runs; items past the room would go atomically)
            long long items = 0;
            for (int ci = 0; ci < (tune_auto ? kTuneCount : 1); ++ci) {
                const vdwdf_tuning *t = tune_auto ? &kTuneCandidates[ci] : use;
                const Launch ln = choose_launch(precision, false, t, table, std::max<long long>(1, gsum / (k1 - k0)),
                                                gskew, k1 - k0);
                long long it = 0;
                for (int k = k0; k < k1; ++k) it += pair_items(geo[k].N, ln.jt);
                items = std::max(items, it);
            }
            double *b = nullptr;
            if (scratch_malloc(reinterpret_cast<void **>(&b), sizeof(double) * std::max<long long>(items, 1)) != cudaSuccess) {
                delete bp;
                return VDWDF_EALLOC;
            }
            bp->item_bufs.push_back(b);
            bp->item_caps.push_back(items);
        }
        // VDWDF_TUNE_AUTO: the autotuner times every candidate shape on this very
        // batch (the whole pass, uncaptured, on the caller's stream, twice; the
        // second run counts) and the fastest is recorded.  The energy-mode default
        // is a candidate, so the choice is never slower than it by more than noise.
        if (tune_auto) {
            Timer tt;
            double best_ms = -1.0;
            for (int ci = 0; ci < kTuneCount && rc == VDWDF_OK; ++ci) {
                const vdwdf_tuning &cd = kTuneCandidates[ci];
                if (precision == VDWDF_FP64 && cd.smem_rows != 0) continue;
                bool ok = true;
                for (int k = 0; k < ninst; ++k) ok = ok && check_tuning(&cd, geo[k].skew) == VDWDF_OK;
                if (!ok) continue;
                for (int rep = 0; rep < 2 && rc == VDWDF_OK; ++rep) {
                    tt.mark(0, st);
                    rc = record_batch(*bp, ninst, n_dev, n_cut, table, precision, &cd, d64, d32, st);
                    tt.mark(1, st);
                    if (rc == VDWDF_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = VDWDF_ECUDA;
                }
                const double ms = tt.ms(0, 1);
                if (rc == VDWDF_OK && ms > 0.0 && (best_ms < 0.0 || ms < best_ms)) {
                    best_ms = ms;
                    tuned = cd;
                }
            }
            if (rc != VDWDF_OK) {
                delete bp;
                return rc;
            }
            use = &tuned;
            bp->tuned = tuned;
        }
        // record the whole batch into a graph on a private stream
        cudaStream_t cs = nullptr;
        if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
            delete bp;
            return VDWDF_ECUDA;
        }
        const long long l0 = g_launches.load();
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            rc = record_batch(*bp, ninst, n_dev, n_cut, table, precision, use, d64, d32, cs);
            e = cudaStreamEndCapture(cs, &graph);
        }
        if (e == cudaSuccess && rc == VDWDF_OK) e = cudaGraphInstantiate(&bp->exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        cudaStreamDestroy(cs);
        bp->launches_per_replay = static_cast<int>(g_launches.load() - l0);
        g_launches.fetch_sub(bp->launches_per_replay);  // recorded, not launched
        if (e != cudaSuccess || rc != VDWDF_OK) {
            if (e != cudaSuccess) note_cuda_error(e, "graph capture", __FILE__, __LINE__);
            delete bp;
            return rc != VDWDF_OK ? rc : VDWDF_ECUDA;
        }
        g_batches[key] = bp;
    }
    bp->last_use = ++g_batch_clock;
    Timer tm;
    tm.mark(0, st);
    VDWDF_CUDA_TRY(cudaGraphLaunch(bp->exec, st));
    count_launches(bp->launches_per_replay);
    tm.mark(1, st);
    std::vector<Stats> hs(ninst);
    for (int k = 0; k < ninst; ++k)
        VDWDF_CUDA_TRY(cudaMemcpyAsync(&hs[k], bp->work[k].stats, sizeof(Stats), cudaMemcpyDeviceToHost, st));
    VDWDF_CUDA_TRY(cudaStreamSynchronize(st));
    int status = VDWDF_OK;
    vdwdf_result tot;
    std::memset(&tot, 0, sizeof(tot));
    for (int k = 0; k < ninst; ++k) {
        vdwdf_result r;
        fill_result(hs[k], bp->geo[k], table, &r);
        E_out[k] = r.E;
        tot.E += r.E;
        tot.E_diag += r.E_diag;
        tot.n_active += r.n_active;
        tot.pairs += r.pairs;
        tot.pairs_evaluated += r.pairs_evaluated;
        tot.n_clamped += r.n_clamped;
        if (hs[k].guard_trips) status = VDWDF_ETIMEOUT;
    }
    if (out) {
        *out = tot;
        out->ms_pairs = tm.ms(0, 1);
        out->launches = static_cast<int32_t>(g_launches.load() - launches0);
        out->smem_row0 = precision == VDWDF_FP32 ? (bp->row0 >= 0 ? bp->row0 : hs[0].band_row0) : -1;
        out->pair_threads = bp->threads;
    }
    return status;
}

int vdwdf_autotune(const vdwdf_grid *grid, const double *n_dev, double n_cut, double r_cut,
                   const vdwdf_table *table, int precision, vdwdf_tuning *best, void *cuda_stream) {
    if (!best) return VDWDF_EINVAL;
    Geom G;
    int rc = check_grid(grid, G);
    if (rc) return rc;
    rc = check_cut(n_cut, r_cut, G);
    if (rc) return rc;
    if (!n_dev) return VDWDF_EINVAL;
    if (!table) return VDWDF_ENOTABLE;
    if (precision != VDWDF_FP32 && precision != VDWDF_FP64) return VDWDF_EINVAL;
    return autotune_one(G, n_dev, n_cut, table, precision, best, static_cast<cudaStream_t>(cuda_stream));
}

}  // extern "C"

// ---------------------------------------------------------------------------
// The energy without any allocation: all scratch of one call lives in a
// static device array of the library.
// ---------------------------------------------------------------------------
namespace vdwdf {
namespace {

constexpr long long kNoAllocMaxPoints = 65536;       // grid points per call
constexpr int kNoAllocMaxBricks = 65536;             // 4x4x4 bricks per call
constexpr size_t kNoAllocBytes = size_t(8) << 20;    // 8 MiB
constexpr int kNoAllocMaxDevices = 64;

// One per device (module static data); cleared where needed by each call.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mu;  // held for a whole call: calls never overlap in a process
unsigned char *g_noalloc_addr[kNoAllocMaxDevices] = {};
std::pair<uint64_t, int> g_noalloc_keys[kNoAllocMaxBricks];  // host staging, no heap
int g_noalloc_order[kNoAllocMaxBricks];

size_t round256(size_t b) { return (b + 255) & ~static_cast<size_t>(255); }

// Device address of the static scratch, looked up once per device.
int noalloc_base(unsigned char **p) {
    int dev = 0;
    VDWDF_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocMaxDevices) return VDWDF_EUNSUPPORTED;
    if (!g_noalloc_addr[dev]) {
        void *a = nullptr;
        VDWDF_CUDA_TRY(cudaGetSymbolAddress(&a, g_noalloc_scratch));
        g_noalloc_addr[dev] = static_cast<unsigned char *>(a);
    }
    *p = g_noalloc_addr[dev];
    return VDWDF_OK;
}

// The table's device copies if they already exist on the current device.
int table_resident(const vdwdf_table *tc, double **d64, float **d32) {
    vdwdf_table *t = const_cast<vdwdf_table *>(tc);
    int dev = 0;
    VDWDF_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(t->mu);
    auto it = t->dev.find(dev);
    if (it == t->dev.end()) return VDWDF_ENOTABLE;
    *d64 = it->second.first;
    *d32 = it->second.second;
    return VDWDF_OK;
}

long long brick_count(const int dims[3]) {
    return static_cast<long long>((dims[0] + kBrick - 1) / kBrick) * ((dims[1] + kBrick - 1) / kBrick) *
           ((dims[2] + kBrick - 1) / kBrick);
}

// The Morton order of the bricks (as brick_order), built in host statics and
// copied to order_dev on the stream.
int noalloc_order(const int dims[3], int *order_dev, cudaStream_t st) {
    const int bx = (dims[0] + kBrick - 1) / kBrick, by = (dims[1] + kBrick - 1) / kBrick,
              bz = (dims[2] + kBrick - 1) / kBrick;
    const int n = bx * by * bz;
    for (int x = 0; x < bx; ++x)
        for (int y = 0; y < by; ++y)
            for (int z = 0; z < bz; ++z) {
                const int id = (x * by + y) * bz + z;
                g_noalloc_keys[id] = {spread3(x) << 2 | spread3(y) << 1 | spread3(z), id};
            }
    std::sort(g_noalloc_keys, g_noalloc_keys + n);
    for (int i = 0; i < n; ++i) g_noalloc_order[i] = g_noalloc_keys[i].second;
    VDWDF_CUDA_TRY(cudaMemcpyAsync(order_dev, g_noalloc_order, sizeof(int) * n, cudaMemcpyHostToDevice, st));
    return VDWDF_OK;
}

}  // namespace
}  // namespace vdwdf

extern "C" {

int vdwdf_energy_noalloc(const vdwdf_grid *grid, const double *n_dev, const double *grad_dev,
                         double n_cut, double r_cut, const vdwdf_table *table, int precision,
                         vdwdf_result *out, void *cuda_stream) {
    using namespace vdwdf;
    Geom G;
    int rc = check_grid(grid, G);
    if (rc) return rc;
    rc = check_cut(n_cut, r_cut, G);
    if (rc) return rc;
    if (!n_dev) return VDWDF_EINVAL;
    if (!table) return VDWDF_ENOTABLE;
    if (precision != VDWDF_FP32 && precision != VDWDF_FP64) return VDWDF_EINVAL;
    // size limits, checked before any device work
    if (G.N > kNoAllocMaxPoints) return VDWDF_EUNSUPPORTED;
    const long long nbl = brick_count(G.dims);
    if (nbl > kNoAllocMaxBricks) return VDWDF_EUNSUPPORTED;
    const int nb = static_cast<int>(nbl);
    const bool fp64 = precision == VDWDF_FP64;
    const size_t o_order = round256(layout(G, nb, false, fp64, nullptr, nullptr));
    const size_t o_items = o_order + round256(sizeof(int) * nb);
    if (o_items + 256 * sizeof(double) > kNoAllocBytes) return VDWDF_EUNSUPPORTED;
    const unsigned int item_space = static_cast<unsigned int>((kNoAllocBytes - o_items) / sizeof(double));

    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const long long launches0 = g_launches.load();
    // the call proper; every return of it, error or not, is followed by the stream
    // synchronisation below, so that nothing of this call is still queued on the
    // shared array when the lock is released
    auto run = [&]() -> int {
        double *d64 = nullptr;
        float *d32 = nullptr;
        rc = table_resident(table, &d64, &d32);
        if (rc) return rc;
        unsigned char *base = nullptr;
        rc = noalloc_base(&base);
        if (rc) return rc;
        Work w;
        layout(G, nb, false, fp64, &w, base);
        int *order_dev = reinterpret_cast<int *>(base + o_order);
        double *item_E = reinterpret_cast<double *>(base + o_items);

        // as vdwdf_energy: gradient, q0, trimming and tiles, then the pair sum with
        // one partial per work item summed in a fixed order
        rc = noalloc_order(G.dims, order_dev, st);
        if (rc) return rc;
        rc = reset_stats(w.stats, st);  // counters start at zero (q0 minimum above all floats)
        if (rc) return rc;
        const double *g_use = nullptr;
        rc = q0_gradient(G, n_dev, grad_dev, w.gsp, w.coef, &g_use, st);
        if (rc) return rc;
        rc = launch_grad_q0(G.dims, G.am, n_dev, g_use, w.q0, w.qn, w.qg, st);
        if (rc) return rc;
        rc = launch_compact(G.dims, n_dev, n_cut, w.q0, order_dev, nb, w.cnt, w.off, nullptr, w.p32, w.n32,
                            w.p64, w.n64, w.blo, w.bhi, w.stats, st);
        if (rc) return rc;
        if (G.skew) {
            rc = launch_tiles_cart(w.p32, w.stats, G.vrow, w.clo, w.chi, G.N, st);
            if (rc) return rc;
        }
        Stats hs;
        std::memset(&hs, 0, sizeof(hs));
        VDWDF_CUDA_TRY(cudaMemcpyAsync(&hs, w.stats, sizeof(Stats), cudaMemcpyDeviceToHost, st));
        VDWDF_CUDA_TRY(cudaStreamSynchronize(st));
        int row0 = 0, threads = 0;
        if (hs.n_active > 0) {
            Launch ln = choose_launch(precision, false, nullptr, table, hs.n_active, G.skew);
            row0 = ln.ks0;
            threads = ln.threads;
            VDWDF_CUDA_TRY(cudaMemsetAsync(w.queue, 0, sizeof(unsigned int), st));  // work-queue head
            PairLaunch pl;
            std::memset(&pl, 0, sizeof(pl));
            const long long items = pair_items(hs.n_active, ln.jt);
            if (items > 0xFFFFFFF0LL) return VDWDF_EINVAL;
            fill_shared(table, d64, d32, ln, w.queue, static_cast<unsigned int>(items + 2), pl.sh);
            // every item below item_cap writes its partial; any beyond it are added atomically
            pl.sh.item_E = item_E;
            pl.sh.item_cap = static_cast<unsigned int>(std::min<long long>(items, item_space));
            pl.ninst = 1;
            fill_params(G, w, pl.inst[0]);
            if (ln.ks0 < 0) {
                rc = launch_band_choose(pl, w.hist, st);
                if (rc) return rc;
            }
            rc = launch_pair(precision, false, G.skew, ln.threads, pl, ln.nctas, st);
            if (rc) return rc;
            rc = launch_reduce_items(pl, st);
            if (rc) return rc;
        }
        VDWDF_CUDA_TRY(cudaMemcpyAsync(&hs, w.stats, sizeof(Stats), cudaMemcpyDeviceToHost, st));
        VDWDF_CUDA_TRY(cudaStreamSynchronize(st));
        if (hs.guard_trips) return VDWDF_ETIMEOUT;
        if (out) {
            std::memset(out, 0, sizeof(*out));
            fill_result(hs, G, table, out);
            out->launches = static_cast<int32_t>(g_launches.load() - launches0);
            out->smem_row0 = precision == VDWDF_FP32 ? (row0 >= 0 ? row0 : hs.band_row0) : -1;
            out->pair_threads = threads;
        }
        return VDWDF_OK;
    };
    const int status = run();
    const cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        note_cuda_error(e, "cudaStreamSynchronize", __FILE__, __LINE__);
        return status != VDWDF_OK ? status : VDWDF_ECUDA;
    }
    return status;
}

}  // extern "C"
