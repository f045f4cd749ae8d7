// Internal declarations shared by the libvdwdf translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "vdwdf.h"

namespace vdwdf {

#define VDWDF_CUDA_TRY(expr)                                                   \
    do {                                                                       \
        cudaError_t err__ = (expr);                                            \
        if (err__ != cudaSuccess) {                                            \
            ::vdwdf::note_cuda_error(err__, #expr, __FILE__, __LINE__);        \
            return VDWDF_ECUDA;                                                \
        }                                                                      \
    } while (0)

void note_cuda_error(cudaError_t e, const char *what, const char *file, int line);
void count_launches(int n);

constexpr int kTile = 32;               // points per tile: one warp's i set, one staged j tile
constexpr int kBrick = 4;               // 4 x 4 x 4 grid bricks order the active list
constexpr int kMaxSmemBytes = 232448;   // 227 KiB opt-in shared memory per block (cc 10.x)
constexpr int kMaxInst = 24;            // instances per pair-kernel launch

// FP64 point record (x, y, z in grid index units, q0).
struct __align__(32) dvec4 {
    double x, y, z, w;
};

// Device-side counters of one instance (zeroed before use).
struct Stats {
    double E_pair;             // sum over ordered pairs of n_i n_j phi (self term included)
    double n2sum;              // sum over active points of n^2
    unsigned long long pairs;  // ordered pair interactions other than the self term
    unsigned long long evals;  // pair evaluations done
    unsigned long long clamped;
    unsigned int guard_trips;  // work loops that hit their iteration cap
    unsigned int qmin_bits, qmax_bits;  // q0 range of active points (FP32 bits; q0 > 0)
    int n_active;
    int band_row0;             // FP32 pair kernel: first table row of the shared band when
                               // chosen on the device (the first instance of a launch)
};

// Derivatives along the grid axes to Cartesian components: the gradient is
// g_c = sum_a S[3a + c] (8 (f_{+1} - f_{-1}) - (f_{+2} - f_{-2}))_a with
// S[3a + c] = N_a B_a[c] / 12, B_a the reciprocal rows of the cell (B_a . M_b =
// delta_ab).  On a diagonal cell S[4a] = (1/h_a)/12, the rest 0, and general = 0.
struct AxisMap {
    double S[9];
    int general;
};

// Rows v_a = M_a / N_a of a general cell (float): grid point (i, j, k) sits at
// i v_0 + j v_1 + k v_2.
struct CellRows {
    float v[9];
};

// Per-instance inputs of the pair kernel.
struct PairParams {
    double h2[3];        // metric in index units, diagonal: |M_a|^2 / N_a^2
    double g2x[3];       // 2 x off-diagonal metric (01, 02, 12): r^2 = sum h2_a d_a^2
                         //   + g2x[0] d_0 d_1 + g2x[1] d_0 d_2 + g2x[2] d_1 d_2
    float cull_h2[3];    // culling metric: h2 on orthogonal cells, the smallest
                         //   eigenvalue of the metric on skewed ones (a lower bound)
    float rcm[3];        // cutoff extent in index units along each axis (widened)
    double rc2;          // squared cutoff times (1 + 1e-12): inside iff r^2 <= rc2
    int dims[3];
    int M[3];            // max |image index| per axis (0: not periodic)
    int use_cut;
    const float4 *p32;   // active points: x, y, z (index units), q0
    const float *n32;
    const dvec4 *p64;
    const double *n64;
    const float4 *blo, *bhi;  // bounding boxes of kTile-point tiles (index units)
    const float4 *clo, *chi;  // skewed cells: Cartesian bounding boxes of the tiles
    CellRows vrow;            // skewed cells: v_a = M_a / N_a
    double *A, *U;       // potential mode: per active point, accumulated
    Stats *stats;
};

// The pair loop's constants, computed on the host in the loop's own precision,
// so that the device reads them as they are (no conversion or division in the
// kernel that the compiler could repeat inside the loop).
template <typename R>
struct LoopConsts {
    R cD, cd;            // cells per unit of D (times 1/2: tD = r (q_i + q_j) cD) and of delta
    R tDmax, tDclamp;    // nD - 1, and the largest R below it (FP32) or nD - 1 (FP64)
    R tdmax, tdclamp;    // the same along delta
    R C;                 // 12 (4 pi / 9)^3 of eq. (17)
    R iDmax, om_rho0;    // 1 / Dmax; 1 - rho(0)
    int kmax, lmax;      // last cell index along D and delta
};

// Inputs shared by all instances of a launch.
struct PairShared {
    const double *tab64;  // (nD + 2) x (nd + 2) B-spline coefficients / 36, D outer,
    const float *tab32;   // then nd + 2 coefficients / 6 of rho(delta) (beyond-table factor)
    int S;                // row stride (nd + 2)
    int nD, nd;
    double cD, cd;        // tD = r (q_i + q_j) cD,  td = |q_i - q_j|/(q_i + q_j) cd
    double C_asym;
    double om_rho0;       // 1 - rho(0), rho(0) = phi(Dmax, 0) / phi17(Dmax, 0)
    LoopConsts<float> k32;   // the same constants for the FP32 ...
    LoopConsts<double> k64;  // ... and the FP64 pair loop
    int ks0, ksn;         // FP32: table rows [ks0, ks0 + ksn) resident in shared memory;
                          // ks0 < 0: ks0 is inst[0].stats->band_row0 (set by launch_band_choose)
    int jtiles_per_item;  // j tiles per work item
    unsigned int item_limit;  // process at most item_limit items (autotuning) ...
    unsigned int item_stride; // ... taking every item_stride-th one (1: all in order)
    unsigned int max_iters;   // cap on the work loop of one CTA
    unsigned int *queue;      // work-queue head (zeroed before launch)
    double *item_E;           // energy mode: one partial sum per work item (then reduced in
    unsigned int item_cap;    // a fixed order, so that E is reproducible bit for bit)
};

struct PairLaunch {
    PairShared sh;
    int ninst;
    PairParams inst[kMaxInst];
};

// Semilocal energies (LDA, PBE, revPBE): scratch of semilocal_scratch_doubles()
// doubles; the last six hold Ex_lda, Ec_lda, Ex_pbe, Ec_pbe, Ex_revpbe (sums of
// n eps, not yet times dV) and the number of points with n > 0.
int semilocal_scratch_doubles();
int launch_semilocal(const int dims[3], const AxisMap &am, const double *n, const double *grad_in,
                     double *scratch, cudaStream_t st);
// Cartesian bounding boxes of the tiles of a general cell (rows v_a = M_a / N_a).
int launch_tiles_cart(const float4 *p32, const Stats *stats, const CellRows &vrow, float4 *clo, float4 *chi,
                      long long n_max, cudaStream_t st);
// The 4th-order finite-difference gradient (Cartesian, 3 planes of N) of n.
int launch_gradient_fd(const int dims[3], const AxisMap &am, const double *n, double *grad, cudaStream_t st);
int launch_grad_q0(const int dims[3], const AxisMap &am, const double *n, const double *grad_in,
                   double *q0, double *dq0dn, double *dq0dg, cudaStream_t st);
int launch_compact(const int dims[3], const double *n, double n_cut, const double *q0,
                   const int *brick_order, int nbricks, int *brick_cnt, int *brick_off, int *slot,
                   float4 *p32, float *n32, dvec4 *p64, double *n64, float4 *blo, float4 *bhi,
                   Stats *stats, cudaStream_t st);
// skew: some instance has a non-diagonal metric (the kernel adds the cross terms)
int launch_pair(int precision, bool potential, bool skew, int threads, const PairLaunch &pl, int nctas,
                cudaStream_t st);
// Row stride of the shared-memory table band: odd, so that one column of
// consecutive rows falls in distinct banks.
__host__ __device__ inline int band_stride(int S) { return S | 1; }
int pair_smem_bytes(int precision, int threads, int ksn, int S);
// The shared band's first row from the pairs of a launch: a sampled histogram
// of the table's D cell over the (i, j, image) evaluations of every instance
// (kBandBins counters in hist), then the start whose ksn rows hold the most
// sampled stencils, written to inst[0].stats->band_row0.  Tables with more than
// kBandBins + 1 rows along D keep row 0.
constexpr int kBandBins = 1024;
int launch_band_choose(const PairLaunch &pl, unsigned int *hist, cudaStream_t st);
// Sum the energy-mode item partials of every instance in a fixed order into its
// Stats::E_pair (one block per instance).
int launch_reduce_items(const PairLaunch &pl, cudaStream_t st);
// Work items of an instance with n_active points and jt j tiles per item.
__host__ __device__ inline long long pair_items(long long n_active, int jt) {
    const long long nT = (n_active + kTile - 1) / kTile;
    return nT * ((nT + jt - 1) / jt);
}
// v = dV (chi (A + U dq0/dn) - div), div the divergence term: div_pre when given
// (the spectral gradient's, from launch_div_spectral), else the 4th-order stencil's.
int launch_assemble(const int dims[3], const AxisMap &am, double dV, const int *slot,
                    const double *A, const double *U, const double *dq0dn, const double *dq0dg,
                    const double *div_pre, double *v, double *A_grid, double *U_grid, cudaStream_t st);
// Reciprocal rows of the cell, B[3a + c] = (B_a)_c with B_a . M_b = delta_ab.
struct Recip {
    double B[9];
};
// The spectral (FFT) gradient: grad (3 planes of N, Cartesian) of n; coef holds
// N0 + N1 + N2 doubles of scratch.  VDWDF_EUNSUPPORTED beyond 12,800 points per axis.
int launch_gradient_spectral(const int dims[3], const Recip &R, const double *n, double *grad, double *coef,
                             cudaStream_t st);
// The divergence term of the potential with the spectral gradient:
// div = sum_a D_a W_a, W_a = sum_c (B_a)_c U dq0/dg_c (0 at inactive points), so
// that v = dV (chi (A + U dq0/dn) - div).  W: 3 planes of N scratch.
int launch_div_spectral(const int dims[3], const Recip &R, const int *slot, const double *U, const double *qg,
                        double *W, double *div, double *coef, cudaStream_t st);
int launch_energy_from_A(int n_max, const double *A, const double *n64, Stats *stats,
                         cudaStream_t st);
// Voxel-averaged diagonal: voxel rows v (M_a / N_a), the small-D model below D1
// and the tensor rule (nn nodes per axis on [0, 1]; xw = nodes then weights).
struct Phi0Rule {
    double v[9];
    double D1, psi0, c2;
    int nn;
};
// part: 8 nq doubles of scratch (one per q and sign octant)
int launch_phi0(const PairShared &sh, const Phi0Rule &rule, int nq, const double *q, const double *xw,
                double *part, double *out, cudaStream_t st);
// Grid passes of the diagonal: q0 range and count of the points with n >= n_cut
// (mm[0] = min bits, mm[1] = max bits of the positive doubles, mm[2] = count),
// then sums[0] = sum n^2 phi0(q0) (phi0 from the log-q table by 4-point
// Lagrange interpolation) and sums[1] = sum n^2, one pair per block in part.
int launch_diag_range(long long N, const double *n, const double *q0, double n_cut,
                      unsigned long long *mm, cudaStream_t st);
int launch_diag_sum(long long N, const double *n, const double *q0, double n_cut, const double *tab,
                    int nq, double lnq0, double dlnq, double *part, double *sums, cudaStream_t st);
int launch_diag_AU(long long N, const double *n, const double *q0, double n_cut, const double *tab, int nq,
                   double lnq0, double dlnq, double phi00, int *slot, double *A, double *U, cudaStream_t st);
// The far field past the cutoff (tail.cu): planes of grid axis ax (np of them, or
// np = 1 for the whole cell), nodes of the trapezoidal rule x_k = x0 + k hx in
// ln s; F (nodes x np) and Tk (nodes) scratch; out = scale sum_k hx e^{x_k} Tk[k]
// with Tk[k] = sum_{p,p'} K(p, p') F_k(p) F_k(p'),
// K = c2 / max(rc, |p - p'| dz)^4 (np > 1) or c3 (np = 1).
// G (nodes x np, nullable) keeps G_k(p) = sum_{p'} K(p, p') F_k(p') for the potential.
int launch_far_tail(const int dims[3], int ax, int np, const double *n, const double *q0, double n_cut,
                    double x0, double hx, int nodes, double dz, double rc, double c2, double c3, double scale,
                    double *F, double *Tk, double *G, double *out, cudaStream_t st);
// One periodic axis ax: flags[ib * N_c + ic] = 1 for the lines along ax (b < c the
// other axes) that hold an active point (flags zeroed by the caller).
int launch_far_tail_line_flags(const int dims[3], int ax, const double *n, double n_cut, int *flags,
                               cudaStream_t st);
// One periodic axis: the same sums over the La active lines `lines` (line ids):
// F (nodes x La), K between lines (pref I(rho, x0), rho^2 from the index
// differences through gbb, gbc, gcc) as a table Kt (N_b x (2 N_c - 1)) over the
// index differences, G (nodes x La) = K F, Tk (nodes) and out as launch_far_tail.
int launch_far_tail_lines(const int dims[3], int ax, int La, const int *lines, const double *n, const double *q0,
                          double n_cut, double x0, double hx, int nodes, double gbb, double gbc, double gcc,
                          double rc, double pref, double scale, double *F, double *Kt, double *G, double *Tk,
                          double *out, cudaStream_t st);
// The far field's potential in the pair sum's adjoint form on the grid: A, U (N)
// at active points with slot[m] = m, slot[m] = -1 elsewhere (for launch_assemble).
// line_slot (one periodic axis; else NULL): the active-line index of every line,
// which then indexes G (np = La).
int launch_far_tail_AU(const int dims[3], int ax, int np, const int *line_slot, const double *n, const double *q0,
                       double n_cut, double x0, double hx, int nodes, const double *G, double C, int *slot,
                       double *A, double *U, cudaStream_t st);
int launch_kernel_eval(int precision, const PairShared &sh, int64_t npts, const double *r,
                       const double *qi, const double *qj, double *phi, double *rdphi,
                       cudaStream_t st);

}  // namespace vdwdf
