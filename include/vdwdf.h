/*
 * vdwdf.h -- C ABI of libvdwdf, a GB300 (sm_103a) implementation of the hot
 * path of the vdW-DF nonlocal correlation post-processing method of JuNoLo
 * (Lazic et al., arXiv 0810.2273).
 *
 * The method (paper section 2, eqs. (1)-(2)):
 *     E_c^nl = 1/2 sum_i sum_j n(r_i) phi(q0_i |r_i - r_j|, q0_j |r_i - r_j|) n(r_j) dV^2
 * over the points of a charge density on an equidistant grid whose density is
 * at least a cutoff (section 3, "trimming"), including the periodic images of
 * the cell for periodic problems (section 3, "repeated in space"), with the
 * kernel phi of Dion et al. (PRL 92, 246401, eq. 14) tabulated in the
 * variables D and delta (section 2) and its large-D asymptote (Dion eq. 17).
 * q0 follows Dion eqs. 11-12 (LDA correlation plus gradient-corrected
 * exchange, Zab = -0.8491) from n and |grad n|, with grad n by 4th-order
 * central finite differences along the grid axes or by FFT, the two options of
 * section 3 (vdwdf_grid.gradient), or given by the caller.
 *
 * Units: Hartree atomic units (bohr, Hartree) at the boundary, FP64.
 *
 * Conventions common to every entry point:
 *  - Return value: VDWDF_OK (0) on success, a negative VDWDF_E* code on
 *    failure; vdwdf_strerror() names it.  No C++ exception crosses the ABI.
 *    Invalid arguments are rejected on the host before any launch, and then
 *    no output is written.
 *  - Device pointers ("_dev") are ordinary CUDA global-memory pointers owned
 *    by the caller, on the current device; they must stay valid until the
 *    call returns.  Grids are row-major [n0][n1][n2] FP64.
 *  - cuda_stream is a cudaStream_t (NULL = legacy default stream).  All
 *    device work of a call is ordered on that stream.  Calls that return
 *    host results (vdwdf_result, E_out) synchronise that stream before
 *    returning; the others return without waiting.
 *  - Scratch device memory is taken with cudaMallocAsync on the call's stream
 *    and freed on it before return; the library owns it.
 *  - Fault injection for tests (host side only; no device fault is caused):
 *    with the environment variable VDWDF_FAIL_ALLOC=1 every scratch
 *    allocation fails (VDWDF_EALLOC); with VDWDF_MAX_ITERS=k the persistent
 *    pair kernels stop after k work items per CTA, as their iteration guard
 *    does, and the call returns VDWDF_ETIMEOUT.  The next call without them
 *    works as before.
 *  - vdwdf_energy and vdwdf_potential return VDWDF_EINVAL when the energy
 *    comes out non-finite (an Inf density value, or a NaN next to an active
 *    point).
 *  - Cells: the rows of vdwdf_grid.cell are the lattice vectors M_0, M_1,
 *    M_2 (section 2: equidistant grid, axes need not be orthogonal); grid
 *    point (i_0, i_1, i_2) sits at sum_a (i_a / n_a) M_a.  A singular cell is
 *    VDWDF_EINVAL.  On a non-diagonal cell the finite differences along each
 *    grid axis give d/du_a (u_a = i_a / n_a) and grad n = sum_a (d/du_a) B_a,
 *    with B_a the reciprocal rows (B_a . M_b = delta_ab); the pair sum uses
 *    the full metric.
 */
#ifndef VDWDF_H
#define VDWDF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VDWDF_VERSION 10000

/* status codes */
#define VDWDF_OK 0
#define VDWDF_EINVAL (-1)        /* bad argument: null pointer, size, value   */
#define VDWDF_EUNSUPPORTED (-2)  /* valid, but beyond what the entry point supports */
#define VDWDF_ECUDA (-3)         /* a CUDA runtime call failed                */
#define VDWDF_EALLOC (-4)        /* host or device allocation failed          */
#define VDWDF_ETIMEOUT (-5)      /* a device-side work loop hit its iteration cap */
#define VDWDF_ENOTABLE (-6)      /* table handle missing or of another size   */

/* arithmetic of the pair sum */
#define VDWDF_FP32 0  /* FP32 pair arithmetic and interpolation, FP64 accumulation */
#define VDWDF_FP64 1  /* FP64 throughout                                         */

/* How the library differentiates the density (section 3: the gradient comes
 * from an FFT, from real-space finite differences, or from the caller).  Both
 * treat every axis of the grid as periodic.
 *   VDWDF_GRAD_FD: 4th-order central differences along each grid axis,
 *     (n_{-2} - 8 n_{-1} + 8 n_{+1} - n_{+2})/12 per index step;
 *   VDWDF_GRAD_SPECTRAL: the band-limited (FFT) derivative along each grid axis:
 *     the discrete Fourier transform times 2 pi i m, m in (-N/2, N/2), with the
 *     Nyquist frequency of an even axis mapped to zero (the real part of the
 *     inverse transform), applied as its circulant matrix; axes up to 12800
 *     points.
 * Either gives d/du_a along the fractional coordinates, and grad n = sum_a
 * (d/du_a n) B_a with the reciprocal rows B_a.  The potential uses the transpose
 * of the same operator. */
#define VDWDF_GRAD_FD 0
#define VDWDF_GRAD_SPECTRAL 1

/* The grid: cell rows a, b, c in bohr (grid point (i,j,k) sits at
 * i/n0 a + j/n1 b + k/n2 c), points per axis, and per-axis periodicity
 * (section 2: "equidistant division in all three spatial dimensions";
 * Appendix A input: perx, pery, perz).  The density array is [n0][n1][n2].
 * gradient: VDWDF_GRAD_FD (0, the default of a zeroed struct) or
 * VDWDF_GRAD_SPECTRAL; other values are VDWDF_EINVAL. */
typedef struct {
    double cell[3][3];
    int32_t n[3];
    int32_t periodic[3];
    int32_t gradient;
} vdwdf_grid;

/* Opaque kernel table: phi on the node grid D_k = Dmax k/(nD-1),
 * delta_l = l/ndelta (section 2: the kernel as a function of D >= 0 and
 * 0 <= delta < 1; section 7: limits and divisions fixed by refinement), its
 * FP64 and FP32 cubic-spline coefficients, and their device copies.  Owned by
 * the library; free with vdwdf_table_free.
 * The kernel the pair sum uses:
 *  - 0 <= D <= Dmax: the tensor-product interpolating cubic spline of the
 *    nodes, zero slope at D = 0 and delta = 0, zero curvature at the last
 *    node of each axis;
 *  - D > Dmax: Dion eq. 17 times g = rho(delta*) + (1 - rho(0)) (1 - (Dmax/D)^2),
 *    delta* = max(0, 1 - min(d1, d2)/Dmax), with rho the cubic spline (same
 *    end conditions) of phi(Dmax, delta_l) / eq. 17 (Dmax, delta_l): the
 *    kernel is continuous at Dmax for every delta, and g tends to 1 (the
 *    kernel to eq. 17) as both d1 and d2 grow;
 *  - delta above the last node: the spline's linear continuation in delta
 *    (its curvature is zero there), counted in vdwdf_result.n_clamped. */
typedef struct vdwdf_table vdwdf_table;

/* Per-call report. */
typedef struct {
    double E;                /* E_c^nl, Hartree                                     */
    double E_diag;           /* self-term part, 1/2 dV^2 sum_i n_i^2 phi(0,0)       */
    int64_t n_active;        /* grid points with n >= n_cut                         */
    int64_t pairs;           /* ordered pair interactions (i, j, L) other than the
                                self term, within r_cut when r_cut > 0              */
    int64_t pairs_evaluated; /* lane slots run by the pair kernel: (i, j, image)
                                candidates left after culling, each unordered pair
                                once (i<->j folded), outside-cutoff tests included */
    int64_t n_clamped;       /* evaluations with delta past the last node (spline continued linearly) */
    double q0_min, q0_max;   /* over active points                                 */
    float ms_prep;           /* device time: gradient, q0, trimming, tiling        */
    float ms_pairs;          /* device time: pair kernel(s)                         */
    float ms_post;           /* device time: potential assembly and reductions      */
    int32_t launches;        /* kernels launched by this call                      */
    int32_t smem_row0;       /* FP32 pair kernel: first table row held in shared
                                memory (given, or chosen from the call's pairs);
                                -1 on the FP64 path                                */
    int32_t pair_threads;    /* the pair kernel's threads per CTA (0: not launched) */
} vdwdf_result;

/* Optional launch shape of the pair kernel (NULL = defaults / tuned).  Values
 * outside those listed are VDWDF_EINVAL; 256 or 1024 threads on a skewed cell
 * are VDWDF_EUNSUPPORTED (both before any device work). */
#define VDWDF_TUNE_AUTO (-1)  /* threads: vdwdf_energy_batched only -- the fastest
                                 candidate shape on the batch itself is used (the
                                 other fields are ignored) */
typedef struct {
    int32_t threads;      /* threads per CTA: 256, 384, 448, 512 or 1024 (0 = default:
                             FP32 E + v 448, or 384 on skewed cells; 512 otherwise);
                             skewed cells take 384, 448 or 512; VDWDF_TUNE_AUTO in
                             vdwdf_energy_batched                                    */
    int32_t items_per_sm; /* target work items per warp slot for load balance (0 = 256) */
    int32_t smem_rows;    /* FP32 path: table rows resident in shared memory
                             (0 = as many as fit, -1 = none)                          */
    int32_t smem_row0;    /* FP32 path: first resident table row (-1 = chosen on the
                             device from a sampled histogram of the table's D cell
                             over the call's pair evaluations: the start whose rows
                             hold the most; a NULL tuning chooses the same way;
                             problems under 16384 active points keep row 0)         */
} vdwdf_tuning;

/* --------------------------------------------------------------------- */
/* Kernel table (host, FP64)                                              */
/* --------------------------------------------------------------------- */

/* Build the table by double quadrature of Dion eq. (14) on the host in FP64
 * (section 2: "formula (14) ... requires a double integration"), OpenMP over
 * nodes.  Row D = 0, where eq. (14) diverges like -(2/pi) ln D, holds the
 * value at D = 0 of the even quadratic through rows 1 and 2.
 *   nD >= 4 nodes in D over [0, Dmax] (Dmax > 0); ndelta >= 4 nodes
 *   delta_l = l/ndelta.  quad_level: 0 = fast (~1e-6 of max|phi|),
 *   1 = standard (~1e-10), 2 = fine.  phi_nodes_out: NULL or host array of
 *   nD*ndelta doubles (D outer).  *out receives the handle.
 * Errors: VDWDF_EINVAL, VDWDF_EALLOC. */
int vdwdf_table_build(int nD, double Dmax, int ndelta, int quad_level,
                      double *phi_nodes_out, vdwdf_table **out);

/* Make a table from given node values (host, nD*ndelta doubles, D outer),
 * e.g. a saved table (section 5: the kernel file is loaded, not recomputed).
 * Same grid conventions and errors as vdwdf_table_build. */
int vdwdf_table_from_nodes(int nD, double Dmax, int ndelta, const double *phi_nodes,
                           vdwdf_table **out);

/* Copy a table's node values to host memory (nD*ndelta doubles). */
int vdwdf_table_nodes(const vdwdf_table *t, double *phi_nodes_out);

/* Query a table's grid. Any output pointer may be NULL. */
int vdwdf_table_info(const vdwdf_table *t, int *nD, double *Dmax, int *ndelta);

/* Release a table and its device copies (NULL is ignored). */
void vdwdf_table_free(vdwdf_table *t);

/* Evaluate the kernel as the pair sum uses it, on the device, at npts pairs:
 * inputs r (bohr), q_i, q_j (device FP64 arrays); outputs phi and
 * r dphi/dd1 (d1 = q_i r, d2 = q_j r).  precision as in vdwdf_energy.  For
 * checking the interpolation path in isolation. */
int vdwdf_kernel_eval(const vdwdf_table *t, int precision, int64_t npts,
                      const double *r_dev, const double *qi_dev, const double *qj_dev,
                      double *phi_dev, double *rdphi_dev, void *cuda_stream);

/* --------------------------------------------------------------------- */
/* q0 (Dion eqs. 11-12)                                                    */
/* --------------------------------------------------------------------- */

/* q0 = -(4 pi/3) [eps_c^LDA + eps_x^LDA (1 - (Zab/9) s^2)],
 * s = |grad n|/(2 k_F n), with eps_c^LDA of Perdew-Wang 1992, at every grid
 * point; points with n <= 0 give 0.  grad_dev: NULL (the library's gradient of
 * the kind grid->gradient names) or a [3][N] FP64 device array (Cartesian).
 * Outputs q0_dev [N] and, when not NULL, dq0dn_dev [N], dq0dg_dev [3][N].
 * n_cut is not used (reserved). Asynchronous. */
int vdwdf_q0(const vdwdf_grid *grid, const double *n_dev, const double *grad_dev,
             double n_cut, double *q0_dev, double *dq0dn_dev, double *dq0dg_dev,
             void *cuda_stream);

/* The library's gradient of n_dev ([N] FP64) of the kind grid->gradient names,
 * into grad_dev ([3][N] FP64, Cartesian components, caller-owned).  The
 * spectral kind allocates N0 + N1 + N2 doubles of stream-ordered scratch.
 * VDWDF_EINVAL for null pointers or a bad grid.  Asynchronous. */
int vdwdf_gradient(const vdwdf_grid *grid, const double *n_dev, double *grad_dev, void *cuda_stream);

/* --------------------------------------------------------------------- */
/* The double sum (paper section 2 eq. (2), section 3)                     */
/* --------------------------------------------------------------------- */

/* E_c^nl of the density n_dev ([N] FP64) on grid.  Points with n >= n_cut
 * take part; the self term i = j, L = 0 is n_i^2 phi(0,0).  Periodic axes add
 * all images L with |r_i - r_j + L| <= r_cut (required > 0 when any axis is
 * periodic); r_cut <= 0 means no cutoff for open cells.  grad_dev as in
 * vdwdf_q0.  A pair is inside the cutoff iff |r_i - r_j + L|^2 <= r_cut^2 (1 + 1e-12)
 * (distances equal to r_cut up to rounding count as inside, in both precisions).
 * Image shifts run over |m_a| <= M_a = ceil(r_cut |B_a|) + 1 along each
 * periodic axis a (B_a the reciprocal row, |B_a| = 1/L_a on a diagonal cell);
 * M_a above 64 (a cutoff more than about 63 cell lengths) returns VDWDF_EINVAL
 * before any device work.
 * precision: VDWDF_FP32 or VDWDF_FP64.  Synchronises the stream.
 * Errors: VDWDF_EINVAL, VDWDF_EUNSUPPORTED, VDWDF_ENOTABLE, VDWDF_ECUDA,
 * VDWDF_EALLOC, VDWDF_ETIMEOUT. */
int vdwdf_energy(const vdwdf_grid *grid, const double *n_dev, const double *grad_dev,
                 double n_cut, double r_cut, const vdwdf_table *table, int precision,
                 const vdwdf_tuning *tuning, vdwdf_result *out, void *cuda_stream);

/* E_c^nl and its potential v = (1/dV) dE/dn at every grid point (mask of
 * active points frozen), written to v_dev [N] FP64:
 *   v_m = dV [chi_m (A_m + U_m dq0/dn_m) - sum_axes D_h(U dq0/dgrad n)_m],
 *   A_i = sum_{j,L} n_j phi_ijL,  U_i = n_i sum_{j,L} n_j r dphi/dd1,
 * chi the active mask and D_h the library's gradient of the kind
 * grid->gradient names (so the gradient is always computed by the library
 * here; D_h is antisymmetric for both kinds, so its transpose is -D_h).  A_dev, U_dev: NULL or
 * [N] FP64 grid arrays that receive A and U (0 at inactive points).
 * Synchronises the stream. Errors as vdwdf_energy. */
int vdwdf_potential(const vdwdf_grid *grid, const double *n_dev, double n_cut, double r_cut,
                    const vdwdf_table *table, int precision, const vdwdf_tuning *tuning,
                    double *v_dev, double *A_dev, double *U_dev, vdwdf_result *out,
                    void *cuda_stream);

/* E_c^nl of ninst independent densities (grids[k], n_dev[k]), 1 <= ninst <=
 * 4096, in one persistent launch of the pair kernel per 24 instances (in
 * order: instances 0..23, 24..47, ...), recorded once into a CUDA graph and
 * replayed on later calls that would record the same graph: the same device,
 * pointers, shapes, cells, periodicity, gradient kind, cutoffs, precision,
 * tuning and table (binding curves, section 6.1).  Up to 8 recorded graphs are
 * kept (the least recently used is dropped first, with its scratch); freeing a
 * table drops the graphs that read it.  tuning->threads = VDWDF_TUNE_AUTO makes
 * the call time every candidate shape of vdwdf_autotune on this batch (the
 * whole pass, twice each, when the graph is first recorded) and record the
 * fastest; out->pair_threads reports it.  E_out:
 * host array of ninst doubles.  Synchronises the stream.  Errors as
 * vdwdf_energy. */
int vdwdf_energy_batched(int ninst, const vdwdf_grid *grids, const double *const *n_dev,
                         double n_cut, double r_cut, const vdwdf_table *table, int precision,
                         const vdwdf_tuning *tuning, double *E_out, vdwdf_result *out,
                         void *cuda_stream);

/* --------------------------------------------------------------------- */
/* Semilocal energies (paper section 2, eq. (3))                           */
/* --------------------------------------------------------------------- */

typedef struct {
    double Ex_lda;       /* LDA exchange, Hartree                                 */
    double Ec_lda;       /* LDA correlation (Perdew-Wang 1992)                   */
    double Ex_pbe;       /* PBE exchange                                          */
    double Ec_pbe;       /* PBE correlation                                       */
    double Ex_revpbe;    /* revPBE exchange                                       */
    int64_t n_points;    /* grid points with n > 0 (the others contribute 0)      */
    float ms;            /* device time of the call                               */
    int32_t launches;    /* kernels launched by the call                          */
} vdwdf_semilocal_result;

/* The semilocal terms that eq. (3) combines with E_c^nl.  Section 2 has JuNoLo
 * evaluate them from the density itself, because the DFT code may not report
 * them; E_x^revPBE is the optional replacement of E_x^PBE in eq. (3).
 * Spin-unpolarised, FP64, Hartree:
 *   eps_x^LDA = -3 k_F/(4 pi), k_F = (3 pi^2 n)^(1/3);
 *   GGA exchange eps_x^LDA F_x(s), F_x = 1 + kappa - kappa/(1 + mu s^2/kappa),
 *     s = |grad n|/(2 k_F n), mu = beta pi^2/3, kappa = 0.804 (PBE, Perdew,
 *     Burke and Ernzerhof 1996) or 1.245 (revPBE, Zhang and Yang 1998);
 *   eps_c^LDA: Perdew-Wang 1992; eps_c^PBE = eps_c^LDA + H with
 *     H = gamma ln[1 + (beta/gamma) t^2 (1 + A t^2)/(1 + A t^2 + A^2 t^4)],
 *     t = |grad n|/(2 k_s n), k_s = (4 k_F/pi)^(1/2),
 *     A = (beta/gamma)/(exp(-eps_c^LDA/gamma) - 1),
 *     beta = 0.06672455060314922, gamma = (1 - ln 2)/pi^2;
 *   E = dV sum of n eps over every grid point with n > 0 (no density cutoff).
 * grad_dev as in vdwdf_q0.  The sum is reproducible: fixed blocks, fixed order.
 * Synchronises the stream.
 * Errors: VDWDF_EINVAL, VDWDF_ECUDA, VDWDF_EALLOC. */
int vdwdf_semilocal(const vdwdf_grid *grid, const double *n_dev, const double *grad_dev,
                    vdwdf_semilocal_result *out, void *cuda_stream);

/* Exchange functional of eq. (3)'s bracket. */
#define VDWDF_X_PBE 0     /* E_x^PBE: the PBE exchange stays                        */
#define VDWDF_X_REVPBE 1  /* E_x^revPBE replaces it (the alternative after eq. 3)  */

/* Eq. (3): the total energy with the nonlocal correlation, from the total energy
 * of a PBE calculation, the semilocal terms of its density (vdwdf_semilocal)
 * and E_c^nl (vdwdf_energy or vdwdf_potential), all in Hartree:
 *   E_tot^NL = E_tot^DFT - E_x^PBE - E_c^PBE + (E_x + E_c^LDA + E_c^nl),
 * E_x = E_x^PBE or E_x^revPBE as `exchange` says.  Host arithmetic only.
 * Errors: VDWDF_EINVAL for a NULL pointer, another exchange value or a
 * non-finite input (E_out is then untouched). */
int vdwdf_total_energy_nl(double E_tot_dft, const vdwdf_semilocal_result *semi, double E_c_nl, int exchange,
                          double *E_out);

/* --------------------------------------------------------------------- */
/* Far field past the cutoff (section 7: image sums sped up by the kernel's */
/* asymptotic form, named there as future work)                           */
/* --------------------------------------------------------------------- */

typedef struct {
    double T;            /* the far field past r_cut, Hartree: E(r_cut -> inf) reads E + T */
    int64_t n_active;    /* grid points with n >= n_cut                          */
    int32_t nodes;       /* nodes of the quadrature in ln s                       */
    int32_t planes;      /* groups the sums run over: grid planes along the open axis
                            (two periodic axes), grid lines along the periodic axis
                            that hold an active point (one), 1 (three)            */
    float ms;            /* device time of the call                               */
    int32_t launches;    /* kernels launched by the call                          */
} vdwdf_tail_result;

/* The pair sum's far field beyond r_cut, from eq. (17) alone (sections 3 and
 * 6.2 repeat the cell until the energy converges; section 7 proposes the
 * asymptote for the far images).  Reading: every pair beyond r_cut takes
 *   phi17 = -C / (q_i^2 q_j^2 (q_i^2 + q_j^2) r^6),  C = 12 (4 pi / 9)^3,
 * and the lattice images beyond r_cut are replaced by the lattice continuum:
 *   T = 1/2 dV^2 sum_{i,j active} n_i n_j (-C / (q_i^2 q_j^2 (q_i^2 + q_j^2))) K_ij,
 *   K_ij = (2 pi / A) / (4 max(r_cut, |z_ij|)^4)   two periodic axes (A the
 *          area of the periodic plane, z_ij the separation normal to it),
 *   K    = (4 pi / V) / (3 r_cut^3)                 three periodic axes,
 *   K_ij = (2 / |a|) I(rho_ij, x0),  I(rho, x0) = int_{x0}^inf dx / (rho^2 + x^2)^3,
 *          x0 = sqrt(max(0, r_cut^2 - rho_ij^2))    one periodic axis a (rho_ij
 *          the distance of r_i - r_j from the direction of a).
 * E(r_cut) + T estimates the fully converged periodic energy; the estimate
 * is exact for the continuum of images and tends to the lattice sum of eq.
 * (17) as r_cut grows.  The library evaluates T in FP64, with
 * 1/(a + b) = int exp(-(a + b) s) ds by the trapezoidal rule in ln s
 * (relative error below 2e-13; below 3e-12 for the potential's
 * 1/(a + b)^2), from per-plane sums over the grid (per-line sums with one
 * periodic axis, and K between lines with an active point, as a table over
 * their index differences: at most 65536 such lines).
 * v_dev: NULL, or an [N] FP64 device array that receives T's potential,
 * v_T = dT/dn / dV with the active mask frozen, in the pair sum's adjoint form
 * (vdwdf_potential) with
 *   A_m = -C sum_j n_j f(u_m, u_j) K_mj,
 *   U_m = -2 C n_m q0_m sum_j n_j (df/du_m)(u_m, u_j) K_mj,
 * f(a, b) = 1/(a b (a + b)), u = q0^2; so v + v_T is the potential of E + T.
 * grid as in vdwdf_energy with one, two or three periodic axes; grad_dev
 * as in vdwdf_q0, and NULL when v_dev is given (the potential needs the
 * library's own gradient); r_cut > 0.  Synchronises the stream.
 * Errors: VDWDF_EINVAL (bad argument, r_cut <= 0, grad_dev with v_dev, a
 * non-finite T from a non-finite density; v_dev is then unspecified),
 * VDWDF_EUNSUPPORTED (no periodic axis, a q0 range needing more than 4096
 * nodes, or more than 65536 active lines), VDWDF_ECUDA, VDWDF_EALLOC. */
int vdwdf_far_tail(const vdwdf_grid *grid, const double *n_dev, const double *grad_dev, double n_cut,
                   double r_cut, double *v_dev, vdwdf_tail_result *out, void *cuda_stream);

/* --------------------------------------------------------------------- */
/* Voxel-averaged diagonal (the "phi0" step of the paper's Appendix A      */
/* output; the paper does not describe its method)                        */
/* --------------------------------------------------------------------- */

typedef struct {
    double E_diag_voxel;   /* 1/2 dV^2 sum_i n_i^2 phi0(q0_i), Hartree            */
    double E_diag_table;   /* the self term the pair sum uses,
                              1/2 dV^2 sum_i n_i^2 phi(0, 0) (table row 0)        */
    double q0_min, q0_max; /* over the points with n >= n_cut                      */
    int64_t n_active;      /* points with n >= n_cut                              */
    int32_t nphi0;         /* q points of the phi0 table                           */
    float ms;              /* device time of the call                              */
    int32_t launches;      /* kernels launched by the call                         */
} vdwdf_diag_result;

/* phi0(q) for the voxel spanned by the rows of voxel[9] (host; v_a = M_a / N_a,
 * bohr) at nq values q_dev (device FP64) into phi0_dev (device FP64):
 *   phi0(q) = int_{[-1,1]^3} prod_a (1 - |t_a|) phi_0(q |sum_a t_a v_a|) d^3t,
 * the kernel at delta = 0 averaged over pairs of points of one voxel (r - r' =
 * sum_a t_a v_a, t_a the difference of two uniform variables).  phi_0(D) is the
 * pair sum's kernel at delta = 0 for D >= D_1 = Dmax/(nD - 1); below, where
 * eq. 14 diverges like -(2/pi) ln D and the table's row 0 is softened, it is
 * -(2/pi) ln D + psi0 + c2 D^2 with psi = phi + (2/pi) ln D fitted at the nodes
 * D_1, D_2 (psi0 = (4 psi1 - psi2)/3, c2 = (psi1 - psi0)/D_1^2).  The eight
 * sign octants times a 48-node graded Gauss rule per axis (agreement with a
 * finer rule: ~1e-5 relative); integrand in FP32, sums in FP64.
 * Synchronises the stream.  Errors: VDWDF_EINVAL, VDWDF_ENOTABLE, VDWDF_ECUDA,
 * VDWDF_EALLOC. */
int vdwdf_phi0_eval(const vdwdf_table *table, const double *voxel, int64_t nq, const double *q_dev,
                    double *phi0_dev, void *cuda_stream);

/* The voxel-averaged self term of the density (reading of the paper's
 * undocumented diagonal step, printed there as E_DIAG_nlc): with n and q0
 * constant over voxel i, the i = j, L = 0 term of eq. (1) is
 *   1/2 dV^2 n_i^2 phi0(q0_i)
 * (phi0 as in vdwdf_phi0_eval for the grid's voxel), summed over the points
 * with n >= n_cut.  phi0 comes from a table of nphi0 (0: 100, the paper's
 * nphi0) log-spaced q over the active q0 range, by 4-point Lagrange
 * interpolation in ln q.  E_c^nl with this diagonal is
 *   E (vdwdf_energy) - E_diag_table + E_diag_voxel.
 * grad_dev as in vdwdf_q0.  Sums in a fixed order (reproducible).
 * Synchronises the stream.  Errors: VDWDF_EINVAL, VDWDF_ENOTABLE,
 * VDWDF_ECUDA, VDWDF_EALLOC. */
int vdwdf_diag_voxel(const vdwdf_grid *grid, const double *n_dev, const double *grad_dev, double n_cut,
                     const vdwdf_table *table, int nphi0, vdwdf_diag_result *out, void *cuda_stream);

/* The change of v = (1/dV) dE/dn when the table self term is replaced by the
 * voxel diagonal of vdwdf_diag_voxel, written to dv_dev [N] FP64 (device):
 * with the active mask frozen,
 *   dv_m = dV [chi_m (A_m + U_m dq0/dn_m) + sum_a (G_a^T w_a)_m],
 *   A_m = n_m (phi0(q0_m) - phi(0, 0)),  U_m = 1/2 n_m^2 phi0'(q0_m),
 *   w_a = chi U dq0/dgrad_a n,
 * the same form as the pair sum's adjoint (phi0' from the derivative of the
 * interpolant in ln q).  v (vdwdf_potential) + dv is the potential of
 * E - E_diag_table + E_diag_voxel.  The library's gradient of the kind
 * grid->gradient names (the adjoint needs it).  out as in vdwdf_diag_voxel.  Synchronises the stream.
 * Errors: as vdwdf_diag_voxel; VDWDF_EINVAL for a NULL dv_dev. */
int vdwdf_diag_voxel_potential(const vdwdf_grid *grid, const double *n_dev, double n_cut,
                               const vdwdf_table *table, int nphi0, double *dv_dev, vdwdf_diag_result *out,
                               void *cuda_stream);

/* vdwdf_energy that allocates nothing.  The paper has no counterpart: JuNoLo
 * allocates its arrays once per run.  This entry point is for callers that
 * cannot allocate device memory while they run, for example:
 *  - a host code that has reserved the device memory for its own arrays;
 *  - code that must not wait on the whole device: cudaMalloc and cudaFree
 *    can wait for work on every stream, while this call waits only for its
 *    own stream (it blocks the calling thread until that is done);
 *  - a loop of many small grids (binding curves, geometry steps) where one
 *    allocation per call costs more than the pair sum.
 * Same arguments, results and errors as vdwdf_energy, with library default
 * tuning.  Limits and conditions:
 *  - Size: at most 65536 grid points and 65536 4x4x4 bricks.  Larger grids
 *    return VDWDF_EUNSUPPORTED before any device work.
 *  - Scratch: all of a call's scratch lives in one 8 MiB static device array
 *    of the library.  It is module data, one copy per device, present as
 *    soon as the library's module is loaded on that device.  The call makes
 *    no cudaMalloc/cudaFree and no call into an allocating library; the
 *    Morton order of the bricks is staged through static host arrays.
 *  - Set-up: the array's device address is taken with cudaGetSymbolAddress
 *    once per device, on the first call on that device.  That lookup may
 *    load the module, so make the first call on each device before any
 *    stream capture.
 *  - Table: the table must already be resident on the current device, that
 *    is, used there once by vdwdf_energy, vdwdf_potential,
 *    vdwdf_energy_batched or vdwdf_kernel_eval (npts >= 1), because making it
 *    resident allocates.  Otherwise the call returns VDWDF_ENOTABLE.
 *  - Overlap: calls overlapping in time would race on the one scratch array.
 *    The library therefore holds a process-wide lock for the whole call, and
 *    the call synchronises its stream before every return that follows its
 *    first device work, errors included, so none of its work is still queued
 *    when the next call starts.  Other code must not write the array.
 *  - Zeroing: everything that must start at zero (the counters and the
 *    work-queue head) is cleared by the call itself on the stream.  Every
 *    per-item energy partial is written before it is read.
 *  - Timings: ms_prep, ms_pairs and ms_post are 0 (no CUDA events are
 *    created). */
int vdwdf_energy_noalloc(const vdwdf_grid *grid, const double *n_dev, const double *grad_dev,
                         double n_cut, double r_cut, const vdwdf_table *table, int precision,
                         vdwdf_result *out, void *cuda_stream);

/* Time candidate launch shapes of the pair kernel on this problem (energy
 * path, on every k-th work item: about 16 items per warp slot spread over the
 * whole pair triangle) and write the fastest to *best: the one with the most
 * pair evaluations per millisecond of its second timed run.  The shape
 * suits vdwdf_energy and the batched path; vdwdf_potential's default shape
 * (448 threads, 384 on skewed cells) was the fastest for the potential pass
 * on every workload measured. */
int vdwdf_autotune(const vdwdf_grid *grid, const double *n_dev, double n_cut, double r_cut,
                   const vdwdf_table *table, int precision, vdwdf_tuning *best,
                   void *cuda_stream);

/* --------------------------------------------------------------------- */
/* Misc                                                                    */
/* --------------------------------------------------------------------- */

/* Static string naming a status code. */
const char *vdwdf_strerror(int status);

/* VDWDF_VERSION of the built library. */
int vdwdf_version(void);

/* Number of kernels this library has launched in this process. */
int64_t vdwdf_launch_count(void);

/* Arithmetic rate of the current device, measured: the denominators of the
 * pair kernels' rooflines.  The pair sum (section 2, eq. (2)) is a
 * gather-and-interpolate on the CUDA cores, so its ceiling is a rate of lane
 * operations (one fused multiply-add of one lane counts as one), not a tensor
 * or memory rate.
 *  kind:           VDWDF_RATE_FP32 (FP32 FMA), VDWDF_RATE_FP32X2 (packed
 *                  FP32x2 FMA, two lane operations per instruction) or
 *                  VDWDF_RATE_FP64 (FP64 FMA).
 *  target_ms:      duration of the timed launch, 1..1000 ms.
 *  lane_ops_per_s: out (host), lane operations per second over the whole
 *                  device.
 *  ms_out:         out (host, may be NULL), the timed launch's duration.
 * Every SM runs as many 512-thread blocks as fit at once, each thread 8
 * independent FMA chains, so the launch measures the pipe's throughput.  One
 * calibration launch sizes the timed one, which is sized again (at most three
 * times) while it lasts under half of target_ms; all are timed with CUDA
 * events on the stream, which the call synchronises: 2 to 4 launches.  A
 * 16-byte device scratch is allocated on the stream and freed before return.
 * Errors: VDWDF_EINVAL for an unknown kind, a NULL lane_ops_per_s or a
 * target_ms outside 1..1000 (checked before any CUDA call); VDWDF_EALLOC;
 * VDWDF_ECUDA. */
#define VDWDF_RATE_FP32 0
#define VDWDF_RATE_FP32X2 1
#define VDWDF_RATE_FP64 2
int vdwdf_lane_rate(int kind, double target_ms, double *lane_ops_per_s, double *ms_out, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* VDWDF_H */
