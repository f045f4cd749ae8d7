// The spectral (FFT) gradient, FP64: the paper's FFTW option for the density
// gradient (section 3), on any cell.
//
// Along grid axis a the band-limited derivative d/du_a (u_a the fractional
// coordinate, period 1) multiplies the discrete Fourier transform by 2 pi i m_a,
// m_a in (-N/2, N/2), and maps the Nyquist frequency of an even axis to zero
// (the real part of the inverse transform drops it).  As an operator on the N
// samples of a line it is the circulant matrix of the periodic sinc interpolant,
//     (d/du f)_l = sum_k c_{(l-k) mod N} f_k,   c_0 = 0,
//     c_j = pi (-1)^j cot(pi j/N)   (N even),   pi (-1)^j / sin(pi j/N)   (N odd),
// which these kernels apply directly, one tile of whole lines per block in shared
// memory: O(N_a) work per point and axis, no transform.  The gradient is then
// grad f = sum_a (d/du_a f) B_a with the reciprocal rows B_a (B_a . M_b = delta_ab).
// The matrix is antisymmetric, so the transpose the potential needs is minus the
// same operator.
#include <cuda_runtime.h>

#include "common.cuh"

namespace vdwdf {

namespace {

constexpr double kPiD = 3.14159265358979323846;

// c_j for the three axes, one after the other (N0 + N1 + N2 values).
__global__ void k_spec_coef(int n0, int n1, int n2, double *__restrict__ c) {
    const int total = n0 + n1 + n2;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const int N = t < n0 ? n0 : (t < n0 + n1 ? n1 : n2);
        const int j = t < n0 ? t : (t < n0 + n1 ? t - n0 : t - n0 - n1);
        double v = 0.0;
        if (j > 0) {
            double s, co;
            sincospi(static_cast<double>(j) / N, &s, &co);
            const double sg = (j & 1) ? -kPiD : kPiD;
            v = (N % 2 == 0) ? sg * co / s : sg / s;
        }
        c[t] = v;
    }
}

// One axis of the derivative on an array viewed as [P][L][Q] (the axis in the
// middle): block b takes line group p = b / nqc and the TQ columns q0 = (b % nqc) TQ
// onwards, stages them with the L coefficients in shared memory, and writes (or,
// with acc, adds) out[p][l][q] = sum_j c_j f[p][(l - j) mod L][q].
__global__ void k_spec_axis(int L, long long Q, int TQ, int nqc, const double *__restrict__ c,
                            const double *__restrict__ f, double *__restrict__ out, int acc) {
    extern __shared__ double sm[];
    double *sc = sm;           // L coefficients
    double *sf = sm + L;       // [L][TQ] tile
    const long long p = blockIdx.x / nqc;
    const long long q0 = static_cast<long long>(blockIdx.x % nqc) * TQ;
    const int tq = static_cast<int>(min(static_cast<long long>(TQ), Q - q0));
    for (int j = threadIdx.x; j < L; j += blockDim.x) sc[j] = c[j];
    for (int e = threadIdx.x; e < L * tq; e += blockDim.x) {
        const int l = e / tq, t = e % tq;
        sf[l * TQ + t] = f[(p * L + l) * Q + q0 + t];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < L * tq; e += blockDim.x) {
        const int l = e / tq, t = e % tq;
        double s = 0.0;
        for (int j = 1; j <= l; ++j) s += sc[j] * sf[(l - j) * TQ + t];
        for (int j = l + 1; j < L; ++j) s += sc[j] * sf[(l - j + L) * TQ + t];
        const long long o = (p * L + l) * Q + q0 + t;
        out[o] = acc ? out[o] + s : s;
    }
}

// In place at every point: the three axis derivatives d_a (planes of N) become the
// Cartesian components g_c = sum_a B[3a + c] d_a.
__global__ void k_to_cart(long long N, const Recip R, double *__restrict__ d) {
    for (long long m = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; m < N;
         m += static_cast<long long>(gridDim.x) * blockDim.x) {
        const double d0 = d[m], d1 = d[N + m], d2 = d[2 * N + m];
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) d[cc * N + m] = R.B[cc] * d0 + R.B[3 + cc] * d1 + R.B[6 + cc] * d2;
    }
}

// The potential's weights along the grid axes: W_a = sum_c B[3a + c] w_c with the
// Cartesian w_c = U dq0/dg_c at active points (slot >= 0) and 0 elsewhere.
__global__ void k_spec_w(long long N, const Recip R, const int *__restrict__ slot, const double *__restrict__ U,
                         const double *__restrict__ qg, double *__restrict__ W) {
    for (long long m = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; m < N;
         m += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int s = slot[m];
        const double u = s >= 0 ? U[s] : 0.0;
        const double w0 = u * qg[m], w1 = u * qg[N + m], w2 = u * qg[2 * N + m];
#pragma unroll
        for (int a = 0; a < 3; ++a) W[a * N + m] = R.B[3 * a] * w0 + R.B[3 * a + 1] * w1 + R.B[3 * a + 2] * w2;
    }
}

int grid_blocks(long long N) {
    long long nb = (N + 255) / 256;
    return static_cast<int>(nb > (1 << 20) ? (1 << 20) : (nb < 1 ? 1 : nb));
}

constexpr size_t kSpecSmem = 200 * 1024;

// d/du_a of f (N values) into out (N values), or added to it with acc.
int spec_axis(const int dims[3], int a, const double *coef, const double *f, double *out, bool acc,
              cudaStream_t st) {
    const int L = dims[a];
    long long Q = 1;
    for (int b = a + 1; b < 3; ++b) Q *= dims[b];
    long long P = 1;
    for (int b = 0; b < a; ++b) P *= dims[b];
    int TQ = static_cast<int>(Q < 32 ? Q : 32);
    while (TQ > 1 && static_cast<size_t>(L) * (TQ + 1) * sizeof(double) > kSpecSmem) TQ >>= 1;
    const size_t smem = static_cast<size_t>(L) * (TQ + 1) * sizeof(double);
    if (smem > kSpecSmem) return VDWDF_EUNSUPPORTED;
    const long long nqc = (Q + TQ - 1) / TQ;
    if (P * nqc > 0x7FFFFFFFLL) return VDWDF_EUNSUPPORTED;
    if (smem > 48 * 1024)
        VDWDF_CUDA_TRY(cudaFuncSetAttribute(k_spec_axis, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            static_cast<int>(smem)));
    const int off = a == 0 ? 0 : (a == 1 ? dims[0] : dims[0] + dims[1]);
    k_spec_axis<<<static_cast<int>(P * nqc), 256, smem, st>>>(L, Q, TQ, static_cast<int>(nqc), coef + off, f, out,
                                                                acc ? 1 : 0);
    count_launches(1);
    VDWDF_CUDA_TRY(cudaGetLastError());
    return VDWDF_OK;
}

int spec_coef(const int dims[3], double *coef, cudaStream_t st) {
    const int total = dims[0] + dims[1] + dims[2];
    k_spec_coef<<<(total + 255) / 256, 256, 0, st>>>(dims[0], dims[1], dims[2], coef);
    count_launches(1);
    VDWDF_CUDA_TRY(cudaGetLastError());
    return VDWDF_OK;
}

}  // namespace

int launch_gradient_spectral(const int dims[3], const Recip &R, const double *n, double *grad, double *coef,
                             cudaStream_t st) {
    const long long N = static_cast<long long>(dims[0]) * dims[1] * dims[2];
    int rc = spec_coef(dims, coef, st);
    for (int a = 0; a < 3 && rc == VDWDF_OK; ++a) rc = spec_axis(dims, a, coef, n, grad + a * N, false, st);
    if (rc) return rc;
    k_to_cart<<<grid_blocks(N), 256, 0, st>>>(N, R, grad);
    count_launches(1);
    VDWDF_CUDA_TRY(cudaGetLastError());
    return VDWDF_OK;
}

int launch_div_spectral(const int dims[3], const Recip &R, const int *slot, const double *U, const double *qg,
                        double *W, double *div, double *coef, cudaStream_t st) {
    const long long N = static_cast<long long>(dims[0]) * dims[1] * dims[2];
    int rc = spec_coef(dims, coef, st);
    if (rc) return rc;
    k_spec_w<<<grid_blocks(N), 256, 0, st>>>(N, R, slot, U, qg, W);
    count_launches(1);
    VDWDF_CUDA_TRY(cudaGetLastError());
    for (int a = 0; a < 3 && rc == VDWDF_OK; ++a) rc = spec_axis(dims, a, coef, W + a * N, div, a > 0, st);
    return rc;
}

}  // namespace vdwdf
