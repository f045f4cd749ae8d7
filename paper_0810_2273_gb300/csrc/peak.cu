// Arithmetic rates of the GPU the library runs on: FP32 fused multiply-adds, the
// same as packed FP32x2 instructions, and FP64 fused multiply-adds.  They are
// the measured denominators of the pair kernels' ALU rooflines (the pair sum is
// a gather-and-interpolate on the CUDA cores, so its peak is a lane rate, not a
// tensor or memory rate).
//
// Every thread runs kChains independent recurrences a <- a m + c, one fused
// multiply-add per lane and step (two per packed FP32x2 instruction), with m just
// below 1 so that the values stay finite.  The step loop is unrolled 16 times, so
// its counter and branch take about 2 % of the issue slots.  kChains chains per thread and full
// occupancy keep far more independent operations in flight per scheduler than
// the pipes' latency needs, so the launch measures the pipe's throughput.  The
// host times one calibration launch, then a launch sized to the requested
// duration (sized again while it comes out under half of it, at most three
// times), with CUDA events on the caller's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace vdwdf {

namespace {

constexpr int kChains = 8;
constexpr int kRateThreads = 512;

// Keeps the chains live: the store happens only if a value went non-finite or
// huge, which a recurrence with 0 < m < 1 and a small start never does.
template <typename T>
__device__ __forceinline__ void keep(T s, T *out) {
    if (!(s == s) || s > T(1e30)) *out = s;
}

__global__ void __launch_bounds__(kRateThreads) k_rate_f32(int steps, float *out) {
    float a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = 1e-3f * static_cast<float>(threadIdx.x + c);
    const float m = 0.99999f, k = 1e-6f;
#pragma unroll 16
    for (int s = 0; s < steps; ++s) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = __fmaf_rn(a[c], m, k);
    }
    float t = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) t += a[c];
    keep(t, out);
}

__global__ void __launch_bounds__(kRateThreads) k_rate_f32x2(int steps, float *out) {
    float2 a[kChains / 2];
#pragma unroll
    for (int c = 0; c < kChains / 2; ++c)
        a[c] = make_float2(1e-3f * static_cast<float>(threadIdx.x + c), 2e-3f * static_cast<float>(threadIdx.x + c));
    const float2 m = make_float2(0.99999f, 0.99999f), k = make_float2(1e-6f, 1e-6f);
#pragma unroll 16
    for (int s = 0; s < steps; ++s) {
#pragma unroll
        for (int c = 0; c < kChains / 2; ++c) a[c] = __ffma2_rn(a[c], m, k);
    }
    float t = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains / 2; ++c) t += a[c].x + a[c].y;
    keep(t, out);
}

__global__ void __launch_bounds__(kRateThreads) k_rate_f64(int steps, double *out) {
    double a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = 1e-3 * static_cast<double>(threadIdx.x + c);
    const double m = 0.99999, k = 1e-6;
#pragma unroll 16
    for (int s = 0; s < steps; ++s) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = __fma_rn(a[c], m, k);
    }
    double t = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) t += a[c];
    keep(t, out);
}

// Resident blocks of the kind's kernel per SM (all launched blocks run in one wave).
int blocks_per_sm(int kind, int *nb) {
    if (kind == VDWDF_RATE_FP32)
        VDWDF_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, k_rate_f32, kRateThreads, 0));
    else if (kind == VDWDF_RATE_FP32X2)
        VDWDF_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, k_rate_f32x2, kRateThreads, 0));
    else
        VDWDF_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, k_rate_f64, kRateThreads, 0));
    return VDWDF_OK;
}

int launch_rate(int kind, int blocks, int steps, void *out, cudaStream_t st) {
    if (kind == VDWDF_RATE_FP32)
        k_rate_f32<<<blocks, kRateThreads, 0, st>>>(steps, static_cast<float *>(out));
    else if (kind == VDWDF_RATE_FP32X2)
        k_rate_f32x2<<<blocks, kRateThreads, 0, st>>>(steps, static_cast<float *>(out));
    else
        k_rate_f64<<<blocks, kRateThreads, 0, st>>>(steps, static_cast<double *>(out));
    count_launches(1);
    VDWDF_CUDA_TRY(cudaGetLastError());
    return VDWDF_OK;
}

}  // namespace

}  // namespace vdwdf

extern "C" int vdwdf_lane_rate(int kind, double target_ms, double *lane_ops_per_s, double *ms_out,
                               void *cuda_stream) {
    using namespace vdwdf;
    if (kind != VDWDF_RATE_FP32 && kind != VDWDF_RATE_FP32X2 && kind != VDWDF_RATE_FP64) return VDWDF_EINVAL;
    if (!lane_ops_per_s || !(target_ms >= 1.0 && target_ms <= 1000.0)) return VDWDF_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0, sms = 0, per_sm = 0;
    VDWDF_CUDA_TRY(cudaGetDevice(&dev));
    VDWDF_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int rc = blocks_per_sm(kind, &per_sm);
    if (rc) return rc;
    if (sms < 1 || per_sm < 1) return VDWDF_ECUDA;
    const int blocks = sms * per_sm;
    void *out = nullptr;
    if (cudaMallocAsync(&out, 16, st) != cudaSuccess) return VDWDF_EALLOC;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double ms = 0.0;
    long long steps = 256;
    auto body = [&]() -> int {
        VDWDF_CUDA_TRY(cudaEventCreate(&e0));
        VDWDF_CUDA_TRY(cudaEventCreate(&e1));
        // calibration: launch overhead makes each estimate of the rate low, so a
        // sized launch lasts at most about target_ms; one that came out shorter
        // than half of it (an overhead-dominated estimate) is sized again, up to
        // three times
        for (int pass = 0; pass < 4; ++pass) {
            VDWDF_CUDA_TRY(cudaEventRecord(e0, st));
            int r = launch_rate(kind, blocks, static_cast<int>(steps), out, st);
            if (r) return r;
            VDWDF_CUDA_TRY(cudaEventRecord(e1, st));
            VDWDF_CUDA_TRY(cudaEventSynchronize(e1));
            float f = 0.0f;
            VDWDF_CUDA_TRY(cudaEventElapsedTime(&f, e0, e1));
            ms = f;
            if (pass > 0 && (ms >= 0.5 * target_ms || steps >= (1LL << 28))) break;
            const double scale = target_ms / std::max(ms, 1e-3);
            steps = std::clamp(static_cast<long long>(static_cast<double>(steps) * scale), 256LL, 1LL << 28);
            steps &= ~15LL;  // whole unrolled blocks of the step loop
        }
        return VDWDF_OK;
    };
    rc = body();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFreeAsync(out, st);
    if (rc == VDWDF_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = VDWDF_ECUDA;
    if (rc) return rc;
    if (!(ms > 0.0)) return VDWDF_ECUDA;
    const double ops = static_cast<double>(blocks) * kRateThreads * kChains * static_cast<double>(steps);
    *lane_ops_per_s = ops / (ms * 1e-3);
    if (ms_out) *ms_out = ms;
    return VDWDF_OK;
}
