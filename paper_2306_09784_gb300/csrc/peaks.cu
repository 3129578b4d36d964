// sar_alu_peaks: throughput microbenchmarks of the two pipes that bound the
// backprojection (FP32 FMA lanes and the MUFU special-function unit), so that
// its ALU roofline can be checked against measured rates instead of only the
// nominal lane counts x clock.
//
// Each kernel runs independent dependency chains (8 per thread, 4 CTAs of 256
// threads per SM) long enough (~1-3 ms) for launch costs to vanish, and
// writes one value per thread so that no chain can be removed.  Rates are
// counted per lane: one FFMA = 1 lane-op, one packed FFMA2 = 2, one
// sin.approx = 1 MUFU op.
#include "sar_internal.h"

namespace {

constexpr int kPeakThreads = 256;
constexpr int kPeakCtasPerSm = 4;
constexpr int kChains = 8;

__global__ void __launch_bounds__(kPeakThreads) fma_peak_kernel(float *out, int iters, float a, float b) {
    float x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = (float)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) x[k] = fmaf(x[k], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kPeakThreads) ffma2_peak_kernel(float *out, int iters, float a, float b) {
    float2 x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = make_float2((float)threadIdx.x, (float)k);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) x[k] = __ffma2_rn(x[k], a2, b2);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k].x + x[k].y;
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kPeakThreads) mufu_peak_kernel(float *out, int iters, float a, float b) {
    float x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = a * (float)(threadIdx.x + k) + b;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) {
            float y;
            asm("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x[k]));
            x[k] = y;
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Best of three timed launches (after one warm-up) of `k`, in seconds.
template <typename K>
int time_kernel(K k, int grid, float *out, int iters, cudaStream_t s, double *seconds) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return SAR_ECUDA;
    }
    int rc = SAR_OK;
    double best = 1e30;
    for (int rep = 0; rep < 4 && rc == SAR_OK; ++rep) {
        cudaEventRecord(e0, s);
        k<<<grid, kPeakThreads, 0, s>>>(out, iters, 0.999f, 0.001f);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            rc = SAR_ECUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) best = ms < best ? ms : best;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (cudaGetLastError() != cudaSuccess) rc = SAR_ECUDA;
    *seconds = best * 1e-3;
    return rc;
}

}  // namespace

extern "C" int sar_alu_peaks(double *fma_lane_ops_per_s, double *ffma2_lane_ops_per_s, double *mufu_ops_per_s) {
    if (!fma_lane_ops_per_s || !ffma2_lane_ops_per_s || !mufu_ops_per_s) return SAR_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        return SAR_ECUDA;
    const int grid = sms * kPeakCtasPerSm;
    const long long threads = (long long)grid * kPeakThreads;
    float *out = nullptr;
    if (cudaMalloc((void **)&out, sizeof(float) * (size_t)threads) != cudaSuccess) {
        cudaGetLastError();
        return SAR_ENOMEM;
    }
    cudaStream_t s = nullptr;
    int rc = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess ? SAR_OK : SAR_ECUDA;
    const int it_fma = 1 << 15, it_mufu = 1 << 12;
    double t = 0.0;
    if (rc == SAR_OK) rc = time_kernel(fma_peak_kernel, grid, out, it_fma, s, &t);
    if (rc == SAR_OK) *fma_lane_ops_per_s = (double)threads * kChains * it_fma / t;
    if (rc == SAR_OK) rc = time_kernel(ffma2_peak_kernel, grid, out, it_fma, s, &t);
    if (rc == SAR_OK) *ffma2_lane_ops_per_s = 2.0 * (double)threads * kChains * it_fma / t;
    if (rc == SAR_OK) rc = time_kernel(mufu_peak_kernel, grid, out, it_mufu, s, &t);
    if (rc == SAR_OK) *mufu_ops_per_s = (double)threads * kChains * it_mufu / t;
    if (s) cudaStreamDestroy(s);
    cudaFree(out);
    return rc;
}
